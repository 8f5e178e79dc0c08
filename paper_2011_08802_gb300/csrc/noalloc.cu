// Residual and potential of the phase-field model for callers that cannot
// allocate device memory.
//
// pfm_residual needs a handle, and pfm_create allocates the handle's level
// hierarchy, Hessian stores and solver vectors with cudaMalloc. Some callers
// cannot do that: code running inside a framework that owns all device memory
// through its own allocator (a custom op of an array framework, a plugin of a
// larger solver), code that must not pay allocation latency or fragment a
// memory pool in the middle of a time step, or a device that is already full.
// pfm_residual_noalloc serves them: the caller passes the inputs and the
// output, and the only working memory is the fixed file-scope scratch array
// below, which every GPU that loads the library holds until the process exits.
#include <mutex>
#include <string>

#include "common.cuh"
#include "params.h"

namespace pfm {
namespace {

// Scratch: the per-node Dirichlet bit masks built from the caller's byte mask
// (NOALLOC_MAX_NODES entries of 2 bytes), then the energy accumulator and the
// invalid-mask flag.
constexpr int64_t NOALLOC_MAX_NODES = int64_t(1) << 22;  // 4,194,304 nodes (e.g. 160^3 hexes)
constexpr size_t MASK_BYTES = size_t(NOALLOC_MAX_NODES) * sizeof(dmask_t);
constexpr size_t ENERGY_OFF = MASK_BYTES;                 // double
constexpr size_t FLAG_OFF = ENERGY_OFF + 256;             // int
constexpr size_t SCRATCH_BYTES = FLAG_OFF + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_dev[MAX_DEVICES] = {nullptr};
// one message per host thread, so that two threads that fail at once do not
// write the same string
thread_local std::string g_noalloc_error;

// Device address of the scratch array on the current device. The name of a
// __device__ variable in host code is only a host-side stand-in, so the
// address is looked up once per device with that device current.
pfm_status scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
    g_noalloc_error = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return PFM_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      g_noalloc_error = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return PFM_ERR_CUDA;
    }
    g_scratch_dev[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_dev[dev];
  return PFM_OK;
}

}  // namespace
}  // namespace pfm

using namespace pfm;

extern "C" {

pfm_status pfm_residual_noalloc(const pfm_mesh_desc* mesh, const pfm_params* params, const uint8_t* mask_dev,
                                const double* U_dev, const double* Un_dev, double* R_dev, double* energy_host,
                                void* stream) {
  if (!mesh || !params || !mask_dev || !U_dev || !Un_dev || !R_dev) {
    g_noalloc_error = "null argument";
    return PFM_ERR_INVALID_ARG;
  }
  if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1 || !(mesh->Lx > 0) || !(mesh->Ly > 0) || !(mesh->Lz > 0) ||
      !(params->tau > 0) || params->hencky < 0 || params->hencky > 3) {
    g_noalloc_error = "invalid mesh size, box length, tau or Hencky mode";
    return PFM_ERR_INVALID_ARG;
  }
  Grid g{mesh->nx, mesh->ny, mesh->nz, mesh->Lx / mesh->nx, mesh->Ly / mesh->ny, mesh->Lz / mesh->nz};
  if (g.nn() > NOALLOC_MAX_NODES) {
    g_noalloc_error = "mesh has " + std::to_string(g.nn()) + " nodes; pfm_residual_noalloc supports at most " +
                      std::to_string(NOALLOC_MAX_NODES);
    return PFM_ERR_INVALID_ARG;
  }
  unsigned char* scratch = nullptr;
  pfm_status st = scratch_for_current_device(&scratch);
  if (st != PFM_OK) return st;
  dmask_t* mask = reinterpret_cast<dmask_t*>(scratch);
  double* energy = reinterpret_cast<double*>(scratch + ENERGY_OFF);
  int* flag = reinterpret_cast<int*>(scratch + FLAG_OFF);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DevParams dp;
  make_dev_params(*params, dp);
  const int64_t n = int64_t(NF) * g.nn();
  // the scratch keeps the previous call's contents: clear what accumulates
  cudaError_t e = cudaMemsetAsync(energy, 0, sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(R_dev, 0, sizeof(double) * n, s);
  if (e != cudaSuccess) {
    g_noalloc_error = std::string("cudaMemsetAsync: ") + cudaGetErrorString(e);
    return PFM_ERR_CUDA;
  }
  launch_build_mask(g.nn(), mask_dev, mask, flag, s);
  launch_residual(g, dp, U_dev, Un_dev, mask, R_dev, energy, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_noalloc_error = std::string("kernel launch: ") + cudaGetErrorString(e);
    return PFM_ERR_CUDA;
  }
  double host_vals[1] = {0.0};
  int bad = 0;
  e = cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_vals, energy, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    g_noalloc_error = std::string("cudaMemcpyAsync/cudaStreamSynchronize: ") + cudaGetErrorString(e);
    return PFM_ERR_CUDA;
  }
  if (bad) {
    g_noalloc_error = "only displacement DOFs (fields 0..2) may be prescribed";
    return PFM_ERR_INVALID_ARG;
  }
  if (energy_host) *energy_host = host_vals[0];
  return PFM_OK;
}

const char* pfm_noalloc_last_error(void) { return g_noalloc_error.c_str(); }

}  // extern "C"
