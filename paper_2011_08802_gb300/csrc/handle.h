// Internal state of a problem handle and helpers shared by the host-side
// translation units of libpfm (api.cu: single-problem drivers; batch.cu:
// the batched engine). Not part of the public ABI.
#pragma once

#include <chrono>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/pfm.h"
#include "common.cuh"

namespace pfm {

struct Level {
  Grid g{};
  int64_t nn = 0, ne = 0, nblk = 0;
  double* U = nullptr;
  double* Un = nullptr;
  dmask_t* mask = nullptr;
  double* H64 = nullptr;
  float* H32 = nullptr;
  float* H32lo = nullptr;  // finest level, mixed mode: H64 - H32 rounded to FP32
  __half* H16 = nullptr;   // binary16 copy of s H32 for the preconditioner (optional)
  float h16_scale = 0.f;   // s, 0 while the copy is not current
  double* D64 = nullptr;
  float* D32 = nullptr;
  float *x32 = nullptr, *b32 = nullptr, *y32 = nullptr, *r32 = nullptr, *d32 = nullptr;
  double *x64 = nullptr, *b64 = nullptr, *y64 = nullptr, *r64 = nullptr, *d64 = nullptr;
  double lam = 0.0;  // estimate of lambda_max(D^-1 J) for the Chebyshev smoother
  double* Kc64 = nullptr;  // contact Hessians at the top-face Gauss points (6 per point)
  float* Kc32 = nullptr;
};

template <typename T> struct LvVec;
template <> struct LvVec<float> {
  static float*& x(Level& l) { return l.x32; }
  static float*& b(Level& l) { return l.b32; }
  static float*& y(Level& l) { return l.y32; }
  static float*& r(Level& l) { return l.r32; }
  static float*& d(Level& l) { return l.d32; }
  static float*& D(Level& l) { return l.D32; }
  static float*& H(Level& l) { return l.H32; }
  static float*& Kc(Level& l) { return l.Kc32; }
};
template <> struct LvVec<double> {
  static double*& x(Level& l) { return l.x64; }
  static double*& b(Level& l) { return l.b64; }
  static double*& y(Level& l) { return l.y64; }
  static double*& r(Level& l) { return l.r64; }
  static double*& d(Level& l) { return l.d64; }
  static double*& D(Level& l) { return l.D64; }
  static double*& H(Level& l) { return l.H64; }
  static double*& Kc(Level& l) { return l.Kc64; }
};

constexpr int MAX_COARSE_DOFS = 5000;
constexpr int MAX_RESTART = 64;

inline double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace pfm

struct pfm_handle {
  pfm_params params{};
  pfm::DevParams dp{};
  std::vector<pfm::Level> L;
  cudaStream_t stream = 0;
  std::string err;
  bool have_state = false;
  bool have_dirval = false;
  bool linearized = false;
  pfm_precision lin_prec = PFM_F64;
  double* dirval = nullptr;
  double* energy_dev = nullptr;
  int* flag_dev = nullptr;
  double* diag_part = nullptr;  // per-plane partial sums of the diagnostics
  bool contact_on = false;      // penalty contact with a rigid sphere (pfm_set_contact)
  pfm::ContactParams contact{};
  double* load_dev = nullptr;
  // solver work (finest level, FP64)
  double* R = nullptr;
  double* dU = nullptr;
  double* wv = nullptr;
  double* rv = nullptr;
  double* zd = nullptr;
  double* ir_r = nullptr;  // iterative refinement: outer residual and inner correction
  double* ir_d = nullptr;
  double* partial = nullptr;
  double* hdev = nullptr;
  // Krylov basis
  int kry_m = 0;
  pfm_precision kry_prec = PFM_F64;
  double* V = nullptr;
  void* Z = nullptr;
  // coarse dense operator [K | I] reduced by Gauss-Jordan, its inverse, work
  double* Kaug = nullptr;
  double* Kinv = nullptr;
  unsigned long long* gj_keys = nullptr;
  int* gj_used = nullptr;
  int* gj_piv = nullptr;
  int nc_dofs = 0;
  // per-(element, node) diagonal-block contributions (linearisation scratch)
  void* bd_scratch = nullptr;
  size_t bd_bytes = 0;
  // staging for the host-buffer entry point, and its slab pipeline
  void* stage_in = nullptr;
  void* stage_out = nullptr;
#ifndef PFM_PIPE_SLABS
#define PFM_PIPE_SLABS 8
#endif
  static constexpr int PIPE_SLABS = PFM_PIPE_SLABS;
  cudaStream_t pipe_in = nullptr, pipe_out = nullptr;
  cudaEvent_t pipe_ev_in[PIPE_SLABS] = {}, pipe_ev_done[PIPE_SLABS] = {};
  cudaEvent_t pipe_ev_start = nullptr;
  int power_its = 10;     // Lanczos steps of the smoother's eigenvalue estimate
  double* lz = nullptr;   // their alpha and beta^2 (device), and one norm
  int lz_cap = 0;
  bool outer_df = true;  // outer operator of the mixed solve in double-float arithmetic
  bool lin_df = false;   // FP64-class linearisation in double-float instead of FP64 arithmetic
  bool res_df = false;   // residual point physics in double-float instead of FP64 arithmetic
  bool pre_h16 = false;  // FP32 preconditioner reads binary16 Hessian copies
  bool det = false;      // atomic-free element kernels (pfm_set_deterministic or opts.deterministic)
  unsigned* amax_dev = nullptr;  // one word for the store's max |entry|
  // pinned host slots for Hessenberg columns and scalars
  double* hpin = nullptr;
  // captured V-cycle (valid until the next linearisation)
  bool use_graphs = false;
  cudaGraphExec_t vgraph = nullptr;
  int vgraph_prec = -1;
  struct { int nu_pre, nu_post, type; double omega, lo, hi; int gamma; double growth; bool det; } vgraph_cfg{};
  // device timing of hot phases (pairs of events per timed launch)
  bool prof = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev[PFM_PROF_COUNT];
  int64_t prof_n[PFM_PROF_COUNT] = {0};
  double prof_ms[PFM_PROF_COUNT] = {0};

  // A non-finite result may come from a staged tangent application whose
  // bounded wait for its copies gave up (it writes NaN into its output); such
  // events are reported as PFM_ERR_TIMEOUT.
  pfm_status fail(pfm_status s, const std::string& m) {
    if (s == PFM_ERR_NONFINITE) {
      const int n = pfm::take_wait_timeouts();
      if (n > 0) {
        err = m + " (" + std::to_string(n) + " bounded waits of the staged tangent application gave up)";
        return PFM_ERR_TIMEOUT;
      }
    }
    err = m;
    return s;
  }
};


struct pfm_batch;
namespace pfm {
struct BatchEngine;  // batched multigrid/FGMRES engine (batch.cu)
void batch_engine_free(BatchEngine* e);
bool batch_engine_supports(const pfm_solve_opts& o, const pfm_batch* b);
pfm_status batch_engine_newton(pfm_batch* b, const pfm_solve_opts& o, double* const* U_inout,
                               pfm_solve_report* reports);
}  // namespace pfm

struct pfm_batch {
  std::vector<pfm_handle*> hs;
  std::vector<cudaStream_t> streams;
  std::string err;
  int mode = 0;  // 0: batched engine where supported; 1: per-problem lockstep driver
  pfm::BatchEngine* engine = nullptr;
  pfm_status fail(pfm_status st, const std::string& m) {
    err = m;
    return st;
  }
};

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return h->fail(e_ == cudaErrorMemoryAllocation ? PFM_ERR_OOM : PFM_ERR_CUDA,            \
                     std::string(#call) + ": " + cudaGetErrorString(e_));                     \
  } while (0)

#define CKL()                                                                                 \
  do {                                                                                        \
    cudaError_t e_ = cudaGetLastError();                                                      \
    if (e_ != cudaSuccess)                                                                    \
      return h->fail(PFM_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_));  \
  } while (0)

// CKL with the name of the step that launched the kernels in the message
#define CKL_AT(what)                                                                                   \
  do {                                                                                                 \
    cudaError_t e_ = cudaGetLastError();                                                               \
    if (e_ != cudaSuccess)                                                                             \
      return h->fail(PFM_ERR_CUDA, std::string("kernel launch (") + (what) + "): " + cudaGetErrorString(e_)); \
  } while (0)

#define TRY(expr)                     \
  do {                                \
    pfm_status s_ = (expr);           \
    if (s_ != PFM_OK) return s_;      \
  } while (0)

namespace pfm {

template <typename T>
pfm_status dalloc(pfm_handle* h, T** p, size_t count) {
  if (*p) return PFM_OK;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (count > 0 ? count : 1));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return h->fail(PFM_ERR_OOM, std::string("cudaMalloc of ") + std::to_string(sizeof(T) * count) +
                                    " bytes failed: " + cudaGetErrorString(e));
  }
  return PFM_OK;
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

inline int64_t ndof(const Level& l) { return int64_t(NF) * l.nn; }

}  // namespace pfm
