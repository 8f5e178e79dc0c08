// Microstructure diagnostics of Sec. 5.3 on the nodal state: the violation
// index I_v = sum_{i=0}^{N} |<eta_i>_-| of the constraints eta_i >= 0, the
// diffuseness index I_d = 1 - sum_{i=0}^{N} eta_i^4 and the composite
// parameter eta* = eta_3 - eta_1, with eta_0 = 1 - sum_k eta_k (Sec. 3.1);
// and, per horizontal plane z = k h_z, the mean and the maximum of I_v and of
// I_d over its nodes (the paper plots both against z).
//
// HBM-bound: N FP64 loads per node (48 B for N = 6) plus the optional per-node outputs.
// Grid (chunks, planes): a block reduces one contiguous chunk of one plane in
// a fixed order (strided per thread, then a fixed shuffle tree), and a second
// kernel sums the chunks of each plane in order, so results are bitwise
// reproducible for a given grid.
#include <algorithm>

#include "common.cuh"

namespace pfm {

constexpr int DIAG_THREADS = 256;

__device__ inline void diag_node(const double* __restrict__ U, int64_t nn, int64_t n, double& Iv, double& Id,
                                 double& es) {
  double eta[NPH];
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    eta[k + 1] = U[int64_t(3 + k) * nn + n];
    s += eta[k + 1];
  }
  eta[0] = 1.0 - s;
  Iv = 0.0;
  double q = 0.0;
#pragma unroll
  for (int i = 0; i < NPH; ++i) {
    Iv += eta[i] < 0.0 ? -eta[i] : 0.0;
    const double e2 = eta[i] * eta[i];
    q += e2 * e2;
  }
  Id = 1.0 - q;
  es = eta[3] - eta[1];
}

// partial[(plane * chunks + chunk) * 4 + {0,1,2,3}] = (sum I_v, max I_v, sum I_d, max I_d)
__global__ void __launch_bounds__(DIAG_THREADS) k_diag(int64_t nn, int per_plane, int chunks, const double* __restrict__ U,
                                                       double* __restrict__ Iv_out, double* __restrict__ Id_out,
                                                       double* __restrict__ es_out, double* __restrict__ partial) {
  const int chunk = blockIdx.x, plane = blockIdx.y;
  const int len = (per_plane + chunks - 1) / chunks;
  const int lo = chunk * len;
  const int hi = min(per_plane, lo + len);
  double sv = 0.0, mv = 0.0, sd = 0.0, md = -1e300;
  for (int i = lo + threadIdx.x; i < hi; i += DIAG_THREADS) {
    const int64_t n = int64_t(plane) * per_plane + i;
    double Iv, Id, es;
    diag_node(U, nn, n, Iv, Id, es);
    if (Iv_out) Iv_out[n] = Iv;
    if (Id_out) Id_out[n] = Id;
    if (es_out) es_out[n] = es;
    sv += Iv;
    mv = fmax(mv, Iv);
    sd += Id;
    md = fmax(md, Id);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sv += __shfl_down_sync(0xffffffffu, sv, o);
    mv = fmax(mv, __shfl_down_sync(0xffffffffu, mv, o));
    sd += __shfl_down_sync(0xffffffffu, sd, o);
    md = fmax(md, __shfl_down_sync(0xffffffffu, md, o));
  }
  __shared__ double sh[DIAG_THREADS / 32][4];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sh[w][0] = sv;
    sh[w][1] = mv;
    sh[w][2] = sd;
    sh[w][3] = md;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < DIAG_THREADS / 32; ++k) {
      sv += sh[k][0];
      mv = fmax(mv, sh[k][1]);
      sd += sh[k][2];
      md = fmax(md, sh[k][3]);
    }
    double* p = partial + (int64_t(plane) * chunks + chunk) * 4;
    p[0] = sv;
    p[1] = mv;
    p[2] = sd;
    p[3] = md;
  }
}

__global__ void k_diag_planes(int nplanes, int per_plane, int chunks, const double* __restrict__ partial,
                              double* __restrict__ stats) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nplanes) return;
  double sv = 0.0, mv = 0.0, sd = 0.0, md = -1e300;
  for (int c = 0; c < chunks; ++c) {
    const double* p = partial + (int64_t(k) * chunks + c) * 4;
    sv += p[0];
    mv = fmax(mv, p[1]);
    sd += p[2];
    md = fmax(md, p[3]);
  }
  stats[4 * k + 0] = sv / per_plane;
  stats[4 * k + 1] = mv;
  stats[4 * k + 2] = sd / per_plane;
  stats[4 * k + 3] = md;
}

int diag_chunks(const Grid& g) {
  const int nplanes = g.nz + 1;
  const int per_plane = (g.nx + 1) * (g.ny + 1);
  int chunks = (4 * 152 + nplanes - 1) / nplanes;  // about four blocks per SM in all
  chunks = std::min(chunks, std::max(1, per_plane / DIAG_THREADS));
  return std::max(1, std::min(chunks, DIAG_MAX_CHUNKS));
}

void launch_diagnostics(const Grid& g, const double* U, double* Iv, double* Id, double* es, double* partial,
                        double* stats, cudaStream_t s) {
  const int nplanes = g.nz + 1;
  const int per_plane = (g.nx + 1) * (g.ny + 1);
  const int chunks = diag_chunks(g);
  k_diag<<<dim3(chunks, nplanes), DIAG_THREADS, 0, s>>>(g.nn(), per_plane, chunks, U, Iv, Id, es, partial);
  count_launches(1);
  if (stats) {
    k_diag_planes<<<(nplanes + 127) / 128, 128, 0, s>>>(nplanes, per_plane, chunks, partial, stats);
    count_launches(1);
  }
}

}  // namespace pfm
