// Batched engine: many independent problems of uneven size advance through
// one Newton step together, and every phase is ONE launch over all of them
// (the batching configuration of the Newton-step solve, Sec. 3.4 applied to
// a batch of problems). Work items of a phase are numbered across the batch
// (element blocks for element kernels, (problem, node) for nodal kernels); an
// element kernel finds the problem of a block by binary search over the
// per-problem block offsets, a nodal kernel takes the problem from
// blockIdx.y. Per-problem FGMRES scalars (Hessenberg matrix, Givens rotations,
// convergence flags) live on the device, so one FGMRES iteration of the whole
// batch is a fixed launch sequence that is captured once per inner index j as
// a CUDA graph and replayed; the host reads one flag word per iteration.
//
// Supported: the mixed-precision solve (FP32 V-cycle with Chebyshev
// smoothing inside FP64 FGMRES, double-float outer operator). Other options
// use the per-problem lockstep driver of api.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "fe_device.cuh"
#include "handle.h"
#include "mg_device.cuh"

namespace pfm {

constexpr int BMAXM = MAX_RESTART;  // FGMRES restart length bound
constexpr int BCH = 16;             // chunks per problem of the segmented reductions
constexpr int BT = 256;             // threads of the nodal kernels

// One multigrid level of one problem inside a launch set.
struct BLev {
  Grid g;
  JParams<float> jp;
  const dmask_t* mask;
  const float* H;
  const float* D;
  float* vec[5];   // x, b, y, r, d
  int64_t blk0;    // first element block of this level in the set's numbering
  float inv_theta, inv_delta;  // Chebyshev coefficients 1/theta, 1/delta
  int pad[2];
};
enum { VX = 0, VB = 1, VY = 2, VR = 3, VD = 4 };

// Transfer between level l (fine) and l+1 (coarse) of one problem.
struct BTr {
  Grid f, c;
  const dmask_t* mf;
  const dmask_t* mc;
  const float* rf;  // fine residual (restriction input)
  float* bc;        // coarse right-hand side (restriction output)
  const float* xc;  // coarse correction (prolongation input)
  float* xf;        // fine iterate (prolongation output)
};

// Dense coarse solve x = Kinv b of one problem.
struct BCo {
  int n;
  const double* Kinv;
  const float* b;
  float* x;
};

// Linearisation of one level of one problem.
struct BLin {
  Grid g;
  const DevParams* P;
  const double* U;
  const double* Un;
  double* H64;
  float* H32;
  float* H32lo;
  int64_t blk0;
};

// State injection level l-1 -> l of one problem.
struct BInj {
  Grid f, c;
  const double* Uf;
  double* Uc;
  const double* Unf;
  double* Unc;
};

// Diagonal blocks of one level of one problem.
struct BBd {
  Grid g;
  JParams<float> jp;
  const float* H;
  float* D;
  const dmask_t* mask;
  int64_t e0;  // first element of this level in the set's numbering
};

// Gauss-Jordan inverse of one problem's dense coarse operator.
struct BGj {
  double* M;
  int n;
  unsigned long long* keys;
  int* used;
  int* piv;
  double* Ainv;
};

// Outer (finest-level, FP64) data of one problem.
struct BOut {
  Grid g;
  int64_t n;  // 9 * nodes
  DfConst dk;
  JParams<double> jp64;
  const float* Hhi;
  const float* Hlo;
  const double* H64;
  const dmask_t* mask;
  double* V;     // (m+1) basis vectors
  float* Z;      // m preconditioned vectors
  double* w;     // work vector (J z, then the orthogonalised vector)
  double* x;     // solution (Newton correction)
  double* b;     // right-hand side -R (R on entry)
  double* r;     // restart residual
  double* U;     // Newton iterate
  float* b32;    // finest level V-cycle input
  float* x32;    // finest level V-cycle output
  int64_t blk0;
};

// Per-problem FGMRES scalars (device).
struct BFgm {
  double beta0, beta, tol, relres, hinv;
  int total, active, converged, status;
  int upd, restart, kdone, pad;
  double H[(BMAXM + 1) * BMAXM];
  double cs[BMAXM], sn[BMAXM], g[BMAXM + 1], y[BMAXM];
};
enum { BF_OK = 0, BF_NONFINITE = 1, BF_BREAKDOWN = 2, BF_NOTCONV = 3 };

namespace {

inline unsigned gdiv(int64_t a, int64_t b) { return unsigned(std::max<int64_t>(1, (a + b - 1) / b)); }

// index of the entry of a set whose [blk0, next blk0) range holds blk
template <typename S>
__device__ __forceinline__ int find_entry(const S* __restrict__ set, int ns, int64_t blk) {
  int lo = 0, hi = ns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (set[mid].blk0 <= blk) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// FP32 V-cycle kernels

// y += J v over all element blocks of the set; v = vec[vsel], y = vec[ysel].
// Each warp caches the descriptor of its current problem in shared memory.
__global__ void __launch_bounds__(256) k_b_japply(const BLev* __restrict__ S, int ns, int64_t nblk, int vsel,
                                                  int ysel) {
  __shared__ BLev cache[8];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t wg = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  int cur = -1;
  for (int64_t blk = wg; blk < nblk; blk += nw) {
    const int p = find_entry(S, ns, blk);
    if (p != cur) {
      __syncwarp();
      const int* src = reinterpret_cast<const int*>(S + p);
      int* dst = reinterpret_cast<int*>(cache + wid);
      for (int i = lane; i < int(sizeof(BLev) / 4); i += 32) dst[i] = src[i];
      __syncwarp();
      cur = p;
    }
    const BLev& L = cache[wid];
    if (blk - L.blk0 < L.g.nblk())
      japply_block<float>(L.g, L.jp, L.H, L.mask, L.vec[vsel], L.vec[ysel], blk - L.blk0, lane);
  }
}

// y = v at Dirichlet DOFs, 0 elsewhere (identity rows of J).
__global__ void k_b_init(const BLev* __restrict__ S, int vsel, int ysel) {
  const BLev& L = S[blockIdx.y];
  const int64_t nn = L.g.nn();
  const float* v = L.vec[vsel];
  float* y = L.vec[ysel];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < NF * nn; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = ((L.mask[i % nn] >> int(i / nn)) & 1) ? v[i] : 0.f;
}

__global__ void k_b_cheb_first(const BLev* __restrict__ S, int srcsel, bool copy_r, bool zero_x) {
  const BLev& L = S[blockIdx.y];
  const int64_t nn = L.g.nn();
  for (int64_t node = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; node < nn; node += int64_t(gridDim.x) * blockDim.x)
    cheb_first_node<float>(nn, L.D, L.vec[srcsel], L.inv_theta, copy_r, zero_x, L.vec[VR], L.vec[VD], L.vec[VX], node);
}

__global__ void k_b_cheb_step(const BLev* __restrict__ S, float a, float c) {
  const BLev& L = S[blockIdx.y];
  const int64_t nn = L.g.nn();
  const float cp = c * L.inv_delta;
  for (int64_t node = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; node < nn; node += int64_t(gridDim.x) * blockDim.x)
    cheb_step_node<float>(nn, L.D, L.vec[VY], a, cp, L.vec[VR], L.vec[VD], L.vec[VX], node);
}

// out = vec[asel] - vec[bsel]
__global__ void k_b_sub(const BLev* __restrict__ S, int asel, int bsel, int osel) {
  const BLev& L = S[blockIdx.y];
  const int64_t n = NF * L.g.nn();
  const float* a = L.vec[asel];
  const float* b = L.vec[bsel];
  float* o = L.vec[osel];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    o[i] = a[i] - b[i];
}

__global__ void k_b_restrict(const BTr* __restrict__ T) {
  const BTr& t = T[blockIdx.y];
  const int64_t nnc = t.c.nn();
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < nnc; idx += int64_t(gridDim.x) * blockDim.x)
    restrict_node<float>(t.f, t.c, t.rf, t.mc, t.bc, idx);
}

__global__ void k_b_prolong(const BTr* __restrict__ T) {
  const BTr& t = T[blockIdx.y];
  const int64_t nnf = t.f.nn();
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < nnf; idx += int64_t(gridDim.x) * blockDim.x)
    prolong_node<float>(t.f, t.c, t.xc, t.mf, t.xf, idx);
}

// x = Kinv b, one warp per row; blockIdx.y = problem.
__global__ void k_b_coarse_solve(const BCo* __restrict__ C) {
  const BCo& c = C[blockIdx.y];
  const int lane = threadIdx.x & 31;
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < c.n; row += (gridDim.x * blockDim.x) >> 5) {
    const double* Ar = c.Kinv + int64_t(row) * c.n;
    double s = 0.0;
    for (int k = lane; k < c.n; k += 32) s += Ar[k] * double(c.b[k]);
    for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    if (lane == 0) c.x[row] = float(s);
  }
}

// ---------------------------------------------------------------------------
// Linearisation kernels

__global__ void k_b_inject(const BInj* __restrict__ I) {
  const BInj& t = I[blockIdx.y];
  const int64_t nnc = t.c.nn();
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < nnc; idx += int64_t(gridDim.x) * blockDim.x) {
    inject_node(t.f, t.c, t.Uf, t.Uc, idx);
    inject_node(t.f, t.c, t.Unf, t.Unc, idx);
  }
}

template <typename TC>
__global__ void __launch_bounds__(128) k_b_linearize(const BLin* __restrict__ S, int ns, int64_t nblk) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t blk = tid >> 5;
  if (blk >= nblk) return;
  const BLin& L = S[find_entry(S, ns, blk)];
  linearize_lane<TC>(L.g, *L.P, L.U, L.Un, L.H64, L.H32, L.H32lo, blk - L.blk0, int(tid & 31));
}

__global__ void k_b_zero_D(const BBd* __restrict__ S) {
  const BBd& L = S[blockIdx.y];
  const int64_t n = 81 * L.g.nn();
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    L.D[i] = 0.f;
}

// (element, local node) threads numbered across the set: e0 = first element
template <typename S>
__device__ __forceinline__ int find_elem(const S* __restrict__ set, int ns, int64_t e) {
  int lo = 0, hi = ns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (set[mid].e0 <= e) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(128) k_b_blockdiag(const BBd* __restrict__ S, int ns, int64_t ne) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t e = tid >> 3;
  if (e >= ne) return;
  const BBd& L = S[find_elem(S, ns, e)];
  blockdiag_elem_node<float>(L.g, L.jp, L.H, L.D, e - L.e0, int(tid & 7));
}

__global__ void k_b_block_invert(const BBd* __restrict__ S, int* singular) {
  const BBd& L = S[blockIdx.y];
  const int64_t nn = L.g.nn();
  for (int64_t node = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; node < nn; node += int64_t(gridDim.x) * blockDim.x)
    block_invert_node<float>(nn, L.mask, L.D, singular, node);
}

// power iteration: x = start vector
__global__ void k_b_power_init(const BLev* __restrict__ S) {
  const BLev& L = S[blockIdx.y];
  const int64_t nn = L.g.nn();
  float* x = L.vec[VX];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < NF * nn; i += int64_t(gridDim.x) * blockDim.x)
    x[i] = float(power_init_value(i, nn, L.mask));
}

// r = D^-1 y (one point-block Jacobi step from zero)
__global__ void k_b_dinv(const BLev* __restrict__ S) {
  const BLev& L = S[blockIdx.y];
  const int64_t nn = L.g.nn();
  const float* y = L.vec[VY];
  float* r = L.vec[VR];
  for (int64_t node = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; node < nn; node += int64_t(gridDim.x) * blockDim.x) {
    float yv[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) yv[f] = y[f * nn + node];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      float s = 0.f;
#pragma unroll
      for (int c = 0; c < NF; ++c) s += L.D[(f * 9 + c) * nn + node] * yv[c];
      r[f * nn + node] = s;
    }
  }
}

// partial[(entry * BCH + chunk)] = sum over the chunk of vec[sel]^2 (FP64 accumulation)
__global__ void __launch_bounds__(BT) k_b_norm2_32(const BLev* __restrict__ S, int sel, double* __restrict__ partial) {
  const BLev& L = S[blockIdx.y];
  const int64_t n = NF * L.g.nn();
  const float* a = L.vec[sel];
  double acc = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    acc += double(a[i]) * double(a[i]);
  __shared__ double red[BT / 32];
  for (int m = 16; m > 0; m >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < BT / 32; ++q) s += red[q];
    partial[int64_t(blockIdx.y) * gridDim.x + blockIdx.x] = s;
  }
}

// out[entry] = sum of the entry's chunks (fixed order)
__global__ void k_b_reduce_chunks(int ns, int chunks, const double* __restrict__ partial, double* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ns) return;
  double s = 0.0;
  for (int c = 0; c < chunks; ++c) s += partial[int64_t(e) * chunks + c];
  out[e] = s;
}

// x = r / sqrt(dot[entry])  (power iteration normalisation)
__global__ void k_b_normalise(const BLev* __restrict__ S, int src, const double* __restrict__ dot) {
  const BLev& L = S[blockIdx.y];
  const int64_t n = NF * L.g.nn();
  const double d = dot[blockIdx.y];
  const float s = d > 0.0 ? float(1.0 / sqrt(d)) : 0.f;
  const float* a = L.vec[src];
  float* x = L.vec[VX];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i] = a[i] * s;
}

// Gauss-Jordan over the batch: blockIdx.y = problem
__global__ void k_b_gj_first_key(const BGj* __restrict__ G) {
  const BGj& q = G[blockIdx.y];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < q.n; i += gridDim.x * blockDim.x)
    atomicMax(&q.keys[0], pivot_key(q.M[int64_t(i) * 2 * q.n], i));
}

__global__ void __launch_bounds__(256) k_b_gj_step(const BGj* __restrict__ G, int k, int* singular) {
  const BGj& q = G[blockIdx.y];
  if (k >= q.n) return;
  gj_step_row(q.M, q.n, 2 * q.n, k, q.keys, q.used, q.piv, singular, int(blockIdx.x), blockIdx.x == 0);
}

__global__ void k_b_gj_extract(const BGj* __restrict__ G) {
  const BGj& q = G[blockIdx.y];
  const int k = blockIdx.x;
  if (k >= q.n) return;
  const int p = q.piv[k];
  const double inv = 1.0 / q.M[int64_t(p) * 2 * q.n + k];
  for (int c = threadIdx.x; c < q.n; c += blockDim.x) q.Ainv[int64_t(k) * q.n + c] = q.M[int64_t(p) * 2 * q.n + q.n + c] * inv;
}

// ---------------------------------------------------------------------------
// Outer FGMRES kernels (FP64); every kernel skips problems that are not active

__global__ void k_b_cast_in(const BOut* __restrict__ O, const BFgm* __restrict__ F, int j) {
  const int p = blockIdx.y;
  if (!F[p].active) return;
  const BOut& o = O[p];
  const double* v = o.V + int64_t(j) * o.n;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < o.n; i += int64_t(gridDim.x) * blockDim.x)
    o.b32[i] = float(v[i]);
}

// Z_j = x32 (the V-cycle output) and w = Z_j at Dirichlet DOFs, 0 elsewhere
__global__ void k_b_store_z(const BOut* __restrict__ O, const BFgm* __restrict__ F, int j) {
  const int p = blockIdx.y;
  if (!F[p].active) return;
  const BOut& o = O[p];
  const int64_t nn = o.g.nn();
  float* z = o.Z + int64_t(j) * o.n;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < o.n; i += int64_t(gridDim.x) * blockDim.x) {
    const float v = o.x32[i];
    z[i] = v;
    o.w[i] = ((o.mask[i % nn] >> int(i / nn)) & 1) ? double(v) : 0.0;
  }
}

// w += J Z_j in double-float arithmetic over all element blocks
__global__ void __launch_bounds__(256) k_b_japply_df(const BOut* __restrict__ O, const BFgm* __restrict__ F, int np,
                                                     int64_t nblk, int j) {
  const int lane = threadIdx.x & 31;
  const int64_t wg = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t blk = wg; blk < nblk; blk += nw) {
    const int p = find_entry(O, np, blk);
    if (!F[p].active) continue;
    const BOut& o = O[p];
    const int64_t b = blk - o.blk0;
    if (b < o.g.nblk()) japply_df_block(o.g, o.dk, o.Hhi, o.Hlo, o.mask, o.Z + int64_t(j) * o.n, o.w, b, lane);
  }
}

// w += J x (FP64 kernel; restart residual)
__global__ void __launch_bounds__(256) k_b_japply64(const BOut* __restrict__ O, const BFgm* __restrict__ F, int np,
                                                    int64_t nblk) {
  const int lane = threadIdx.x & 31;
  const int64_t wg = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t blk = wg; blk < nblk; blk += nw) {
    const int p = find_entry(O, np, blk);
    if (!F[p].restart) continue;
    const BOut& o = O[p];
    const int64_t b = blk - o.blk0;
    if (b < o.g.nblk()) japply_block<double>(o.g, o.jp64, o.H64, o.mask, o.x, o.w, b, lane);
  }
}

// partial[(p * BCH + chunk) * stride + jj] = chunk sum of V_{j0+jj} . w (jj < cnt); with
// self_dot the single product is w . w
constexpr int BMDOT = 8;
__global__ void __launch_bounds__(BT) k_b_mdot(const BOut* __restrict__ O, const BFgm* __restrict__ F, int j0,
                                               int cnt, bool self_dot, double* __restrict__ partial, int stride) {
  const int p = blockIdx.y;
  if (!F[p].active && !F[p].restart) return;
  const BOut& o = O[p];
  double acc[BMDOT];
#pragma unroll
  for (int jj = 0; jj < BMDOT; ++jj) acc[jj] = 0.0;
  const double* src = self_dot ? (F[p].restart ? o.r : o.w) : o.w;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < o.n; i += int64_t(gridDim.x) * blockDim.x) {
    const double wi = src[i];
    if (self_dot) {
      acc[0] += wi * wi;
    } else {
#pragma unroll
      for (int jj = 0; jj < BMDOT; ++jj)
        if (jj < cnt) acc[jj] += o.V[int64_t(j0 + jj) * o.n + i] * wi;
    }
  }
  __shared__ double red[BT / 32][BMDOT];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int jj = 0; jj < BMDOT; ++jj) {
    double v = acc[jj];
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    if (lane == 0) red[wid][jj] = v;
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double s = 0.0;
    for (int q = 0; q < BT / 32; ++q) s += red[q][threadIdx.x];
    partial[(int64_t(p) * BCH + blockIdx.x) * stride + j0 + threadIdx.x] = s;
  }
}

// out[p * stride + jj] = sum over chunks, jj < k (fixed order); blockIdx.y = problem
__global__ void k_b_mdot_final(const BFgm* __restrict__ F, int k, const double* __restrict__ partial, int stride,
                               double* __restrict__ out) {
  const int p = blockIdx.y;
  if (!F[p].active && !F[p].restart) return;
  const int jj = threadIdx.x;
  if (jj >= k) return;
  double s = 0.0;
  for (int c = 0; c < BCH; ++c) s += partial[(int64_t(p) * BCH + c) * stride + jj];
  out[int64_t(p) * stride + jj] = s;
}

// w -= sum_{jj<k} h[p][jj] V_jj
__global__ void k_b_maxpy(const BOut* __restrict__ O, const BFgm* __restrict__ F, int k, const double* __restrict__ h,
                          int stride) {
  const int p = blockIdx.y;
  if (!F[p].active) return;
  const BOut& o = O[p];
  const double* hp = h + int64_t(p) * stride;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < o.n; i += int64_t(gridDim.x) * blockDim.x) {
    double s = o.w[i];
    for (int jj = 0; jj < k; ++jj) s -= hp[jj] * o.V[int64_t(jj) * o.n + i];
    o.w[i] = s;
  }
}

// Hessenberg column j of every active problem from the two Gram-Schmidt
// passes and ||w||^2, Givens rotations, residual estimate, and the decision:
// continue (hinv = 1/h_{j+1,j}), or finish the cycle (y = R^-1 g, upd = 1;
// restart = 1 if neither converged nor out of iterations).
__global__ void k_b_givens(BFgm* __restrict__ F, int np, int j, int m, int max_lin_it, const double* __restrict__ h1,
                           const double* __restrict__ h2, const double* __restrict__ hn, int stride) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  BFgm& s = F[p];
  s.upd = 0;
  if (!s.active) return;
  s.total += 1;
  const double hnorm = sqrt(hn[int64_t(p) * stride]);
  if (!isfinite(hnorm)) {
    s.active = 0;
    s.status = BF_NONFINITE;
    return;
  }
  for (int i = 0; i <= j; ++i) s.H[i * BMAXM + j] = h1[int64_t(p) * stride + i] + h2[int64_t(p) * stride + i];
  s.H[(j + 1) * BMAXM + j] = hnorm;
  for (int i = 0; i < j; ++i) {
    const double a = s.H[i * BMAXM + j], bb = s.H[(i + 1) * BMAXM + j];
    s.H[i * BMAXM + j] = s.cs[i] * a + s.sn[i] * bb;
    s.H[(i + 1) * BMAXM + j] = -s.sn[i] * a + s.cs[i] * bb;
  }
  const double a = s.H[j * BMAXM + j], bb = s.H[(j + 1) * BMAXM + j];
  const double rr = hypot(a, bb);
  if (rr == 0.0) {
    s.active = 0;
    s.status = BF_BREAKDOWN;
    return;
  }
  s.cs[j] = a / rr;
  s.sn[j] = bb / rr;
  s.H[j * BMAXM + j] = rr;
  s.H[(j + 1) * BMAXM + j] = 0.0;
  s.g[j + 1] = -s.sn[j] * s.g[j];
  s.g[j] = s.cs[j] * s.g[j];
  s.relres = fabs(s.g[j + 1]) / s.beta0;
  const bool conv = fabs(s.g[j + 1]) <= s.tol;
  const bool happy = hnorm <= 1e-300;
  if (!conv && !happy && j + 1 < m && s.total < max_lin_it) {
    s.hinv = 1.0 / hnorm;
    return;
  }
  // finish the cycle: y = R^-1 g by back substitution
  const int kd = j + 1;
  for (int i = kd - 1; i >= 0; --i) {
    double acc = s.g[i];
    for (int k2 = i + 1; k2 < kd; ++k2) acc -= s.H[i * BMAXM + k2] * s.y[k2];
    s.y[i] = acc / s.H[i * BMAXM + i];
  }
  s.kdone = kd;
  s.upd = 1;
  s.active = 0;
  if (conv) {
    s.converged = 1;
  } else if (s.total >= max_lin_it) {
    s.status = BF_NOTCONV;
  } else {
    s.restart = 1;  // true residual and a new cycle
  }
}

// V_{j+1} = w * hinv for problems that continue
__global__ void k_b_next_basis(const BOut* __restrict__ O, const BFgm* __restrict__ F, int j) {
  const int p = blockIdx.y;
  if (!F[p].active) return;
  const BOut& o = O[p];
  const double s = F[p].hinv;
  double* v = o.V + int64_t(j + 1) * o.n;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < o.n; i += int64_t(gridDim.x) * blockDim.x)
    v[i] = o.w[i] * s;
}

// x += sum_{i<kdone} y_i Z_i for problems that finished a cycle
__global__ void k_b_update(const BOut* __restrict__ O, const BFgm* __restrict__ F) {
  const int p = blockIdx.y;
  if (!F[p].upd) return;
  const BOut& o = O[p];
  const int kd = F[p].kdone;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < o.n; i += int64_t(gridDim.x) * blockDim.x) {
    double s = o.x[i];
    for (int k = 0; k < kd; ++k) s += F[p].y[k] * double(o.Z[int64_t(k) * o.n + i]);
    o.x[i] = s;
  }
}

// flags word: number of active problems (read by the host after each iteration)
__global__ void k_b_count(const BFgm* __restrict__ F, int np, int* out) {
  __shared__ int cnt[2];
  if (threadIdx.x < 2) cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    if (F[p].active) atomicAdd(&cnt[0], 1);
    if (F[p].restart) atomicAdd(&cnt[1], 1);
  }
  __syncthreads();
  if (threadIdx.x < 2) out[threadIdx.x] = cnt[threadIdx.x];
}

// Restart, step 1: w = J x at Dirichlet DOFs (identity), 0 elsewhere.
__global__ void k_b_restart_init(const BOut* __restrict__ O, const BFgm* __restrict__ F) {
  const int p = blockIdx.y;
  if (!F[p].restart) return;
  const BOut& o = O[p];
  const int64_t nn = o.g.nn();
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < o.n; i += int64_t(gridDim.x) * blockDim.x)
    o.w[i] = ((o.mask[i % nn] >> int(i / nn)) & 1) ? o.x[i] : 0.0;
}

// Restart, step 2: r = b - w
__global__ void k_b_restart_res(const BOut* __restrict__ O, const BFgm* __restrict__ F) {
  const int p = blockIdx.y;
  if (!F[p].restart) return;
  const BOut& o = O[p];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < o.n; i += int64_t(gridDim.x) * blockDim.x)
    o.r[i] = o.b[i] - o.w[i];
}

// Begin a cycle from r (restart) or from b (first cycle, begin == true):
// beta = ||r||, convergence check, g = beta e_1, hinv = 1/beta.
__global__ void k_b_cycle_state(BFgm* __restrict__ F, int np, const double* __restrict__ nrm2, int stride,
                                bool begin, double rtol, int max_lin_it) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  BFgm& s = F[p];
  if (!(begin || s.restart)) return;
  const double beta = sqrt(nrm2[int64_t(p) * stride]);
  s.restart = 0;
  if (begin) {
    s.total = 0;
    s.converged = 0;
    s.status = BF_OK;
    s.beta0 = beta;
    s.tol = rtol * beta;
    s.relres = beta > 0.0 ? 1.0 : 0.0;
    if (!isfinite(beta)) {
      s.status = BF_NONFINITE;
      s.active = 0;
      return;
    }
    if (beta == 0.0) {
      s.converged = 1;
      s.active = 0;
      return;
    }
  } else {
    s.relres = beta / s.beta0;
    if (beta <= s.tol) {
      s.converged = 1;
      s.active = 0;
      return;
    }
    if (s.total >= max_lin_it) {
      s.status = BF_NOTCONV;
      s.active = 0;
      return;
    }
  }
  s.beta = beta;
  for (int i = 0; i <= BMAXM; ++i) s.g[i] = 0.0;
  s.g[0] = beta;
  s.hinv = 1.0 / beta;
  s.active = 1;
}

// V_0 = src / beta (src = b on the first cycle, r on a restart); x = 0 on the first
__global__ void k_b_first_basis(const BOut* __restrict__ O, const BFgm* __restrict__ F, bool begin) {
  const int p = blockIdx.y;
  if (!F[p].active) return;
  const BOut& o = O[p];
  const double s = F[p].hinv;
  const double* src = begin ? o.b : o.r;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < o.n; i += int64_t(gridDim.x) * blockDim.x) {
    o.V[i] = src[i] * s;
    if (begin) o.x[i] = 0.0;
  }
}

// b = -R (in place), ready for the solve
__global__ void k_b_negate(const BOut* __restrict__ O, const int* __restrict__ act) {
  const int p = blockIdx.y;
  if (!act[p]) return;
  const BOut& o = O[p];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < o.n; i += int64_t(gridDim.x) * blockDim.x)
    o.b[i] = -o.b[i];
}

// U += x for the listed problems
__global__ void k_b_newton_update(const BOut* __restrict__ O, const int* __restrict__ act) {
  const int p = blockIdx.y;
  if (!act[p]) return;
  const BOut& o = O[p];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < o.n; i += int64_t(gridDim.x) * blockDim.x)
    o.U[i] += o.x[i];
}

// ||R||^2 partial sums of the listed problems (R held in b)
__global__ void __launch_bounds__(BT) k_b_res_norm2(const BOut* __restrict__ O, const int* __restrict__ act,
                                                    double* __restrict__ partial) {
  const int p = blockIdx.y;
  double acc = 0.0;
  if (act[p]) {
    const BOut& o = O[p];
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < o.n; i += int64_t(gridDim.x) * blockDim.x)
      acc += o.b[i] * o.b[i];
  }
  __shared__ double red[BT / 32];
  for (int m = 16; m > 0; m >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < BT / 32; ++q) s += red[q];
    partial[int64_t(p) * gridDim.x + blockIdx.x] = s;
  }
}

}  // namespace
}  // namespace pfm
