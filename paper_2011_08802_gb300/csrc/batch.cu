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
// smoothing inside FP64 FGMRES, double-float outer operator), with the FP32
// stores or, when every problem has the binary16 option on, their binary16
// copies in the V-cycle. Other options use the per-problem lockstep driver
// of api.cu.
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
  int problem;     // index of the problem in the batch (gate lookup)
  int level;       // level of the problem
  __half* H16;     // binary16 copy s H of the store (engines with the binary16 option)
  float h16s;      // its power-of-two scale s
  float wh;        // weight w / s of its Hessian part
};

// Per-problem on/off gate of a launch: on[problem * stride] != 0. The V-cycle
// is gated by the FGMRES activity flags, the linearisation by the Newton
// activity flags.
struct Gate {
  const int* on;
  int stride;
  __device__ __forceinline__ bool operator()(int p) const { return on[int64_t(p) * stride] != 0; }
};
enum { VX = 0, VB = 1, VY = 2, VR = 3, VD = 4 };

// Transfer between level l (fine) and l+1 (coarse) of one problem.
struct BTr {
  int problem;
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
  int problem;
  int n;
  const double* Kinv;
  const float* b;
  float* x;
};

// Linearisation of one level of one problem.
struct BLin {
  int problem;
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
  int problem;
  Grid f, c;
  const double* Uf;
  double* Uc;
  const double* Unf;
  double* Unc;
};

// Diagonal blocks of one level of one problem.
struct BBd {
  int problem;
  Grid g;
  JParams<float> jp;
  const float* H;
  float* D;
  const dmask_t* mask;
  int64_t e0;  // first element of this level in the set's numbering
};

// Gauss-Jordan inverse of one problem's dense coarse operator.
struct BGj {
  int problem;
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

// y += J v over all element blocks of the set; v = vec[vsel], y = vec[ysel],
// from the FP32 stores or (H16) from their binary16 copies.
// Each warp caches the descriptor of its current problem in shared memory.
template <bool H16>
__global__ void __launch_bounds__(256) k_b_japply(const BLev* __restrict__ S, int ns, int64_t nblk, int vsel,
                                                  int ysel, Gate on) {
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
    if (on(L.problem) && blk - L.blk0 < L.g.nblk()) {
      if constexpr (H16)
        japply_block_h16<false>(L.g, L.jp, L.wh, L.H16, L.mask, L.vec[vsel], L.vec[ysel], blk - L.blk0, lane);
      else
        japply_block<float>(L.g, L.jp, L.H, L.mask, L.vec[vsel], L.vec[ysel], blk - L.blk0, lane);
    }
  }
}

// max |H| of every level's FP32 store, as float bits in amax[entry]
// (non-negative floats order as their bit patterns; NaN counts as +infinity)
__global__ void k_b_absmax(const BLev* __restrict__ S, unsigned* __restrict__ amax, Gate on) {
  const BLev& L = S[blockIdx.y];
  if (!on(L.problem)) return;
  const int64_t n = L.g.nblk() * HBLK;
  float m = 0.f;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    m = absmax_step(m, L.H[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax + blockIdx.y, __float_as_uint(m));
}

// binary16 copy h16s H of every level's FP32 store
__global__ void k_b_to_half(const BLev* __restrict__ S, Gate on) {
  const BLev& L = S[blockIdx.y];
  if (!on(L.problem)) return;
  const int64_t nvec = L.g.nblk() * HBLK / 8;
  uint4* out = reinterpret_cast<uint4*>(L.H16);
  const float4* in = reinterpret_cast<const float4*>(L.H);
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nvec; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = half_vector(in, L.h16s, i);
}

// y = v at Dirichlet DOFs, 0 elsewhere (identity rows of J).
__global__ void k_b_init(const BLev* __restrict__ S, int vsel, int ysel, Gate on) {
  const BLev& L = S[blockIdx.y];
  if (!on(L.problem)) return;
  const int64_t nn = L.g.nn();
  const float* v = L.vec[vsel];
  float* y = L.vec[ysel];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < NF * nn; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = ((L.mask[i % nn] >> int(i / nn)) & 1) ? v[i] : 0.f;
}

__global__ void k_b_cheb_first(const BLev* __restrict__ S, int srcsel, bool copy_r, bool zero_x, Gate on) {
  const BLev& L = S[blockIdx.y];
  if (!on(L.problem)) return;
  const int64_t nn = L.g.nn();
  for (int64_t node = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; node < nn; node += int64_t(gridDim.x) * blockDim.x)
    cheb_first_node<float>(nn, L.D, L.vec[srcsel], L.inv_theta, copy_r, zero_x, L.vec[VR], L.vec[VD], L.vec[VX], node);
}

__global__ void k_b_cheb_step(const BLev* __restrict__ S, float a, float c, Gate on) {
  const BLev& L = S[blockIdx.y];
  if (!on(L.problem)) return;
  const int64_t nn = L.g.nn();
  const float cp = c * L.inv_delta;
  for (int64_t node = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; node < nn; node += int64_t(gridDim.x) * blockDim.x)
    cheb_step_node<float>(nn, L.D, L.vec[VY], a, cp, L.vec[VR], L.vec[VD], L.vec[VX], node);
}

// out = vec[asel] - vec[bsel]
__global__ void k_b_sub(const BLev* __restrict__ S, int asel, int bsel, int osel, Gate on) {
  const BLev& L = S[blockIdx.y];
  if (!on(L.problem)) return;
  const int64_t n = NF * L.g.nn();
  const float* a = L.vec[asel];
  const float* b = L.vec[bsel];
  float* o = L.vec[osel];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    o[i] = a[i] - b[i];
}

__global__ void k_b_restrict(const BTr* __restrict__ T, Gate on) {
  const BTr& t = T[blockIdx.y];
  if (!on(t.problem)) return;
  const int64_t nnc = t.c.nn();
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < nnc; idx += int64_t(gridDim.x) * blockDim.x)
    restrict_node<float>(t.f, t.c, t.rf, t.mc, t.bc, idx);
}

__global__ void k_b_prolong(const BTr* __restrict__ T, Gate on) {
  const BTr& t = T[blockIdx.y];
  if (!on(t.problem)) return;
  const int64_t nnf = t.f.nn();
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < nnf; idx += int64_t(gridDim.x) * blockDim.x)
    prolong_node<float>(t.f, t.c, t.xc, t.mf, t.xf, idx);
}

// x = Kinv b, one warp per row; blockIdx.y = problem.
__global__ void k_b_coarse_solve(const BCo* __restrict__ C, Gate on) {
  const BCo& c = C[blockIdx.y];
  if (!on(c.problem)) return;
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

__global__ void k_b_inject(const BInj* __restrict__ I, Gate on) {
  const BInj& t = I[blockIdx.y];
  if (!on(t.problem)) return;
  const int64_t nnc = t.c.nn();
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < nnc; idx += int64_t(gridDim.x) * blockDim.x) {
    inject_node(t.f, t.c, t.Uf, t.Uc, idx);
    inject_node(t.f, t.c, t.Unf, t.Unc, idx);
  }
}

template <typename TC>
__global__ void __launch_bounds__(128) k_b_linearize(const BLin* __restrict__ S, int ns, int64_t nblk, Gate on) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t blk = tid >> 5;
  if (blk >= nblk) return;
  const BLin& L = S[find_entry(S, ns, blk)];
  if (!on(L.problem)) return;
  linearize_lane<TC>(L.g, *L.P, L.U, L.Un, L.H64, L.H32, L.H32lo, blk - L.blk0, int(tid & 31));
}

__global__ void k_b_zero_D(const BBd* __restrict__ S, Gate on) {
  const BBd& L = S[blockIdx.y];
  if (!on(L.problem)) return;
  const int64_t n = NF2 * L.g.nn();
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

__global__ void __launch_bounds__(128) k_b_blockdiag(const BBd* __restrict__ S, int ns, int64_t ne, Gate on) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t e = tid >> 3;
  if (e >= ne) return;
  const BBd& L = S[find_elem(S, ns, e)];
  if (!on(L.problem)) return;
  blockdiag_elem_node<float>(L.g, L.jp, L.H, L.D, e - L.e0, int(tid & 7));
}

__global__ void k_b_block_invert(const BBd* __restrict__ S, int* singular, Gate on) {
  const BBd& L = S[blockIdx.y];
  if (!on(L.problem)) return;
  const int64_t nn = L.g.nn();
  for (int64_t node = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; node < nn; node += int64_t(gridDim.x) * blockDim.x)
    block_invert_node<float>(nn, L.mask, L.D, singular, node);
}

// power iteration: x = start vector
__global__ void k_b_power_init(const BLev* __restrict__ S, Gate on) {
  const BLev& L = S[blockIdx.y];
  if (!on(L.problem)) return;
  const int64_t nn = L.g.nn();
  float* x = L.vec[VX];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < NF * nn; i += int64_t(gridDim.x) * blockDim.x)
    x[i] = float(power_init_value(i, nn, L.mask));
}

// vec[dst] = D^-1 vec[src] (one point-block Jacobi step from zero)
__global__ void k_b_dinv(const BLev* __restrict__ S, int src, int dst, Gate on) {
  const BLev& L = S[blockIdx.y];
  if (!on(L.problem)) return;
  const int64_t nn = L.g.nn();
  const float* y = L.vec[src];
  float* r = L.vec[dst];
  for (int64_t node = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; node < nn; node += int64_t(gridDim.x) * blockDim.x) {
    float yv[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) yv[f] = y[f * nn + node];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      float s = 0.f;
#pragma unroll
      for (int c = 0; c < NF; ++c) s += L.D[(f * NF + c) * nn + node] * yv[c];
      r[f * nn + node] = s;
    }
  }
}

// partial[(entry * BCH + chunk)] = sum over the chunk of vec[sa] . vec[sb] (FP64 accumulation)
__global__ void __launch_bounds__(BT) k_b_dot_32(const BLev* __restrict__ S, int sa, int sb,
                                                 double* __restrict__ partial, Gate on) {
  const BLev& L = S[blockIdx.y];
  const int64_t n = on(L.problem) ? NF * L.g.nn() : 0;
  const float* a = L.vec[sa];
  const float* c = L.vec[sb];
  double acc = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    acc += double(a[i]) * double(c[i]);
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

// vec[dst] = vec[src] / sqrt(dot[entry]) (0 for a non-positive dot)
__global__ void k_b_scale(const BLev* __restrict__ S, int src, int dst, const double* __restrict__ dot, Gate on) {
  const BLev& L = S[blockIdx.y];
  if (!on(L.problem)) return;
  const int64_t n = NF * L.g.nn();
  const double d = dot[blockIdx.y];
  const float sc = d > 0.0 ? float(1.0 / sqrt(d)) : 0.f;
  const float* a = L.vec[src];
  float* x = L.vec[dst];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i] = a[i] * sc;
}

// vec[sel] = 0
__global__ void k_b_zero(const BLev* __restrict__ S, int sel, Gate on) {
  const BLev& L = S[blockIdx.y];
  if (!on(L.problem)) return;
  const int64_t n = NF * L.g.nn();
  float* x = L.vec[sel];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i] = 0.f;
}

// Lanczos step of every entry: vec[u] -= alpha[e] vec[q] + sqrt(beta2prev[e]) vec[qp]
__global__ void k_b_lanczos_orth(const BLev* __restrict__ S, int usel, int qsel, int qpsel,
                                 const double* __restrict__ alpha, const double* __restrict__ beta2prev, Gate on) {
  const BLev& L = S[blockIdx.y];
  if (!on(L.problem)) return;
  const int64_t n = NF * L.g.nn();
  const float a = float(alpha[blockIdx.y]);
  const float bq = beta2prev ? float(sqrt(beta2prev[blockIdx.y])) : 0.f;
  float* u = L.vec[usel];
  const float* q = L.vec[qsel];
  const float* qp = L.vec[qpsel];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    u[i] -= a * q[i] + (beta2prev ? bq * qp[i] : 0.f);
}

// Gauss-Jordan over the batch: blockIdx.y = problem
__global__ void k_b_gj_first_key(const BGj* __restrict__ G, Gate on) {
  const BGj& q = G[blockIdx.y];
  if (!on(q.problem)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < q.n; i += gridDim.x * blockDim.x)
    atomicMax(&q.keys[0], pivot_key(q.M[int64_t(i) * 2 * q.n], i));
}

__global__ void __launch_bounds__(256) k_b_gj_step(const BGj* __restrict__ G, int k, int* singular, Gate on) {
  const BGj& q = G[blockIdx.y];
  if (k >= q.n || !on(q.problem)) return;
  gj_step_row(q.M, q.n, 2 * q.n, k, q.keys, q.used, q.piv, singular, int(blockIdx.x), blockIdx.x == 0);
}

__global__ void k_b_gj_extract(const BGj* __restrict__ G, Gate on) {
  const BGj& q = G[blockIdx.y];
  const int k = blockIdx.x;
  if (k >= q.n || !on(q.problem)) return;
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

// w += J Z_j in double-float arithmetic over all element blocks (2 CTAs per
// SM at 128 registers, as the single-problem kernel)
__global__ void __launch_bounds__(256, (PFM_NV == 6 ? 2 : 1)) k_b_japply_df(const BOut* __restrict__ O, const BFgm* __restrict__ F, int np,
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
  if (!s.restart) return;
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

// V_0 = r / beta for problems that start a cycle
__global__ void k_b_first_basis(const BOut* __restrict__ O, const BFgm* __restrict__ F) {
  const int p = blockIdx.y;
  if (!F[p].active) return;
  const BOut& o = O[p];
  const double s = F[p].hinv;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < o.n; i += int64_t(gridDim.x) * blockDim.x)
    o.V[i] = o.r[i] * s;
}

// start of a solve: the listed problems get x = 0 and the restart flag (their
// first cycle is built from r = b like a restart); everything else is idle
__global__ void k_b_begin(const BOut* __restrict__ O, BFgm* __restrict__ F, const int* __restrict__ act) {
  const int p = blockIdx.y;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    F[p].restart = act[p];
    F[p].active = 0;
    F[p].upd = 0;
  }
  if (!act[p]) return;
  const BOut& o = O[p];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < o.n; i += int64_t(gridDim.x) * blockDim.x)
    o.x[i] = 0.0;
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

// ===========================================================================
// Host side of the engine

namespace pfm {

struct BatchEngine {
  std::vector<uint64_t> sig;  // buffers and parameters the descriptors were built from
  // options the captured graphs depend on
  int m = 0, nu_pre = 0, nu_post = 0, max_lin_it = 0;
  double lo = 0, hi = 0, growth = 0, rtol = 0;
  cudaStream_t s = nullptr;
  int np = 0, depth = 0;
  std::vector<int> nlev;
  struct DSet {
    std::vector<BLev> S;
    BLev* dS = nullptr;
    int64_t nblk = 0, maxnn = 0;
    std::vector<BTr> T;
    BTr* dT = nullptr;
    int64_t maxnnf = 0, maxnnc = 0;
    std::vector<BCo> C;
    BCo* dC = nullptr;
    int maxn = 0;
  };
  std::vector<DSet> D;
  std::vector<BLev> A;  // every non-coarsest level (power iteration)
  BLev* dA = nullptr;
  int64_t nblkA = 0, maxnnA = 0;
  std::vector<std::pair<int, int>> Aidx;
  std::vector<BLin> L64, L32;
  BLin* dL64 = nullptr;
  BLin* dL32 = nullptr;
  int64_t nblk64 = 0, nblk32 = 0;
  std::vector<std::vector<BInj>> Inj;
  std::vector<BInj*> dInj;
  std::vector<int64_t> maxnnInj;
  std::vector<BBd> Bd;
  BBd* dBd = nullptr;
  int64_t neBd = 0, maxnnBd = 0;
  std::vector<BGj> G;
  BGj* dG = nullptr;
  int maxnG = 0;
  std::vector<BOut> O;
  BOut* dO = nullptr;
  int64_t nblkO = 0, maxnO = 0;
  DevParams* dP = nullptr;
  BFgm* dF = nullptr;
  double *partial = nullptr, *h1 = nullptr, *h2 = nullptr, *hn = nullptr, *dots = nullptr;
  int* flags = nullptr;
  int* dact = nullptr;
  int* singular = nullptr;
  int* hflags = nullptr;   // pinned: active count, restart count
  double* hres = nullptr;  // pinned: per-problem norms / lambda estimates
  int* hact = nullptr;     // pinned: Newton activity
  int grid_japply = 0, grid_df = 0, grid_j64 = 0;
  bool h16 = false;             // the V-cycle applies the binary16 copies of the stores
  unsigned* amax = nullptr;     // per A-set level: max |H| bits
  double* lz = nullptr;         // Lanczos alpha, beta^2 and start norms of the A-set levels
  double* hlz = nullptr;        // pinned copy of alpha and beta^2
  size_t lz_cap = 0;
  unsigned* hamax = nullptr;    // pinned copy
  cudaGraphExec_t vgraph = nullptr;
  std::vector<cudaGraphExec_t> itg;
  std::vector<int64_t> itg_launches;  // kernels in each iteration graph
  std::vector<void*> dmem;

  template <typename T>
  cudaError_t alloc(T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(T) * std::max<size_t>(count, 1));
    if (e == cudaSuccess) dmem.push_back(q);
    *p = static_cast<T*>(q);
    return e;
  }
  template <typename T>
  cudaError_t upload(T** dp, const std::vector<T>& v) {
    if (v.empty()) {
      *dp = nullptr;
      return cudaSuccess;
    }
    cudaError_t e = alloc(dp, v.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dp, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
  }
  ~BatchEngine() {
    if (vgraph) cudaGraphExecDestroy(vgraph);
    for (auto g : itg)
      if (g) cudaGraphExecDestroy(g);
    for (void* q : dmem) cudaFree(q);
    if (hflags) cudaFreeHost(hflags);
    if (hres) cudaFreeHost(hres);
    if (hact) cudaFreeHost(hact);
    if (hamax) cudaFreeHost(hamax);
    if (hlz) cudaFreeHost(hlz);
  }
  Gate gate_fgm() const { return Gate{&dF[0].active, int(sizeof(BFgm) / sizeof(int))}; }
  Gate gate_act() const { return Gate{dact, 1}; }
};

void batch_engine_free(BatchEngine* e) { delete e; }

namespace {

#define BCK(call)                                                                                 \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess)                                                                        \
      return b->fail(e_ == cudaErrorMemoryAllocation ? PFM_ERR_OOM : PFM_ERR_CUDA,                \
                     std::string(#call) + ": " + cudaGetErrorString(e_));                         \
  } while (0)

int sm_count_b() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  return sms;
}

template <typename K>
int persistent_blocks(K kernel, int threads, int64_t work_threads) {
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, 0);
  const int64_t full = int64_t(sm_count_b()) * std::max(occ, 1);
  const int64_t need = (work_threads + threads - 1) / threads;
  return int(std::max<int64_t>(1, std::min(full, need)));
}

inline dim3 grid2(int64_t maxn, int ny) { return dim3(std::min<unsigned>(gdiv(maxn, BT), 1024u), unsigned(ny)); }

// Per-handle buffers the engine uses, allocated on the handle (and kept).
pfm_status engine_buffers(pfm_handle* h, int m) {
  const size_t nl = h->L.size();
  for (size_t l = 0; l < nl; ++l) {
    Level& lv = h->L[l];
    const size_t hsz = size_t(lv.nblk) * HBLK;
    const bool fine = l == 0, coarsest = l + 1 == nl;
    if (fine || coarsest) TRY(dalloc(h, &lv.H64, hsz));
    if (fine || !coarsest) TRY(dalloc(h, &lv.H32, hsz));
    if (fine) TRY(dalloc(h, &lv.H32lo, hsz));
    if (h->pre_h16 && !coarsest) TRY(dalloc(h, &lv.H16, hsz));
    if (!coarsest) TRY(dalloc(h, &lv.D32, size_t(NF2) * lv.nn));
    TRY(dalloc(h, &lv.x32, ndof(lv)));
    TRY(dalloc(h, &lv.b32, ndof(lv)));
    TRY(dalloc(h, &lv.y32, ndof(lv)));
    TRY(dalloc(h, &lv.r32, ndof(lv)));
    TRY(dalloc(h, &lv.d32, ndof(lv)));
  }
  const int64_t n = ndof(h->L[0]);
  if (h->kry_m < m || h->kry_prec != PFM_F32) {
    dfree(h->V);
    if (h->Z) cudaFree(h->Z);
    h->Z = nullptr;
    TRY(dalloc(h, &h->V, size_t(m + 1) * n));
    float* z = nullptr;
    TRY(dalloc(h, &z, size_t(m) * n));
    h->Z = z;
    h->kry_m = m;
    h->kry_prec = PFM_F32;
  }
  return PFM_OK;
}

pfm_status engine_build(pfm_batch* b, const pfm_solve_opts& o, BatchEngine** out) {
  auto E = new BatchEngine();
  auto fail = [&](pfm_status st) {
    delete E;
    return st;
  };
  const int np = int(b->hs.size());
  E->np = np;
  E->s = b->streams[0];
  E->m = o.restart;
  E->nu_pre = o.nu_pre;
  E->nu_post = o.nu_post;
  E->lo = o.cheb_lo;
  E->hi = o.cheb_hi;
  E->growth = o.nu_growth > 0 ? o.nu_growth : 1.0;
  E->max_lin_it = o.max_lin_it;
  E->rtol = o.lin_rtol;
  for (int p = 0; p < np; ++p) {
    pfm_status st = engine_buffers(b->hs[p], o.restart);
    if (st != PFM_OK) {
      b->err = "problem " + std::to_string(p) + ": " + b->hs[p]->err;
      return fail(st);
    }
    E->nlev.push_back(int(b->hs[p]->L.size()));
    E->depth = std::max(E->depth, int(b->hs[p]->L.size()));
  }
  // parameters of every problem on the device
  {
    std::vector<DevParams> P(np);
    for (int p = 0; p < np; ++p) P[p] = b->hs[p]->dp;
    if (E->upload(&E->dP, P) != cudaSuccess) return fail(b->fail(PFM_ERR_OOM, "engine parameter table"));
  }
  E->D.resize(E->depth);
  E->Inj.resize(E->depth);
  for (int p = 0; p < np; ++p) {
    pfm_handle* h = b->hs[p];
    const int nl = E->nlev[p];
    for (int l = 0; l < nl; ++l) {
      Level& lv = h->L[l];
      const bool coarsest = l + 1 == nl;
      // linearisation: finest and coarsest levels in FP64, the others in FP32
      BLin li{};
      li.problem = p;
      li.g = lv.g;
      li.P = E->dP + p;
      li.U = lv.U;
      li.Un = lv.Un;
      if (l == 0) {
        li.H64 = lv.H64;
        li.H32 = lv.H32;
        li.H32lo = lv.H32lo;
      } else if (coarsest) {
        li.H64 = lv.H64;
      } else {
        li.H32 = lv.H32;
      }
      auto& Lset = (l == 0 || coarsest) ? E->L64 : E->L32;
      auto& nb = (l == 0 || coarsest) ? E->nblk64 : E->nblk32;
      li.blk0 = nb;
      nb += lv.nblk;
      Lset.push_back(li);
      if (l > 0) {
        Level& fl = h->L[l - 1];
        E->Inj[l].push_back(BInj{p, fl.g, lv.g, fl.U, lv.U, fl.Un, lv.Un});
      }
      if (coarsest) {
        E->D[l].C.push_back(BCo{p, h->nc_dofs, h->Kinv, lv.b32, lv.x32});
        E->D[l].maxn = std::max(E->D[l].maxn, h->nc_dofs);
        E->G.push_back(BGj{p, h->Kaug, h->nc_dofs, h->gj_keys, h->gj_used, h->gj_piv, h->Kinv});
        E->maxnG = std::max(E->maxnG, h->nc_dofs);
        continue;
      }
      BLev L{};
      L.g = lv.g;
      L.jp = make_jparams<float>(lv.g, h->dp);
      L.mask = lv.mask;
      L.H = lv.H32;
      L.D = lv.D32;
      L.vec[VX] = lv.x32;
      L.vec[VB] = lv.b32;
      L.vec[VY] = lv.y32;
      L.vec[VR] = lv.r32;
      L.vec[VD] = lv.d32;
      L.problem = p;
      L.level = l;
      L.H16 = h->pre_h16 ? lv.H16 : nullptr;
      auto& Ds = E->D[l];
      L.blk0 = Ds.nblk;
      Ds.nblk += lv.nblk;
      Ds.maxnn = std::max(Ds.maxnn, lv.nn);
      Ds.S.push_back(L);
      L.blk0 = E->nblkA;
      E->nblkA += lv.nblk;
      E->maxnnA = std::max(E->maxnnA, lv.nn);
      E->A.push_back(L);
      E->Aidx.push_back({p, l});
      Level& cv = h->L[l + 1];
      Ds.T.push_back(BTr{p, lv.g, cv.g, lv.mask, cv.mask, lv.r32, cv.b32, cv.x32, lv.x32});
      Ds.maxnnf = std::max(Ds.maxnnf, lv.nn);
      Ds.maxnnc = std::max(Ds.maxnnc, cv.nn);
      BBd bd{};
      bd.problem = p;
      bd.g = lv.g;
      bd.jp = L.jp;
      bd.H = lv.H32;
      bd.D = lv.D32;
      bd.mask = lv.mask;
      bd.e0 = E->neBd;
      E->neBd += lv.ne;
      E->maxnnBd = std::max(E->maxnnBd, lv.nn);
      E->Bd.push_back(bd);
    }
    Level& f = h->L[0];
    if (!f.H32 || !f.H32lo || !f.H64 || !h->V || !h->Z || !h->Kinv) {
      b->err = "problem " + std::to_string(p) + ": engine buffers missing";
      return fail(PFM_ERR_STATE);
    }
    BOut ob{};
    ob.g = f.g;
    ob.n = ndof(f);
    ob.dk = make_dfconst(f.g, h->dp);
    ob.jp64 = make_jparams<double>(f.g, h->dp);
    ob.Hhi = f.H32;
    ob.Hlo = f.H32lo;
    ob.H64 = f.H64;
    ob.mask = f.mask;
    ob.V = h->V;
    ob.Z = static_cast<float*>(h->Z);
    ob.w = h->wv;
    ob.x = h->dU;
    ob.b = h->R;
    ob.r = h->rv;
    ob.U = f.U;
    ob.b32 = f.b32;
    ob.x32 = f.x32;
    ob.blk0 = E->nblkO;
    E->nblkO += f.nblk;
    E->maxnO = std::max(E->maxnO, ob.n);
    E->O.push_back(ob);
  }
  for (int l = 1; l < E->depth; ++l) {
    int64_t mx = 0;
    for (auto& t : E->Inj[l]) mx = std::max(mx, t.c.nn());
    E->maxnnInj.push_back(mx);
  }
  E->maxnnInj.insert(E->maxnnInj.begin(), 0);
  cudaError_t e = cudaSuccess;
  auto up = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  for (auto& Ds : E->D) {
    up(E->upload(&Ds.dS, Ds.S));
    up(E->upload(&Ds.dT, Ds.T));
    up(E->upload(&Ds.dC, Ds.C));
  }
  E->dInj.assign(E->depth, nullptr);
  for (int l = 1; l < E->depth; ++l) up(E->upload(&E->dInj[l], E->Inj[l]));
  up(E->upload(&E->dA, E->A));
  up(E->upload(&E->dL64, E->L64));
  up(E->upload(&E->dL32, E->L32));
  up(E->upload(&E->dBd, E->Bd));
  up(E->upload(&E->dG, E->G));
  up(E->upload(&E->dO, E->O));
  const int stride = BMAXM + 1;
  up(E->alloc(&E->dF, np));
  up(E->alloc(&E->partial, size_t(std::max<size_t>(np, E->A.size())) * BCH * stride));
  up(E->alloc(&E->h1, size_t(np) * stride));
  up(E->alloc(&E->h2, size_t(np) * stride));
  up(E->alloc(&E->hn, size_t(np) * stride));
  up(E->alloc(&E->dots, std::max<size_t>(np, E->A.size())));
  up(E->alloc(&E->flags, 2));
  up(E->alloc(&E->dact, np));
  up(E->alloc(&E->singular, 1));
  up(E->alloc(&E->amax, std::max<size_t>(E->A.size(), 1)));
  if (e == cudaSuccess) e = cudaMemset(E->dF, 0, sizeof(BFgm) * np);
  if (e == cudaSuccess)
    e = cudaMallocHost(reinterpret_cast<void**>(&E->hamax), sizeof(unsigned) * std::max<size_t>(E->A.size(), 1));
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&E->hflags), sizeof(int) * 2);
  if (e == cudaSuccess)
    e = cudaMallocHost(reinterpret_cast<void**>(&E->hres), sizeof(double) * std::max<size_t>(np, E->A.size()));
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&E->hact), sizeof(int) * np);
  if (e != cudaSuccess) return fail(b->fail(PFM_ERR_OOM, std::string("engine tables: ") + cudaGetErrorString(e)));
  E->h16 = b->hs[0]->pre_h16;  // the same for every problem (batch_engine_supports)
  E->grid_japply = E->h16 ? persistent_blocks(k_b_japply<true>, 256, std::max<int64_t>(E->nblkA, 1) * 32)
                          : persistent_blocks(k_b_japply<false>, 256, std::max<int64_t>(E->nblkA, 1) * 32);
  E->grid_df = persistent_blocks(k_b_japply_df, 256, E->nblkO * 32);
  E->grid_j64 = persistent_blocks(k_b_japply64, 256, E->nblkO * 32);
  *out = E;
  return PFM_OK;
}

// y = J v on every level of a set (identity rows first, then the elements)
void eng_japply(BatchEngine* E, const BLev* dS, int ns, int64_t nblk, int64_t maxnn, int v, int y, Gate g) {
  k_b_init<<<grid2(NF * maxnn, ns), BT, 0, E->s>>>(dS, v, y, g);
  const int blocks = std::max(1, std::min<int>(E->grid_japply, int(gdiv(nblk * 32, 256))));
  if (E->h16)
    k_b_japply<true><<<blocks, 256, 0, E->s>>>(dS, ns, nblk, v, y, g);
  else
    k_b_japply<false><<<blocks, 256, 0, E->s>>>(dS, ns, nblk, v, y, g);
  count_launches(2);
}

// nu Chebyshev steps on depth d (the single-problem smoother, every problem at once)
void eng_smooth(BatchEngine* E, int d, bool zero_x, int nu, bool want_res, Gate g) {
  auto& Ds = E->D[d];
  const int ns = int(Ds.S.size());
  const dim3 gn = grid2(Ds.maxnn, ns), gv = grid2(NF * Ds.maxnn, ns);
  const double sigma = (E->hi + E->lo) / (E->hi - E->lo);
  double rho = 1.0 / sigma;
  if (zero_x) {
    k_b_cheb_first<<<gn, BT, 0, E->s>>>(Ds.dS, VB, true, true, g);
    count_launches(1);
  } else {
    eng_japply(E, Ds.dS, ns, Ds.nblk, Ds.maxnn, VX, VY, g);
    k_b_sub<<<gv, BT, 0, E->s>>>(Ds.dS, VB, VY, VR, g);
    k_b_cheb_first<<<gn, BT, 0, E->s>>>(Ds.dS, VR, false, false, g);
    count_launches(2);
  }
  for (int k = 1; k < nu; ++k) {
    eng_japply(E, Ds.dS, ns, Ds.nblk, Ds.maxnn, VD, VY, g);
    const double rho_n = 1.0 / (2.0 * sigma - rho);
    k_b_cheb_step<<<gn, BT, 0, E->s>>>(Ds.dS, float(rho_n * rho), float(2.0 * rho_n), g);
    count_launches(1);
    rho = rho_n;
  }
  if (want_res) {
    eng_japply(E, Ds.dS, ns, Ds.nblk, Ds.maxnn, VD, VY, g);
    k_b_sub<<<gv, BT, 0, E->s>>>(Ds.dS, VR, VY, VR, g);
    count_launches(1);
  }
}

void eng_vcycle(BatchEngine* E, int d, Gate g) {
  auto& Ds = E->D[d];
  if (!Ds.C.empty()) {
    k_b_coarse_solve<<<dim3(gdiv(int64_t(Ds.maxn) * 32, 256), unsigned(Ds.C.size())), 256, 0, E->s>>>(Ds.dC, g);
    count_launches(1);
  }
  if (Ds.S.empty()) return;
  const double gl = std::pow(E->growth, double(d));
  const int nu_pre = std::max(1, int(std::lround(E->nu_pre * gl)));
  const int nu_post = E->nu_post > 0 ? std::max(1, int(std::lround(E->nu_post * gl))) : 0;
  const int ns = int(Ds.S.size());
  eng_smooth(E, d, true, nu_pre, true, g);
  k_b_restrict<<<grid2(Ds.maxnnc, ns), BT, 0, E->s>>>(Ds.dT, g);
  count_launches(1);
  eng_vcycle(E, d + 1, g);
  k_b_prolong<<<grid2(Ds.maxnnf, ns), BT, 0, E->s>>>(Ds.dT, g);
  count_launches(1);
  if (nu_post > 0) eng_smooth(E, d, false, nu_post, false, g);
}

// Linearisation of every active problem (all levels), smoother eigenvalue
// estimates, dense coarse inverses.
pfm_status eng_linearize(pfm_batch* b, BatchEngine* E, int power_its) {
  cudaStream_t s = E->s;
  const Gate g = E->gate_act();
  for (int l = 1; l < E->depth; ++l) {
    if (E->Inj[l].empty()) continue;
    k_b_inject<<<dim3(std::min<unsigned>(gdiv(E->maxnnInj[l], 128), 1024u), unsigned(E->Inj[l].size())), 128, 0, s>>>(
        E->dInj[l], g);
    count_launches(1);
  }
  BCK(cudaMemsetAsync(E->singular, 0, sizeof(int), s));
  if (E->nblk64 > 0) {
    k_b_linearize<double><<<gdiv(E->nblk64 * 32, 128), 128, 0, s>>>(E->dL64, int(E->L64.size()), E->nblk64, g);
    count_launches(1);
  }
  if (E->nblk32 > 0) {
    k_b_linearize<float><<<gdiv(E->nblk32 * 32, 128), 128, 0, s>>>(E->dL32, int(E->L32.size()), E->nblk32, g);
    count_launches(1);
  }
  const int nA = int(E->A.size());
  if (E->h16 && nA > 0) {
    // binary16 copies of every preconditioner level's store: max |H| of all
    // levels in one launch, the power-of-two scales on the host (as for a
    // single problem), the copies in one launch
    BCK(cudaMemsetAsync(E->amax, 0, sizeof(unsigned) * nA, s));
    const dim3 ga(unsigned(sm_count_b()) * 2, unsigned(nA));
    k_b_absmax<<<ga, BT, 0, s>>>(E->dA, E->amax, g);
    count_launches(1);
    BCK(cudaMemcpyAsync(E->hamax, E->amax, sizeof(unsigned) * nA, cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    for (int i = 0; i < nA; ++i) {
      BLev& L = E->A[i];
      if (!E->hact[L.problem]) continue;
      float amax = 0.f;
      std::memcpy(&amax, &E->hamax[i], sizeof(float));
      if (!std::isfinite(amax))
        return b->fail(PFM_ERR_NONFINITE, "binary16 store: non-finite Hessian entries in problem " +
                                              std::to_string(L.problem));
      L.h16s = half_store_scale(amax);
      L.wh = float(L.g.w() / double(L.h16s));
      b->hs[L.problem]->L[L.level].h16_scale = L.h16s;
      for (auto& Ls : E->D[L.level].S)
        if (Ls.problem == L.problem) {
          Ls.h16s = L.h16s;
          Ls.wh = L.wh;
        }
    }
    BCK(cudaMemcpyAsync(E->dA, E->A.data(), sizeof(BLev) * nA, cudaMemcpyHostToDevice, s));
    for (auto& Ds : E->D)
      if (!Ds.S.empty())
        BCK(cudaMemcpyAsync(Ds.dS, Ds.S.data(), sizeof(BLev) * Ds.S.size(), cudaMemcpyHostToDevice, s));
    k_b_to_half<<<ga, BT, 0, s>>>(E->dA, g);
    count_launches(1);
  }
  if (nA > 0) {
    k_b_zero_D<<<grid2(NF2 * E->maxnnBd, nA), BT, 0, s>>>(E->dBd, g);
    k_b_blockdiag<<<gdiv(E->neBd * 8, 128), 128, 0, s>>>(E->dBd, nA, E->neBd, g);
    k_b_block_invert<<<grid2(E->maxnnBd, nA), BT, 0, s>>>(E->dBd, E->singular, g);
    count_launches(3);
    // Lanczos estimate of lambda_max(D^-1 J) on every non-coarsest level at
    // once (the single-problem estimate_lambda, entry by entry): q = VX / VB
    // alternating with q_prev, z = VD, u = VY, w = VR
    const int K = power_its;
    const size_t nlz = size_t(2 * K + 1) * nA;
    if (E->lz_cap < nlz) {
      BCK(E->alloc(&E->lz, nlz));
      if (E->hlz) cudaFreeHost(E->hlz);
      E->hlz = nullptr;
      BCK(cudaMallocHost(reinterpret_cast<void**>(&E->hlz), sizeof(double) * nlz));
      E->lz_cap = nlz;
    }
    double* al = E->lz;                     // [K][nA]
    double* be = E->lz + size_t(K) * nA;    // [K][nA]
    double* nrm = E->lz + size_t(2 * K) * nA;
    const dim3 gv(BCH, unsigned(nA));
    const dim3 gn = grid2(E->maxnnA, nA), gf = grid2(NF * E->maxnnA, nA);
    auto dot = [&](int a, int c, double* out) {
      k_b_dot_32<<<gv, BT, 0, s>>>(E->dA, a, c, E->partial, g);
      k_b_reduce_chunks<<<gdiv(nA, 128), 128, 0, s>>>(nA, BCH, E->partial, out);
    };
    int qs = VX, qps = VB;
    k_b_power_init<<<gf, BT, 0, s>>>(E->dA, g);
    k_b_dinv<<<gn, BT, 0, s>>>(E->dA, VX, VD, g);
    dot(VX, VD, nrm);
    k_b_scale<<<gf, BT, 0, s>>>(E->dA, VX, VX, nrm, g);
    k_b_scale<<<gf, BT, 0, s>>>(E->dA, VD, VD, nrm, g);
    k_b_zero<<<gf, BT, 0, s>>>(E->dA, VB, g);
    count_launches(7);
    for (int j = 0; j < K; ++j) {
      eng_japply(E, E->dA, nA, E->nblkA, E->maxnnA, VD, VY, g);
      dot(VD, VY, al + size_t(j) * nA);
      k_b_lanczos_orth<<<gf, BT, 0, s>>>(E->dA, VY, qs, qps, al + size_t(j) * nA,
                                         j > 0 ? be + size_t(j - 1) * nA : nullptr, g);
      k_b_dinv<<<gn, BT, 0, s>>>(E->dA, VY, VR, g);
      dot(VY, VR, be + size_t(j) * nA);
      count_launches(6);
      if (j + 1 < K) {
        std::swap(qs, qps);
        k_b_scale<<<gf, BT, 0, s>>>(E->dA, VY, qs, be + size_t(j) * nA, g);
        k_b_scale<<<gf, BT, 0, s>>>(E->dA, VR, VD, be + size_t(j) * nA, g);
        count_launches(2);
      }
    }
    BCK(cudaMemcpyAsync(E->hlz, E->lz, sizeof(double) * size_t(2 * K) * nA, cudaMemcpyDeviceToHost, s));
  }
  // dense coarse operators (one assembly per problem) and their inverses (one launch per step for all)
  for (int p = 0; p < E->np; ++p) {
    if (!E->hact[p]) continue;
    pfm_handle* h = b->hs[p];
    Level& c = h->L.back();
    launch_coarse_assemble<double>(c.g, h->dp, c.H64, c.mask, h->Kaug, 2 * h->nc_dofs, s);
    BCK(cudaMemsetAsync(h->gj_keys, 0, sizeof(unsigned long long) * (h->nc_dofs + 1), s));
    BCK(cudaMemsetAsync(h->gj_used, 0, sizeof(int) * h->nc_dofs, s));
  }
  const int nG = int(E->G.size());
  k_b_gj_first_key<<<dim3(gdiv(E->maxnG, 256), unsigned(nG)), 256, 0, s>>>(E->dG, g);
  count_launches(1);
  for (int k = 0; k < E->maxnG; ++k) {
    k_b_gj_step<<<dim3(unsigned(E->maxnG), unsigned(nG)), 256, 0, s>>>(E->dG, k, E->singular, g);
    count_launches(1);
  }
  k_b_gj_extract<<<dim3(unsigned(E->maxnG), unsigned(nG)), 256, 0, s>>>(E->dG, g);
  count_launches(1);
  BCK(cudaGetLastError());
  int sing = 0;
  BCK(cudaMemcpyAsync(&sing, E->singular, sizeof(int), cudaMemcpyDeviceToHost, s));
  BCK(cudaStreamSynchronize(s));
  if (sing) return b->fail(PFM_ERR_BREAKDOWN, "singular diagonal block or coarse operator in the batch");
  // Chebyshev coefficients from the eigenvalue estimates
  bool changed = false;
  std::vector<double> ab(size_t(2 * power_its));
  for (int i = 0; i < nA; ++i) {
    if (!E->hact[E->Aidx[i].first]) continue;
    for (int j = 0; j < 2 * power_its; ++j) ab[j] = E->hlz[size_t(j) * nA + i];
    const double lam = tridiag_max_eig(ab.data(), ab.data() + power_its, power_its);
    if (!(lam > 0.0) || !std::isfinite(lam))
      return b->fail(PFM_ERR_BREAKDOWN, "smoother eigenvalue estimate failed for problem " +
                                            std::to_string(E->Aidx[i].first));
    const int p = E->Aidx[i].first, l = E->Aidx[i].second;
    b->hs[p]->L[l].lam = lam;
    const float it = float(2.0 / ((E->hi + E->lo) * lam)), id = float(2.0 / ((E->hi - E->lo) * lam));
    for (auto& L : E->D[l].S)
      if (L.problem == p) {
        L.inv_theta = it;
        L.inv_delta = id;
      }
    changed = true;
  }
  if (changed)
    for (auto& Ds : E->D)
      if (!Ds.S.empty())
        BCK(cudaMemcpyAsync(Ds.dS, Ds.S.data(), sizeof(BLev) * Ds.S.size(), cudaMemcpyHostToDevice, s));
  return PFM_OK;
}

// The fixed launch sequence of FGMRES iteration j for the whole batch:
// z_j = M v_j (batched V-cycle), w = J z_j (double-float), two classical
// Gram-Schmidt passes, ||w||, Givens update and decision, next basis vector,
// solution update of finished problems, and the flag word to the host.
void eng_iteration(BatchEngine* E, int j) {
  cudaStream_t s = E->s;
  const int np = E->np;
  const int stride = BMAXM + 1;
  const dim3 gv = grid2(E->maxnO, np);
  const Gate g = E->gate_fgm();
  k_b_cast_in<<<gv, BT, 0, s>>>(E->dO, E->dF, j);
  count_launches(1);
  eng_vcycle(E, 0, g);
  k_b_store_z<<<gv, BT, 0, s>>>(E->dO, E->dF, j);
  k_b_japply_df<<<E->grid_df, 256, 0, s>>>(E->dO, E->dF, np, E->nblkO, j);
  count_launches(2);
  const dim3 gc(BCH, unsigned(np));
  for (double* h : {E->h1, E->h2}) {
    for (int j0 = 0; j0 <= j; j0 += BMDOT) {
      k_b_mdot<<<gc, BT, 0, s>>>(E->dO, E->dF, j0, std::min(BMDOT, j + 1 - j0), false, E->partial, stride);
      count_launches(1);
    }
    k_b_mdot_final<<<dim3(1, unsigned(np)), 128, 0, s>>>(E->dF, j + 1, E->partial, stride, h);
    k_b_maxpy<<<gv, BT, 0, s>>>(E->dO, E->dF, j + 1, h, stride);
    count_launches(2);
  }
  k_b_mdot<<<gc, BT, 0, s>>>(E->dO, E->dF, 0, 1, true, E->partial, stride);
  k_b_mdot_final<<<dim3(1, unsigned(np)), 128, 0, s>>>(E->dF, 1, E->partial, stride, E->hn);
  k_b_givens<<<gdiv(np, 64), 64, 0, s>>>(E->dF, np, j, E->m, E->max_lin_it, E->h1, E->h2, E->hn, stride);
  k_b_next_basis<<<gv, BT, 0, s>>>(E->dO, E->dF, j);
  k_b_update<<<gv, BT, 0, s>>>(E->dO, E->dF);
  k_b_count<<<1, 256, 0, s>>>(E->dF, np, E->flags);
  count_launches(6);
  cudaMemcpyAsync(E->hflags, E->flags, sizeof(int) * 2, cudaMemcpyDeviceToHost, s);
}

// Start a cycle for every problem with the restart flag: from r = b (x = 0,
// first cycle) or from the true residual r = b - J x (restart).
void eng_cycle_start(BatchEngine* E, bool first) {
  cudaStream_t s = E->s;
  const int np = E->np;
  const int stride = BMAXM + 1;
  const dim3 gv = grid2(E->maxnO, np);
  if (first) {
    k_b_begin<<<gv, BT, 0, s>>>(E->dO, E->dF, E->dact);
    count_launches(1);
  }
  k_b_restart_init<<<gv, BT, 0, s>>>(E->dO, E->dF);
  count_launches(1);
  if (!first) {
    k_b_japply64<<<E->grid_j64, 256, 0, s>>>(E->dO, E->dF, np, E->nblkO);
    count_launches(1);
  }
  k_b_restart_res<<<gv, BT, 0, s>>>(E->dO, E->dF);
  k_b_mdot<<<dim3(BCH, unsigned(np)), BT, 0, s>>>(E->dO, E->dF, 0, 1, true, E->partial, stride);
  k_b_mdot_final<<<dim3(1, unsigned(np)), 128, 0, s>>>(E->dF, 1, E->partial, stride, E->hn);
  k_b_cycle_state<<<gdiv(np, 64), 64, 0, s>>>(E->dF, np, E->hn, stride, first, E->rtol, E->max_lin_it);
  k_b_first_basis<<<gv, BT, 0, s>>>(E->dO, E->dF);
  k_b_count<<<1, 256, 0, s>>>(E->dF, np, E->flags);
  count_launches(6);
  cudaMemcpyAsync(E->hflags, E->flags, sizeof(int) * 2, cudaMemcpyDeviceToHost, s);
}

pfm_status eng_capture(pfm_batch* b, BatchEngine* E, int j, cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  BCK(cudaStreamBeginCapture(E->s, cudaStreamCaptureModeThreadLocal));
  const int64_t c0 = pfm_launch_count();
  eng_iteration(E, j);
  const int64_t nk = pfm_launch_count() - c0;  // counted again at every replay
  count_launches(int(-nk));
  E->itg_launches[j] = nk;
  cudaError_t e = cudaStreamEndCapture(E->s, &graph);
  if (e != cudaSuccess) return b->fail(PFM_ERR_CUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    *out = nullptr;
    return b->fail(PFM_ERR_CUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
  }
  return PFM_OK;
}

// FGMRES for every problem with hact[p] (b = -R in o.b), until all finish.
pfm_status eng_fgmres(pfm_batch* b, BatchEngine* E) {
  cudaStream_t s = E->s;
  eng_cycle_start(E, true);
  BCK(cudaGetLastError());
  BCK(cudaStreamSynchronize(s));
  int j = 0;
  if (E->itg.size() < size_t(E->m)) {
    E->itg.resize(E->m, nullptr);
    E->itg_launches.resize(E->m, 0);
  }
  // each problem runs at most max_lin_it iterations and starts a cycle at most
  // once per iteration, so a correct run makes at most 2 max_lin_it + 1 passes;
  // the loop stops after 2 (max_lin_it + m) + 8 passes (a margin over that
  // count) and reports the solver loop's non-termination as not converged
  const int64_t pass_cap = 2 * (int64_t(E->max_lin_it) + E->m) + 8;
  int64_t passes = 0;
  while (E->hflags[0] > 0 || E->hflags[1] > 0) {
    if (++passes > pass_cap)
      return b->fail(PFM_ERR_NOT_CONVERGED, "batched FGMRES did not end within its pass cap of " +
                                                std::to_string(pass_cap) + " graph launches");
    if (E->hflags[0] == 0) {  // every running cycle has ended: restart the ones that need it
      eng_cycle_start(E, false);
      BCK(cudaGetLastError());
      BCK(cudaStreamSynchronize(s));
      j = 0;
      continue;
    }
    if (j >= E->m) return b->fail(PFM_ERR_CUDA, "batched FGMRES lost track of its cycle");
    if (!E->itg[j]) TRY(eng_capture(b, E, j, &E->itg[j]));
    BCK(cudaGraphLaunch(E->itg[j], s));
    count_launches(int(E->itg_launches[j]));
    BCK(cudaStreamSynchronize(s));
    ++j;
  }
  return PFM_OK;
}

pfm_status eng_residual_norms(pfm_batch* b, BatchEngine* E) {
  cudaStream_t s = E->s;
  for (int p = 0; p < E->np; ++p) {
    if (!E->hact[p]) continue;
    pfm_handle* h = b->hs[p];
    Level& f = h->L[0];
    BCK(cudaMemsetAsync(h->R, 0, sizeof(double) * ndof(f), s));
    launch_residual(f.g, h->dp, f.U, f.Un, f.mask, h->R, nullptr, s);
  }
  k_b_res_norm2<<<dim3(BCH, unsigned(E->np)), BT, 0, s>>>(E->dO, E->dact, E->partial);
  k_b_reduce_chunks<<<gdiv(E->np, 128), 128, 0, s>>>(E->np, BCH, E->partial, E->dots);
  count_launches(2);
  BCK(cudaMemcpyAsync(E->hres, E->dots, sizeof(double) * E->np, cudaMemcpyDeviceToHost, s));
  BCK(cudaGetLastError());
  BCK(cudaStreamSynchronize(s));
  return PFM_OK;
}

// Everything the engine's descriptor tables and graphs capture: the device
// buffers of every handle and a hash of its parameters.
std::vector<uint64_t> engine_signature(const pfm_batch* b) {
  std::vector<uint64_t> sig;
  auto add = [&](const void* q) { sig.push_back(uint64_t(reinterpret_cast<uintptr_t>(q))); };
  for (const pfm_handle* h : b->hs) {
    for (const Level& lv : h->L) {
      add(lv.U); add(lv.Un); add(lv.mask); add(lv.H64); add(lv.H32); add(lv.H32lo); add(lv.D32);
      add(h->pre_h16 ? lv.H16 : nullptr);
      add(lv.x32); add(lv.b32); add(lv.y32); add(lv.r32); add(lv.d32);
    }
    add(h->V); add(h->Z); add(h->wv); add(h->dU); add(h->R); add(h->rv); add(h->Kaug); add(h->Kinv);
    add(h->gj_keys); add(h->gj_used); add(h->gj_piv);
    uint64_t x = 1469598103934665603ull;  // FNV-1a over the parameter block
    const unsigned char* c = reinterpret_cast<const unsigned char*>(&h->dp);
    for (size_t i = 0; i < sizeof(DevParams); ++i) x = (x ^ c[i]) * 1099511628211ull;
    sig.push_back(x);
  }
  return sig;
}

bool engine_matches(const BatchEngine* E, const pfm_solve_opts& o) {
  return E->m == o.restart && E->nu_pre == o.nu_pre && E->nu_post == o.nu_post && E->lo == o.cheb_lo &&
         E->hi == o.cheb_hi && E->growth == (o.nu_growth > 0 ? o.nu_growth : 1.0) &&
         E->max_lin_it == o.max_lin_it && E->rtol == o.lin_rtol;
}

}  // namespace

bool batch_engine_supports(const pfm_solve_opts& o, const pfm_batch* b) {
  if (o.precond != PFM_F32 || o.smoother != 0 || (o.cycle_gamma > 1) || o.restart > BMAXM || o.deterministic ||
      o.krylov != 0)
    return false;
  for (const pfm_handle* h : b->hs)
    if (!h->outer_df || h->contact_on || h->det || h->pre_h16 != b->hs[0]->pre_h16) return false;
  return true;
}

// Newton solve of every problem of the batch with the engine (pfm_batch_newton_solve).
pfm_status batch_engine_newton(pfm_batch* b, const pfm_solve_opts& o, double* const* U_inout,
                               pfm_solve_report* reports) {
  const int np = int(b->hs.size());
  for (int p = 0; p < np; ++p) {
    pfm_status st = engine_buffers(b->hs[p], o.restart);
    if (st != PFM_OK) return b->fail(st, "problem " + std::to_string(p) + ": " + b->hs[p]->err);
  }
  std::vector<uint64_t> sig = engine_signature(b);
  if (b->engine && (!engine_matches(b->engine, o) || b->engine->sig != sig)) {
    batch_engine_free(b->engine);
    b->engine = nullptr;
  }
  if (!b->engine) {
    TRY(engine_build(b, o, &b->engine));
    b->engine->sig = sig;
  }
  const double t_start = now_ms();
  BatchEngine* E = b->engine;
  cudaStream_t s = E->s;
  std::vector<pfm_solve_report> rep(np);
  for (int p = 0; p < np; ++p) {
    pfm_handle* h = b->hs[p];
    Level& f = h->L[0];
    BCK(cudaMemcpyAsync(f.U, U_inout[p], sizeof(double) * ndof(f), cudaMemcpyDeviceToDevice, s));
    if (h->have_dirval) launch_mask_values(f.nn, f.mask, h->dirval, f.U, s);
    h->linearized = false;
    E->hact[p] = 1;
  }
  BCK(cudaMemcpyAsync(E->dact, E->hact, sizeof(int) * np, cudaMemcpyHostToDevice, s));
  double t0 = now_ms();
  TRY(eng_residual_norms(b, E));
  std::vector<double> res(np);
  for (int p = 0; p < np; ++p) {
    res[p] = std::sqrt(E->hres[p]);
    rep[p].res0 = res[p];
    rep[p].ms_residual += now_ms() - t0;
  }
  std::vector<BFgm> Fh(np);
  for (int it = 0; it < o.max_newton; ++it) {
    int nact = 0;
    for (int p = 0; p < np; ++p) {
      bool a = true;
      if (!std::isfinite(res[p])) {
        rep[p].status = PFM_ERR_NONFINITE;
        a = false;
      } else if (res[p] == 0.0 || (it > 0 && res[p] <= o.newton_rtol * rep[p].res0)) {
        a = false;
      }
      E->hact[p] = a ? 1 : 0;
      nact += a;
    }
    if (nact == 0) break;
    BCK(cudaMemcpyAsync(E->dact, E->hact, sizeof(int) * np, cudaMemcpyHostToDevice, s));
    t0 = now_ms();
    TRY(eng_linearize(b, E, b->hs[0]->power_its));
    const double ms_lin = now_ms() - t0;
    t0 = now_ms();
    k_b_negate<<<grid2(E->maxnO, np), BT, 0, s>>>(E->dO, E->dact);
    count_launches(1);
    TRY(eng_fgmres(b, E));
    k_b_newton_update<<<grid2(E->maxnO, np), BT, 0, s>>>(E->dO, E->dact);
    count_launches(1);
    BCK(cudaMemcpy2DAsync(Fh.data(), sizeof(BFgm), E->dF, sizeof(BFgm), offsetof(BFgm, H), np,
                          cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    const double ms_solve = now_ms() - t0;
    for (int p = 0; p < np; ++p) {
      if (!E->hact[p]) continue;
      rep[p].ms_linearize += ms_lin;
      rep[p].ms_solve += ms_solve;
      rep[p].lin_its_total += Fh[p].total;
      rep[p].lin_its_last = Fh[p].total;
      rep[p].lin_res_final = Fh[p].relres;
      if (Fh[p].status == BF_NONFINITE) rep[p].status = PFM_ERR_NONFINITE;
      else if (Fh[p].status == BF_BREAKDOWN) rep[p].status = PFM_ERR_BREAKDOWN;
      else if (!Fh[p].converged) rep[p].status = PFM_ERR_NOT_CONVERGED;
      ++rep[p].newton_its;
    }
    t0 = now_ms();
    TRY(eng_residual_norms(b, E));
    for (int p = 0; p < np; ++p)
      if (E->hact[p]) {
        res[p] = std::sqrt(E->hres[p]);
        rep[p].ms_residual += now_ms() - t0;
      }
  }
  for (int p = 0; p < np; ++p) {
    pfm_handle* h = b->hs[p];
    BCK(cudaMemcpyAsync(U_inout[p], h->L[0].U, sizeof(double) * ndof(h->L[0]), cudaMemcpyDeviceToDevice, s));
    rep[p].res_final = res[p];
    if (rep[p].status == PFM_OK && o.max_newton > 1 && !(res[p] <= o.newton_rtol * rep[p].res0) && res[p] != 0.0)
      rep[p].status = PFM_ERR_NOT_CONVERGED;
    h->linearized = false;
  }
  BCK(cudaStreamSynchronize(s));
  const double total = now_ms() - t_start;
  for (int p = 0; p < np; ++p) rep[p].ms_total = total;
  if (reports)
    for (int p = 0; p < np; ++p) reports[p] = rep[p];
  for (int p = 0; p < np; ++p)
    if (rep[p].status != PFM_OK) return b->fail(rep[p].status, "problem " + std::to_string(p) + " did not converge");
  return PFM_OK;
}

}  // namespace pfm
