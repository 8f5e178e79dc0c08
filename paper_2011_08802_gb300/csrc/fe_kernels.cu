// Element kernels on the structured trilinear-hexahedron grid: residual
// (Sec. 3.4, Eq. FinalRes), linearisation into Gauss-point Hessians (the
// tangent of Eq. linAlgEq), matrix-free tangent application, nodal 9x9
// diagonal blocks for point-block Jacobi (Sec. 3.4) and their inverses.
//
// Thread mapping: 8 consecutive lanes form one element; lane l8 = 0..7 plays
// two roles: local node a = l8 (corner (a&1, a>>1&1, a>>2)) when gathering
// nodal data or scattering nodal results, and Gauss point q = l8 (point
// ((1 -+ 1/sqrt 3)/2) per axis) for the point physics. Values and gradients
// at the 8 points are a tensor product of 1-D 2x2 transforms, applied with
// three xor-shuffles (1, 2, 4) per axis; the scatter is the transposed
// transform. A warp holds 4 elements.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "fe_device.cuh"

namespace pfm {
namespace {

// ---------------------------------------------------------------------------
// Residual (and energy) of the elements, the point physics in TC (FP64, or
// double-float: pairs of FP32 numbers on the FP32 pipes, about 48 bits);
// DET: atomic-free, the nodal results go to the scratch W (node_gather adds
// them up) and each warp's energy to W[9 ws + blk] (summed in a fixed order
// by k_sum_fixed).
#ifndef PFM_RES_MINB
#define PFM_RES_MINB 2
#endif
// Residual rows and energy of one Gauss point (lane = 8 e + q of block blk)
// from its eta gradients ge, energy gradient gr and energy density Wd: the
// gradient-energy flux G grad eta, the nodal rows scattered (DET: to the
// scratch W) with Dirichlet rows left out, the energy summed per warp.
template <typename TC, bool DET>
__device__ __forceinline__ void residual_tail(const Grid& g, const DevParams& P, const TC* ge, const TC* gr, TC Wd,
                                              int64_t node, bool valid, int l8, int64_t blk, int lane,
                                              const dmask_t* __restrict__ mask, double* __restrict__ R,
                                              double* energy, double* __restrict__ W, int64_t ws) {
  const int64_t nn = g.nn();
  const TC ihx = TC(1.0 / g.hx), ihy = TC(1.0 / g.hy), ihz = TC(1.0 / g.hz);
  TC gf[3 * NV];
  TC Wg = TC(0.0);
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      TC s = TC(0.0);
#pragma unroll
      for (int l = 0; l < NV; ++l) s += TC(P.G[k][l]) * ge[3 * l + d];
      gf[3 * k + d] = s;
      Wg += TC(0.5) * ge[3 * k + d] * s;
    }
  const TC w = TC(g.w());
  const dmask_t dm = valid ? mask[node] : dmask_t(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    TC r = q1_scatter_grad(w * gr[3 * i], w * gr[3 * i + 1], w * gr[3 * i + 2], l8, ihx, ihy, ihz);
    scatter_row<DET>(R, W, ws, i, blk, lane, i * nn + node, double(r), valid && !((dm >> i) & 1));
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    TC r = q1_scatter(w * gr[9 + k], w * gf[3 * k], w * gf[3 * k + 1], w * gf[3 * k + 2], l8, ihx,
                      ihy, ihz);
    scatter_row<DET>(R, W, ws, 3 + k, blk, lane, (3 + k) * nn + node, double(r),
                     valid && !((dm >> (3 + k)) & 1));
  }
  if (energy) {
    double en = warp_sum(valid ? double(w * (Wd + Wg)) : 0.0);
    if constexpr (DET) {
      if (lane == 0) W[NF * ws + blk] = en;
    } else {
      if (lane == 0) atomicAdd(energy, en);
    }
  }
}

// Out-of-line copy for the linearisation pass, so that the register
// allocation of its point physics does not see the residual's scatter.
template <typename TC, bool DET>
__device__ __noinline__ void residual_tail_call(const Grid& g, const DevParams& P, const TC* ge, const TC* gr, TC Wd,
                                                int64_t node, bool valid, int l8, int64_t blk, int lane,
                                                const dmask_t* __restrict__ mask, double* __restrict__ R,
                                                double* energy, double* __restrict__ W, int64_t ws) {
  residual_tail<TC, DET>(g, P, ge, gr, Wd, node, valid, l8, blk, lane, mask, R, energy, W, ws);
}

template <typename TC, bool DET>
__global__ void __launch_bounds__(128, PFM_RES_MINB) k_residual(Grid g, DevParams P, const double* __restrict__ U,
                                                  const double* __restrict__ Un,
                                                  const dmask_t* __restrict__ mask,
                                                  double* __restrict__ R, double* energy, double* __restrict__ W,
                                                  int64_t ws) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t e = tid >> 3;
  const int l8 = int(tid & 7);
  const int64_t blk = tid >> 5;
  const int lane = int(tid & 31);
  const bool valid = e < g.ne();
  const int64_t nn = g.nn();
  const int64_t node = valid ? elem_node(g, e, l8) : 0;
  const TC ihx = TC(1.0 / g.hx), ihy = TC(1.0 / g.hy), ihz = TC(1.0 / g.hz);
  TC F[9], eh[NV], ge[3 * NV], ehn[NV];
  gather_state<TC>(U, nn, node, valid, l8, ihx, ihy, ihz, F, eh, ge);
#pragma unroll
  for (int k = 0; k < NV; ++k) ehn[k] = q1_value(valid ? TC(Un[(3 + k) * nn + node]) : TC(0.0));
  TC Wd, gr[NZ];
  qp_local<TC, false>(P, F, eh, ehn, &Wd, gr, nullptr);
  residual_tail<TC, DET>(g, P, ge, gr, Wd, node, valid, l8, blk, lane, mask, R, energy, W, ws);
}

// Node pass of the atomic-free scatter (node_gather) over all nodes.
template <typename TW, typename TV, typename TY>
__global__ void __launch_bounds__(128) k_node_gather(Grid g, const TW* __restrict__ W, int64_t ws,
                                                     const dmask_t* __restrict__ mask, const TV* __restrict__ v,
                                                     TY* __restrict__ y) {
  const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= g.nn()) return;
  node_gather<TW, TV, TY>(g, W, ws, mask, v, y, n);
}

// *out += sum of x[0..n) in a fixed order: one CTA of 1024 threads, thread t
// sums x[t], x[t + 1024], ... in order, then a fixed shared-memory tree.
__global__ void __launch_bounds__(1024) k_sum_fixed(int64_t n, const double* __restrict__ x, double* out) {
  __shared__ double part[1024];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 1024) s += x[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int h = 512; h > 0; h >>= 1) {
    if (int(threadIdx.x) < h) part[threadIdx.x] += part[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out += part[0];
}

// Gauss-point Hessians of one level, computed in TC (FP64 for the finest and
// the coarsest level, FP32 for the intermediate levels of an FP32
// preconditioner) and stored in the requested precisions. Warps walk the
// element blocks with a grid stride, so the launch can bound the number of
// resident threads (and with it the footprint of the per-thread stack of the
// point physics, which then stays in L2).
// RES (FP64 only): the same pass also forms the residual and energy of the
// state (as k_residual: atomics into R and *energy, or with RW set the
// atomic-free scratch for the node pass); a separate instance, so that the
// plain linearisation keeps its own register allocation.
template <typename TC, bool RES = false>
__global__ void __launch_bounds__(128) k_linearize(Grid g, DevParams P, const double* __restrict__ U,
                                                   const double* __restrict__ Un,
                                                   double* __restrict__ H64, float* __restrict__ H32,
                                                   float* __restrict__ H32lo, const dmask_t* __restrict__ mask,
                                                   double* __restrict__ R, double* energy,
                                                   double* __restrict__ RW) {
  const int64_t w0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int lane = int(threadIdx.x & 31);
  for (int64_t blk = w0; blk < g.nblk(); blk += nw) {  // whole warps only (padding lanes stay)
    if constexpr (RES) {
      static_assert(std::is_same<TC, double>::value, "residual pass in FP64 only");
      const int64_t ws = g.nblk() * 32;
      linearize_lane<TC>(g, P, U, Un, H64, H32, H32lo, blk, lane,
                         [&](const TC* ge, const TC* gr, TC Wd, int64_t node, bool valid, int l8) {
                           if (RW)
                             residual_tail_call<TC, true>(g, P, ge, gr, Wd, node, valid, l8, blk, lane, mask, R,
                                                          energy, RW, ws);
                           else
                             residual_tail_call<TC, false>(g, P, ge, gr, Wd, node, valid, l8, blk, lane, mask,
                                                           R, energy, nullptr, 0);
                         });
    } else {
      linearize_lane<TC>(g, P, U, Un, H64, H32, H32lo, blk, lane);
    }
  }
}

// Resident CTAs per SM of the FP64-class linearisation (0: one warp per
// element block, as many CTAs as that takes).
#ifndef PFM_LIN_CTAS_PER_SM
#define PFM_LIN_CTAS_PER_SM 0
#endif

// ---- BEGIN tangent application kernel
// Bulk prefetch of a contiguous global range into L2 by the bulk-copy engine
// (no registers or shared memory involved); address 16-byte aligned, size a
// multiple of 16 bytes.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// y += J v over the elements (y initialised by k_japply_init, or the
// atomic-free form with the scratch W). Persistent warps walk the element
// blocks (4 elements each) with a grid stride; before a warp reads a block's
// Hessians (15 KB in FP32, 30 vector loads per lane) lane 0 requests the
// whole block into L2 with one bulk prefetch, so the block's DRAM reads are
// in flight at once instead of one vector load after the other (measured at
// 128^3: 1.27 against 1.39 ms per FP32 application).
#ifndef PFM_JAPPLY_MINB
#define PFM_JAPPLY_MINB 2
#endif
template <typename T>
__global__ void __launch_bounds__(256, PFM_JAPPLY_MINB) k_japply(Grid g, JParams<T> jp, const T* __restrict__ H,
                                                const dmask_t* __restrict__ mask,
                                                const T* __restrict__ v, T* __restrict__ y) {
  const int64_t nblk = g.nblk();
  const int64_t wg = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int lane = int(threadIdx.x & 31);
  constexpr unsigned BLK_BYTES = unsigned(HBLK * sizeof(T));
  static_assert(BLK_BYTES % 16 == 0, "bulk prefetch size");
  for (int64_t blk = wg; blk < nblk; blk += nw) {
    if (lane == 0) prefetch_l2(H + blk * HBLK, BLK_BYTES);
    japply_block<T>(g, jp, H, mask, v, y, blk, lane);
  }
}

// The atomic-free form (deterministic mode): the same walk, element results
// to the scratch W (9 x 32 x nblk entries) for the node pass.
template <typename T>
__global__ void __launch_bounds__(256, PFM_JAPPLY_MINB) k_japply_det(Grid g, JParams<T> jp, const T* __restrict__ H,
                                                                     const dmask_t* __restrict__ mask,
                                                                     const T* __restrict__ v, T* __restrict__ W,
                                                                     int64_t ws) {
  const int64_t nblk = g.nblk();
  const int64_t wg = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int lane = int(threadIdx.x & 31);
  constexpr unsigned BLK_BYTES = unsigned(HBLK * sizeof(T));
  for (int64_t blk = wg; blk < nblk; blk += nw) {
    if (lane == 0) prefetch_l2(H + blk * HBLK, BLK_BYTES);
    japply_block_det<T>(g, jp, H, mask, v, W, ws, blk, lane);
  }
}

// ---- END tangent application kernel

// Same persistent mapping over a binary16 copy of the store (s H, wh = w / s).
// Its resident-CTA bound is set apart from the FP32/FP64 kernel's: with half
// the bytes per element it is limited by per-element work, not by the store.
#ifndef PFM_JAPPLY_H16_MINB
#define PFM_JAPPLY_H16_MINB PFM_JAPPLY_MINB
#endif
// bulk L2 prefetch of each element block's binary16 Hessians (off: measured
// slower for this kernel, which is limited by its per-element work)
#ifndef PFM_H16_PREFETCH
#define PFM_H16_PREFETCH 0
#endif
template <bool DET>
__global__ void __launch_bounds__(256, PFM_JAPPLY_H16_MINB) k_japply_h16(Grid g, JParams<float> jp, float wh,
                                                    const __half* __restrict__ H,
                                                    const dmask_t* __restrict__ mask,
                                                    const float* __restrict__ v, float* __restrict__ y,
                                                    float* __restrict__ W, int64_t ws) {
  const int64_t nblk = g.nblk();
  const int64_t wg = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int lane = int(threadIdx.x & 31);
#if PFM_H16_PREFETCH
  constexpr unsigned BLK_BYTES = unsigned(HBLK * sizeof(__half));
  for (int64_t blk = wg; blk < nblk; blk += nw) {
    if (lane == 0) prefetch_l2(H + blk * HBLK, BLK_BYTES);
    japply_block_h16<DET>(g, jp, wh, H, mask, v, y, blk, lane, W, ws);
  }
#else
  for (int64_t blk = wg; blk < nblk; blk += nw) japply_block_h16<DET>(g, jp, wh, H, mask, v, y, blk, lane, W, ws);
#endif
}

// ---- BEGIN staged tangent application kernel
// y += J v (FP32 arithmetic) with the Hessian store S (FP32, or the binary16
// copy s H) staged in shared memory by bulk copies. Warp w of the grid takes
// element blocks w, w + nw, w + 2 nw, ...; its lane 0 keeps D blocks in
// flight, each a bulk copy of HBLK entries into one of the warp's D stages
// with completion counted on that stage's mbarrier, and re-arms a stage as
// soon as the warp has consumed it. The reads of the store are thus D - 1 to
// D blocks ahead of the arithmetic whatever the warp's registers, and the
// Dirichlet masks and input values of the next block are loaded while the
// current one computes. A wait longer than
// WAIT_LIMIT_NS gives up: the warp waits (with the same bound) for its other
// copies, counts the event in g_wait_timeouts and writes NaN into y[0],
// which the solver's finiteness checks report.
__device__ int g_wait_timeouts = 0;
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;

// resident CTAs per SM that the shared memory of one shape allows, at most 20
// warps per SM (the binary16 body fits in 96 registers without spills, the
// FP32 body needs about 125 and is limited by shared memory first): the
// register bound of the launch
template <typename S, int D, int WPC>
constexpr int staged_minb() {
  constexpr int per = WPC * D * int(HBLK * sizeof(S)) + 1024;
  constexpr int n = (227 * 1024) / per;
  constexpr int cap = 20 / WPC;
  return n < 1 ? 1 : (n > cap ? cap : n);
}

template <typename S, int D, int WPC>
__global__ void __launch_bounds__(32 * WPC, (staged_minb<S, D, WPC>())) k_japply_tma(
    Grid g, JStaged jp, const S* __restrict__ H, const dmask_t* __restrict__ mask, const float* __restrict__ v,
    float* __restrict__ y) {
  constexpr unsigned STAGE = unsigned(HBLK * sizeof(S));
  static_assert(STAGE % 16 == 0, "bulk copy size");
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[WPC * D];
  const int lane = int(threadIdx.x & 31);
  const int wid = int(threadIdx.x >> 5);
  unsigned char* st = smem + size_t(wid) * D * STAGE;
  uint64_t* fb = bars + wid * D;
  const int64_t nblk = g.nblk();
  const int64_t w0 = int64_t(blockIdx.x) * WPC + wid;
  const int64_t nw = int64_t(gridDim.x) * WPC;
  if (w0 >= nblk) return;  // the whole warp, before any barrier is in use
  uint64_t pol = 0;
  if (lane == 0) {
#pragma unroll
    for (int s = 0; s < D; ++s) mbar_init(fb + s, 1);
    fence_mbar_init();
    pol = l2_evict_first_policy();
#pragma unroll
    for (int s = 0; s < D; ++s) {
      const int64_t b = w0 + s * nw;
      if (b < nblk) {
        mbar_arrive_expect_tx(fb + s, STAGE);
        bulk_g2s(st + s * STAGE, H + b * HBLK, STAGE, fb + s, pol);
      }
    }
  }
  __syncwarp();
  StagedLane nxt;
  staged_load(g, jp, mask, v, w0, lane, nxt);
  unsigned i = 0;
  for (int64_t blk = w0; blk < nblk; blk += nw, ++i) {
    const int s = int(i % D);
    const unsigned par = (i / D) & 1u;
    StagedLane sl = nxt;
    // the next block's mask and input values load while this block computes
    if (blk + nw < nblk) staged_load(g, jp, mask, v, blk + nw, lane, nxt);
    float dz[NZ], ge[3 * NV];
    staged_shuffle(jp, sl, lane, dz, ge);
    if (!mbar_wait_warp(fb + s, par, WAIT_LIMIT_NS)) {
      // outstanding copies: those of blocks i .. i + D - 1 of this warp
      for (int t = 0; t < D; ++t)
        if (blk + t * nw < nblk) mbar_wait_warp(fb + (i + t) % D, ((i + t) / D) & 1u, WAIT_LIMIT_NS);
      if (lane == 0) {
        atomicAdd(&g_wait_timeouts, 1);
        y[0] = __int_as_float(0x7fc00000);
      }
      return;
    }
    staged_contract_scatter<S>(g, jp, st + s * STAGE, sl, y, lane, dz, ge);
    __syncwarp();
    if (lane == 0) {
      const int64_t nb = blk + D * nw;
      if (nb < nblk) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(fb + s, STAGE);
        bulk_g2s(st + s * STAGE, H + nb * HBLK, STAGE, fb + s, pol);
      }
    }
  }
}
// ---- END staged tangent application kernel

// y += J v with v in FP32 (exact input), the tangent as Hhi + Hlo (two FP32
// stores of the FP64 Hessians) and double-float arithmetic throughout; the
// element contributions are added to the FP64 output y (initialised by
// k_japply_init_df). Same persistent warp mapping as k_japply.
#ifndef PFM_DF_MINB
#define PFM_DF_MINB (PFM_NV == 6 ? 2 : 8)
#endif
template <bool DET>
__global__ void __launch_bounds__(256, PFM_DF_MINB) k_japply_df(Grid g, DfConst k, const float* __restrict__ Hhi,
                                                     const float* __restrict__ Hlo,
                                                     const dmask_t* __restrict__ mask,
                                                     const float* __restrict__ v, double* __restrict__ y,
                                                     double* __restrict__ W, int64_t ws) {
  const int64_t nblk = g.nblk();
  const int64_t wg = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int lane = int(threadIdx.x & 31);
  for (int64_t blk = wg; blk < nblk; blk += nw) japply_df_block<DET>(g, k, Hhi, Hlo, mask, v, y, blk, lane, W, ws);
}

// y = v at Dirichlet DOFs, 0 elsewhere (FP32 input, FP64 output).
__global__ void k_japply_init_df(int64_t nn, const dmask_t* __restrict__ mask, const float* __restrict__ v,
                                 double* __restrict__ y) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < NF * nn;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t node = i % nn;
    const int f = int(i / nn);
    y[i] = ((mask[node] >> f) & 1) ? double(v[i]) : 0.0;
  }
}

// y = v at Dirichlet DOFs (identity rows), 0 elsewhere.
template <typename T>
__global__ void k_japply_init(int64_t nn, const dmask_t* __restrict__ mask, const T* __restrict__ v,
                              T* __restrict__ y) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < NF * nn;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t node = i % nn;
    const int f = int(i / nn);
    y[i] = ((mask[node] >> f) & 1) ? v[i] : T(0);
  }
}

// Nodal 9x9 diagonal blocks in two passes without atomics. Pass 1: one warp
// per element block stages the block's Gauss-point Hessians in shared memory
// (one coalesced read of the store) and thread (element, local node a) writes
// that element's 45-entry contribution to node a into W[t][blk*32 + lane].
template <typename T>
__global__ void __launch_bounds__(128) k_blockdiag_elem(Grid g, JParams<T> jp, const T* __restrict__ H,
                                                        T* __restrict__ W) {
  extern __shared__ __align__(16) unsigned char bd_smem[];
  constexpr int V = 16 / sizeof(T);
  using VT = typename Vec16<T>::type;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t blk = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (blk >= g.nblk()) return;
  VT* S = reinterpret_cast<VT*>(bd_smem) + int64_t(wid) * (HBLK / V);
  const VT* src = reinterpret_cast<const VT*>(H) + blk * (HBLK / V);
  for (int i = lane; i < int(HBLK / V); i += 32) S[i] = src[i];
  __syncwarp();
  T Db[NBD];
#pragma unroll
  for (int t = 0; t < NBD; ++t) Db[t] = T(0);
  const int64_t e = blk * 4 + (lane >> 3);
  if (e < g.ne()) blockdiag_accumulate<T>(jp, reinterpret_cast<const T*>(S), 0, (lane >> 3) * 8, lane & 7, Db);
  const int64_t stride = g.nblk() * 32;
#pragma unroll
  for (int t = 0; t < NBD; ++t) W[t * stride + blk * 32 + lane] = Db[t];
}

// Pass 2: node n sums the contributions of its (up to 8) adjacent elements in
// a fixed order and writes its whole block.
template <typename T>
__global__ void __launch_bounds__(128) k_blockdiag_node(Grid g, const T* __restrict__ W, T* __restrict__ D) {
  const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nn = g.nn();
  if (n >= nn) return;
  const int i = int(n % (g.nx + 1));
  const int j = int((n / (g.nx + 1)) % (g.ny + 1));
  const int k = int(n / (int64_t(g.nx + 1) * (g.ny + 1)));
  const int64_t stride = g.nblk() * 32;
  T Db[NBD];
#pragma unroll
  for (int t = 0; t < NBD; ++t) Db[t] = T(0);
  for (int dk = 0; dk < 2; ++dk) {
    const int ek = k - 1 + dk;
    if (ek < 0 || ek >= g.nz) continue;
    for (int dj = 0; dj < 2; ++dj) {
      const int ej = j - 1 + dj;
      if (ej < 0 || ej >= g.ny) continue;
      for (int di = 0; di < 2; ++di) {
        const int ei = i - 1 + di;
        if (ei < 0 || ei >= g.nx) continue;
        const int64_t e = ei + int64_t(g.nx) * (ej + int64_t(g.ny) * ek);
        const int a = (1 - di) + 2 * (1 - dj) + 4 * (1 - dk);
        const int64_t col = (e >> 2) * 32 + (e & 3) * 8 + a;
#pragma unroll
        for (int t = 0; t < NBD; ++t) Db[t] += W[t * stride + col];
      }
    }
  }
  int idx = 0;
#pragma unroll
  for (int r = 0; r < NF; ++r)
#pragma unroll
    for (int c = r; c < NF; ++c) {
      D[(r * NF + c) * nn + n] = Db[idx];
      if (c != r) D[(c * NF + r) * nn + n] = Db[idx];
      ++idx;
    }
}

// In-place inverse of each node's 9x9 block (block_invert_node).
template <typename T>
__global__ void k_block_invert(int64_t nn, const dmask_t* __restrict__ mask, T* __restrict__ D,
                               int* singular) {
  const int64_t node = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (node >= nn) return;
  block_invert_node<T>(nn, mask, D, singular, node);
}

__global__ void k_qp_eval(DevParams P, int64_t n, const double* __restrict__ F,
                          const double* __restrict__ eta, const double* __restrict__ eta_n,
                          double* __restrict__ W, double* __restrict__ grad, double* __restrict__ hess) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double Fl[9], e[NV], en[NV], w, g[NZ], h[NH];
  for (int k = 0; k < 9; ++k) Fl[k] = F[i * 9 + k];
  for (int k = 0; k < NV; ++k) { e[k] = eta[i * NV + k]; en[k] = eta_n[i * NV + k]; }
  qp_local<double, true>(P, Fl, e, en, &w, g, h);
  if (W) W[i] = w;
  if (grad)
    for (int k = 0; k < NZ; ++k) grad[i * NZ + k] = g[k];
  if (hess)
    for (int k = 0; k < NH; ++k) hess[i * NH + k] = h[k];
}

// max |H| over an FP32 store (non-negative floats order as their bit
// patterns, so an integer atomicMax on the bits is a float max; a NaN entry
// gives +infinity).
__global__ void k_absmax(int64_t n, const float* __restrict__ H, unsigned* __restrict__ out) {
  float m = 0.f;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    m = absmax_step(m, H[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// binary16 copy of an FP32 store scaled by s (a power of two): one thread
// per 16-byte output vector (8 entries of one lane), read as two FP32 vectors
// of the same lane.
__global__ void k_store_to_half(int64_t nvec, const float4* __restrict__ H32, float s, uint4* __restrict__ H16) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nvec; i += int64_t(gridDim.x) * blockDim.x)
    H16[i] = half_vector(H32, s, i);
}

inline unsigned grid_for(int64_t threads, int block) {
  return unsigned((threads + block - 1) / block);
}

// y += J v over element blocks [b0, b1) (persistent warps; the slab
// pipeline of the host-buffer entry point).
template <typename T>
__global__ void __launch_bounds__(256, PFM_JAPPLY_MINB) k_japply_range(Grid g, JParams<T> jp, const T* __restrict__ H,
                                                      const dmask_t* __restrict__ mask, const T* __restrict__ v,
                                                      T* __restrict__ y, int64_t b0, int64_t b1) {
  const int64_t wg = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int lane = int(threadIdx.x & 31);
  constexpr unsigned BLK_BYTES = unsigned(HBLK * sizeof(T));
  for (int64_t blk = b0 + wg; blk < b1; blk += nw) {
    if (lane == 0) prefetch_l2(H + blk * HBLK, BLK_BYTES);
    japply_block<T>(g, jp, H, mask, v, y, blk, lane);
  }
}

// y = v at the Dirichlet DOFs of nodes [n0, n1) (their rows are identity;
// element contributions skip them).
template <typename T>
__global__ void k_identity_rows(int64_t nn, const dmask_t* __restrict__ mask, const T* __restrict__ v,
                                T* __restrict__ y, int64_t n0, int64_t n1) {
  const int64_t span = n1 - n0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < NF * span; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t node = n0 + i % span;
    const int f = int(i / span);
    if ((mask[node] >> f) & 1) y[f * nn + node] = v[f * nn + node];
  }
}

}  // namespace

int sm_count();

void launch_residual(const Grid& g, const DevParams& P, const double* U, const double* Un,
                     const dmask_t* mask, double* R, double* energy, cudaStream_t s, double* W, bool df) {
  const int64_t threads = g.nblk() * 32;
  if (!W) {
    if (df)
      k_residual<df64, false><<<grid_for(threads, 128), 128, 0, s>>>(g, P, U, Un, mask, R, energy, nullptr, 0);
    else
      k_residual<double, false><<<grid_for(threads, 128), 128, 0, s>>>(g, P, U, Un, mask, R, energy, nullptr, 0);
    count_launches(1);
    return;
  }
  const int64_t ws = g.nblk() * 32;
  if (df)
    k_residual<df64, true><<<grid_for(threads, 128), 128, 0, s>>>(g, P, U, Un, mask, R, energy, W, ws);
  else
    k_residual<double, true><<<grid_for(threads, 128), 128, 0, s>>>(g, P, U, Un, mask, R, energy, W, ws);
  k_node_gather<double, double, double><<<grid_for(g.nn(), 128), 128, 0, s>>>(g, W, ws, mask, nullptr, R);
  count_launches(2);
  if (energy) {
    k_sum_fixed<<<1, 1024, 0, s>>>(g.nblk(), W + NF * ws, energy);
    count_launches(1);
  }
}

void launch_linearize(const Grid& g, const DevParams& P, const double* U, const double* Un,
                      double* H64, float* H32, float* H32lo, int arith, cudaStream_t s, const LinResidual* res) {
  const int64_t threads = g.nblk() * 32;
  unsigned blocks = grid_for(threads, 128);
  if (arith != LIN_F32 && PFM_LIN_CTAS_PER_SM > 0) {
    const int64_t cap = int64_t(sm_count()) * PFM_LIN_CTAS_PER_SM;
    if (int64_t(blocks) > cap) blocks = unsigned(cap);
  }
  // the residual is formed in the FP64 pass only
  const bool with_res = res && res->R && arith == LIN_F64;
  const dmask_t* mask = with_res ? res->mask : nullptr;
  double* R = with_res ? res->R : nullptr;
  double* energy = with_res ? res->energy : nullptr;
  double* RW = with_res ? res->W : nullptr;
  if (arith == LIN_F32)
    k_linearize<float><<<blocks, 128, 0, s>>>(g, P, U, Un, H64, H32, H32lo, nullptr, nullptr, nullptr, nullptr);
  else if (arith == LIN_DF)
    k_linearize<df64><<<blocks, 128, 0, s>>>(g, P, U, Un, H64, H32, H32lo, nullptr, nullptr, nullptr, nullptr);
  else if (with_res)
    k_linearize<double, true><<<blocks, 128, 0, s>>>(g, P, U, Un, H64, H32, H32lo, mask, R, energy, RW);
  else
    k_linearize<double><<<blocks, 128, 0, s>>>(g, P, U, Un, H64, H32, H32lo, nullptr, nullptr, nullptr, nullptr);
  count_launches(1);
  if (RW) {  // node pass of the atomic-free form, as in launch_residual
    const int64_t ws = g.nblk() * 32;
    k_node_gather<double, double, double><<<grid_for(g.nn(), 128), 128, 0, s>>>(g, RW, ws, mask, nullptr, R);
    count_launches(1);
    if (energy) {
      k_sum_fixed<<<1, 1024, 0, s>>>(g.nblk(), RW + NF * ws, energy);
      count_launches(1);
    }
  }
}

// ---------------------------------------------------------------------------
// Launch-shape autotuner of the tangent application. A launch shape is the
// element tile of one CTA (threads/8 elements: 16 or 32) and the number of
// resident CTAs per SM of the persistent grid. The first application for a
// (precision, size class = floor(log2 element blocks)) key times every
// candidate three times with events and keeps the fastest; the choice is
// cached for the process and, when PFM_AUTOTUNE_FILE names a file, read from
// and written back to it as JSON (format below). No tuning runs while the
// stream is being captured into a graph (the default shape is used).
struct JShape {
  int threads = 256;
  int per_sm = 2;
  double ms = 0.0;  // timed milliseconds per application (0 = not timed)
  int stages = 0;   // > 0: the staged kernel k_japply_tma with this many stages per warp
};

// Shapes of the staged kernel (stages per warp D, threads = 32 x warps per CTA).
constexpr int STAGED_SHAPES[][2] = {{2, 128}, {3, 128}, {2, 64}, {2, 32}, {1, 128}};
bool staged_shape_known(int stages, int threads) {
  for (const auto& sh : STAGED_SHAPES)
    if (sh[0] == stages && sh[1] == threads) return true;
  return false;
}

std::mutex g_tune_mutex;
std::map<std::pair<int, int>, JShape> g_tuned;
bool g_tune_file_read = false;

// The cache file (PFM_AUTOTUNE_FILE) is a JSON array with one object per line:
//   {"kernel": "k_japply", "precision": "f32", "size_class": 17, "threads": 256,
//    "ctas_per_sm": 2, "stages": 0, "ms_per_application": 1.2713}
// (stages 0: the register-fed kernel; 2 or 3: the staged kernel with that
// many shared-memory stages per warp)
void tune_file_read() {
  if (g_tune_file_read) return;
  g_tune_file_read = true;
  const char* path = std::getenv("PFM_AUTOTUNE_FILE");
  if (!path) return;
  std::FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[512];
  while (std::fgets(line, sizeof(line), f)) {
    char prec[8] = {0};
    int cl, th, ps, stg;
    double ms = 0.0;
    if (std::sscanf(line,
                    " {\"kernel\": \"k_japply\", \"precision\": \"%3[f0-9]\", \"size_class\": %d, \"threads\": %d, "
                    "\"ctas_per_sm\": %d, \"stages\": %d, \"ms_per_application\": %lf",
                    prec, &cl, &th, &ps, &stg, &ms) == 6) {
      const int pr = std::strcmp(prec, "f32") == 0   ? 0
                     : std::strcmp(prec, "f64") == 0 ? 1
                     : std::strcmp(prec, "f16") == 0 ? 2
                                                     : -1;
      const bool classic = stg == 0 && (th == 128 || th == 256);
      const bool staged = pr != 1 && staged_shape_known(stg, th);
      if (pr >= 0 && (classic || staged) && ps >= 1 && ps <= 16) g_tuned[{pr, cl}] = JShape{th, ps, ms, stg};
    }
  }
  std::fclose(f);
}

// rewrite the whole cache (entries of this process merged with what was read)
void tune_file_write() {
  const char* path = std::getenv("PFM_AUTOTUNE_FILE");
  if (!path) return;
  std::FILE* f = std::fopen(path, "w");
  if (!f) return;
  std::fprintf(f, "[\n");
  size_t i = 0;
  for (const auto& kv : g_tuned) {
    std::fprintf(f,
                 " {\"kernel\": \"k_japply\", \"precision\": \"%s\", \"size_class\": %d, \"threads\": %d, "
                 "\"ctas_per_sm\": %d, \"stages\": %d, \"ms_per_application\": %.6f}%s\n",
                 kv.first.first == 0 ? "f32" : (kv.first.first == 1 ? "f64" : "f16"), kv.first.second,
                 kv.second.threads, kv.second.per_sm, kv.second.stages,
                 kv.second.ms, ++i < g_tuned.size() ? "," : "");
  }
  std::fprintf(f, "]\n");
  std::fclose(f);
}

int sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  return sms;
}

// ---- staged tangent application (k_japply_tma) ----
JStaged make_jstaged(const Grid& g, const DevParams& P, double wh) {
  JStaged j;
  const double w = g.w();
  for (int k = 0; k < NV; ++k)
    for (int l = 0; l < NV; ++l) j.Gs[k][l] = float(w / wh * P.G[k][l]);
  j.wh = float(wh);
  j.ihx = float(1.0 / g.hx);
  j.ihy = float(1.0 / g.hy);
  j.ihz = float(1.0 / g.hz);
  j.dx = FastDiv::make(uint32_t(g.nx));
  j.dy = FastDiv::make(uint32_t(g.ny));
#if PFM_NV == 6
  // G = alpha I + beta 1 1^T exactly (equal off-diagonal and equal diagonal entries)?
  const double beta = P.G[0][1], diag = P.G[0][0];
  bool ones = true;
  for (int k = 0; k < NV; ++k)
    for (int l = 0; l < NV; ++l)
      if (P.G[k][l] != (k == l ? diag : beta)) ones = false;
  j.g_diag_plus_ones = ones ? 1 : 0;
  j.g_alpha = float(w / wh * (diag - beta));
  j.g_beta = float(w / wh * beta);
#endif
  return j;
}

// the staged kernel indexes elements in 32 bits
bool staged_fits(const Grid& g) { return g.ne() < (int64_t(1) << 31) - 4; }

template <typename S, int D, int WPC>
int staged_prepare() {  // dynamic shared memory attribute; resident CTAs per SM
  constexpr int smem = WPC * D * int(HBLK * sizeof(S));
  static int occ = -1;
  if (occ < 0) {
    occ = 0;
    if (cudaFuncSetAttribute(k_japply_tma<S, D, WPC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
        cudaSuccess)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_japply_tma<S, D, WPC>, 32 * WPC, smem);
    cudaGetLastError();  // a refused shape is simply not offered
  }
  return occ;
}

template <typename S, int D, int WPC>
void staged_launch_t(const Grid& g, const JStaged& jp, const S* H, const dmask_t* mask, const float* v, float* y,
                     int per_sm, cudaStream_t s) {
  constexpr int smem = WPC * D * int(HBLK * sizeof(S));
  const int64_t need = (g.nblk() + WPC - 1) / WPC;
  const int64_t full = int64_t(sm_count()) * per_sm;
  k_japply_tma<S, D, WPC><<<unsigned(need < full ? need : full), 32 * WPC, smem, s>>>(g, jp, H, mask, v, y);
}

template <typename S>
int staged_occupancy(int stages, int threads) {
  if (stages == 2 && threads == 128) return staged_prepare<S, 2, 4>();
  if (stages == 3 && threads == 128) return staged_prepare<S, 3, 4>();
  if (stages == 2 && threads == 64) return staged_prepare<S, 2, 2>();
  if (stages == 2 && threads == 32) return staged_prepare<S, 2, 1>();
  if (stages == 1 && threads == 128) return staged_prepare<S, 1, 4>();
  return 0;
}

template <typename S>
void staged_launch(const Grid& g, const JStaged& jp, const S* H, const dmask_t* mask, const float* v, float* y,
                   const JShape& js, cudaStream_t s) {
  staged_occupancy<S>(js.stages, js.threads);
  if (js.stages == 2 && js.threads == 128) staged_launch_t<S, 2, 4>(g, jp, H, mask, v, y, js.per_sm, s);
  else if (js.stages == 3 && js.threads == 128) staged_launch_t<S, 3, 4>(g, jp, H, mask, v, y, js.per_sm, s);
  else if (js.stages == 2 && js.threads == 64) staged_launch_t<S, 2, 2>(g, jp, H, mask, v, y, js.per_sm, s);
  else if (js.stages == 2 && js.threads == 32) staged_launch_t<S, 2, 1>(g, jp, H, mask, v, y, js.per_sm, s);
  else staged_launch_t<S, 1, 4>(g, jp, H, mask, v, y, js.per_sm, s);
}

// element kernel of the tangent application for a store of type S (wh: weight
// of the Hessian part, used by the scaled binary16 store only)
template <typename T>
void japply_elem(const Grid& g, const JParams<T>& jp, float, const T* H, const dmask_t* mask, const T* v, T* y,
                 T* W, unsigned blocks, int threads, cudaStream_t s) {
  if (W)
    k_japply_det<T><<<blocks, threads, 0, s>>>(g, jp, H, mask, v, W, g.nblk() * 32);
  else
    k_japply<T><<<blocks, threads, 0, s>>>(g, jp, H, mask, v, y);
}
inline void japply_elem(const Grid& g, const JParams<float>& jp, float wh, const __half* H, const dmask_t* mask,
                        const float* v, float* y, float* W, unsigned blocks, int threads, cudaStream_t s) {
  if (W)
    k_japply_h16<true><<<blocks, threads, 0, s>>>(g, jp, wh, H, mask, v, y, W, g.nblk() * 32);
  else
    k_japply_h16<false><<<blocks, threads, 0, s>>>(g, jp, wh, H, mask, v, y, nullptr, 0);
}
template <typename T>
const void* japply_elem_fn(const T*) {
  return reinterpret_cast<const void*>(k_japply<T>);
}
inline const void* japply_elem_fn(const __half*) { return reinterpret_cast<const void*>(k_japply_h16<false>); }

// One tangent application with launch shape js; with a scratch W (9 * 32 *
// nblk entries) atomic-free: element pass into W, then the node pass writes
// every entry of y (no initialisation needed).
// The staged kernel (js.stages > 0) serves the atomic form of FP32 arithmetic
// only; the atomic-free form and FP64 use the register-fed kernel (with the
// default shape when the tuned one is staged).
template <typename T, typename S = T>
void japply_launch_shape(const Grid& g, const JParams<T>& jp, float wh, const S* H, const dmask_t* mask, const T* v,
                         T* y, const JShape& js, cudaStream_t s, T* W = nullptr, const JStaged* jst = nullptr) {
  const int64_t nn = g.nn();
  if (!W) {
    k_japply_init<T><<<grid_for(NF * nn, 256) < 4096 ? grid_for(NF * nn, 256) : 4096, 256, 0, s>>>(nn, mask, v, y);
    count_launches(1);
  }
  if constexpr (std::is_same<T, float>::value) {
    if (js.stages > 0 && !W && jst) {
      staged_launch<S>(g, *jst, H, mask, v, y, js, s);
      count_launches(1);
      return;
    }
  }
  const JShape cs = js.stages > 0 ? JShape{} : js;
  const int64_t need = (g.nblk() * 32 + cs.threads - 1) / cs.threads;
  const int64_t full = int64_t(sm_count()) * cs.per_sm;
  const unsigned blocks = unsigned(need < full ? need : full);
  japply_elem(g, jp, wh, H, mask, v, y, W, blocks, cs.threads, s);
  count_launches(1);
  if (W) {
    k_node_gather<T, T, T><<<grid_for(nn, 128), 128, 0, s>>>(g, W, g.nblk() * 32, mask, v, y);
    count_launches(1);
  }
}

template <typename T, typename S = T>
JShape japply_tune(const Grid& g, const JParams<T>& jp, float wh, const S* H, const dmask_t* mask, const T* v, T* y,
                   cudaStream_t s, const JStaged* jst = nullptr) {
  const int pr = sizeof(S) == 2 ? 2 : (sizeof(T) == 4 ? 0 : 1);
  int cl = 0;
  for (int64_t b = g.nblk(); b > 1; b >>= 1) ++cl;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  tune_file_read();
  auto it = g_tuned.find({pr, cl});
  if (it != g_tuned.end()) return it->second;
  JShape best;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  if (cap != cudaStreamCaptureStatusNone) return best;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best_ms = 1e30f;
  std::vector<JShape> cand;
  for (int threads : {256, 128}) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, japply_elem_fn(H), threads, 0);
    for (int ps = 1; ps <= occ; ++ps) cand.push_back(JShape{threads, ps, 0.0, 0});
  }
  if constexpr (std::is_same<T, float>::value) {
    if (jst && staged_fits(g))
      for (const auto& sh : STAGED_SHAPES) {
        const int occ = staged_occupancy<S>(sh[0], sh[1]);
        for (int ps = 1; ps <= occ; ++ps) cand.push_back(JShape{sh[1], ps, 0.0, sh[0]});
      }
  }
  for (const JShape& js : cand) {
    japply_launch_shape<T, S>(g, jp, wh, H, mask, v, y, js, s, nullptr, jst);  // warm
    // best of three timings of three applications each (the shapes differ
    // by a few per cent, about the run-to-run spread of one timing)
    float ms = 1e30f;
    for (int t = 0; t < 3; ++t) {
      cudaEventRecord(a, s);
      for (int r = 0; r < 3; ++r) japply_launch_shape<T, S>(g, jp, wh, H, mask, v, y, js, s, nullptr, jst);
      cudaEventRecord(b, s);
      cudaEventSynchronize(b);
      float m = 0.f;
      cudaEventElapsedTime(&m, a, b);
      if (m < ms) ms = m;
    }
    if (ms < best_ms) {
      best_ms = ms;
      best = js;
      best.ms = ms / 3.0;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  g_tuned[{pr, cl}] = best;
  tune_file_write();
  return best;
}

template <typename T>
void launch_japply(const Grid& g, const DevParams& P, const T* H, const dmask_t* mask, const T* v,
                   T* y, cudaStream_t s, T* W) {
  const JParams<T> jp = make_jparams<T>(g, P);
  if constexpr (std::is_same<T, float>::value) {
    const JStaged jst = make_jstaged(g, P, g.w());
    const JShape js = japply_tune<T>(g, jp, 0.f, H, mask, v, y, s, &jst);
    japply_launch_shape<T>(g, jp, 0.f, H, mask, v, y, js, s, W, &jst);
  } else {
    const JShape js = japply_tune<T>(g, jp, 0.f, H, mask, v, y, s);
    japply_launch_shape<T>(g, jp, 0.f, H, mask, v, y, js, s, W);
  }
}

void launch_japply_h16(const Grid& g, const DevParams& P, const __half* H, float inv_scale, const dmask_t* mask,
                      const float* v, float* y, cudaStream_t s, float* W) {
  const JParams<float> jp = make_jparams<float>(g, P);
  const float wh = jp.w * inv_scale;
  const JStaged jst = make_jstaged(g, P, g.w() * double(inv_scale));
  const JShape js = japply_tune<float, __half>(g, jp, wh, H, mask, v, y, s, &jst);
  japply_launch_shape<float, __half>(g, jp, wh, H, mask, v, y, js, s, W, &jst);
}

int take_wait_timeouts() {
  int n = 0;
  if (cudaMemcpyFromSymbol(&n, g_wait_timeouts, sizeof(int)) != cudaSuccess) return 0;
  if (n != 0) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_wait_timeouts, &zero, sizeof(int));
  }
  return n;
}

float half_store_scale(float amax) {
  // the largest entry lands in [2^14, 2^15): far from the binary16 maximum
  // (65504) and with 2^-24 / 2^15 ~ 2^-39 of the largest entry still resolved
  int e = 0;
  std::frexp(amax > 0.f ? amax : 1.f, &e);  // amax = m 2^e, m in [0.5, 1)
  return std::ldexp(1.f, 15 - e);
}

float launch_store_to_half(const Grid& g, const float* H32, __half* H16, unsigned* scratch, cudaStream_t s) {
  const int64_t n = g.nblk() * HBLK;
  cudaMemsetAsync(scratch, 0, sizeof(unsigned), s);
  k_absmax<<<unsigned(sm_count()) * 8, 256, 0, s>>>(n, H32, scratch);
  count_launches(1);
  unsigned bits = 0;
  cudaMemcpyAsync(&bits, scratch, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return 0.f;
  float amax = 0.f;
  std::memcpy(&amax, &bits, sizeof(float));
  if (!std::isfinite(amax)) return 0.f;
  const float scale = half_store_scale(amax);
  k_store_to_half<<<unsigned(sm_count()) * 8, 256, 0, s>>>(n / 8, reinterpret_cast<const float4*>(H32), scale,
                                                            reinterpret_cast<uint4*>(H16));
  count_launches(1);
  return scale;
}

void launch_japply_df(const Grid& g, const DevParams& P, const float* Hhi, const float* Hlo, const dmask_t* mask,
                      const float* v, double* y, cudaStream_t s, double* W) {
  const DfConst k = make_dfconst(g, P);
  const int64_t nn = g.nn();
  if (!W) {
    k_japply_init_df<<<grid_for(NF * nn, 256) < 4096 ? grid_for(NF * nn, 256) : 4096, 256, 0, s>>>(nn, mask, v, y);
    count_launches(1);
  }
  static int per_sm = 0;
  if (per_sm == 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_japply_df<false>, 256, 0);
    if (per_sm < 1) per_sm = 1;
  }
  const int64_t need = (g.nblk() * 32 + 255) / 256;
  const int64_t full = int64_t(sm_count()) * per_sm;
  const unsigned blocks = unsigned(need < full ? need : full);
  if (W) {
    const int64_t ws = g.nblk() * 32;
    k_japply_df<true><<<blocks, 256, 0, s>>>(g, k, Hhi, Hlo, mask, v, y, W, ws);
    k_node_gather<double, float, double><<<grid_for(nn, 128), 128, 0, s>>>(g, W, ws, mask, v, y);
    count_launches(2);
    return;
  }
  k_japply_df<false><<<blocks, 256, 0, s>>>(g, k, Hhi, Hlo, mask, v, y, nullptr, 0);
  count_launches(1);
}

template <typename T>
void launch_blockdiag(const Grid& g, const DevParams& P, const T* H, const dmask_t* mask, T* D, T* W,
                      cudaStream_t s) {
  (void)mask;
  // 4 element blocks per CTA in FP32 (60 KB of staged Hessians), 2 in FP64
  const int warps = sizeof(T) == 4 ? 4 : 2;
  const int smem = int(warps * HBLK * sizeof(T));
  static bool attr_set = false;  // one flag per instantiation (element type)
  if (!attr_set) {
    // a failure stays in cudaGetLastError and is reported by the caller's launch check
    if (cudaFuncSetAttribute(k_blockdiag_elem<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess)
      attr_set = true;
  }
  k_blockdiag_elem<T><<<grid_for(g.nblk() * 32, 32 * warps), 32 * warps, smem, s>>>(g, make_jparams<T>(g, P), H, W);
  k_blockdiag_node<T><<<grid_for(g.nn(), 128), 128, 0, s>>>(g, W, D);
  count_launches(2);
}

template <typename T>
void launch_block_invert(int64_t nn, const dmask_t* mask, T* D, int* singular, cudaStream_t s) {
  k_block_invert<T><<<grid_for(nn, 128), 128, 0, s>>>(nn, mask, D, singular);
  count_launches(1);
}

void launch_qp_eval(const DevParams& P, int64_t n, const double* F, const double* eta,
                    const double* eta_n, double* W, double* grad, double* hess, cudaStream_t s) {
  k_qp_eval<<<grid_for(n, 64), 64, 0, s>>>(P, n, F, eta, eta_n, W, grad, hess);
  count_launches(1);
}

template <typename T>
void launch_japply_range(const Grid& g, const DevParams& P, const T* H, const dmask_t* mask, const T* v, T* y,
                         int64_t b0, int64_t b1, int blocks, cudaStream_t s) {
  if (b1 <= b0) return;
  const int64_t need = ((b1 - b0) * 32 + 255) / 256;
  k_japply_range<T><<<unsigned(need < blocks ? need : blocks), 256, 0, s>>>(g, make_jparams<T>(g, P), H, mask, v, y,
                                                                            b0, b1);
  count_launches(1);
}

template <typename T>
void launch_identity_rows(int64_t nn, const dmask_t* mask, const T* v, T* y, int64_t n0, int64_t n1, cudaStream_t s) {
  if (n1 <= n0) return;
  const int64_t t = NF * (n1 - n0);
  k_identity_rows<T><<<grid_for(t, 256) < 2048 ? grid_for(t, 256) : 2048, 256, 0, s>>>(nn, mask, v, y, n0, n1);
  count_launches(1);
}

int japply_range_blocks() {
  static int per_sm = 0;
  if (per_sm == 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_japply_range<float>, 256, 0);
    if (per_sm < 1) per_sm = 1;
  }
  return sm_count() * per_sm;
}

template void launch_japply_range<float>(const Grid&, const DevParams&, const float*, const dmask_t*, const float*,
                                         float*, int64_t, int64_t, int, cudaStream_t);
template void launch_japply_range<double>(const Grid&, const DevParams&, const double*, const dmask_t*,
                                          const double*, double*, int64_t, int64_t, int, cudaStream_t);
template void launch_identity_rows<float>(int64_t, const dmask_t*, const float*, float*, int64_t, int64_t,
                                          cudaStream_t);
template void launch_identity_rows<double>(int64_t, const dmask_t*, const double*, double*, int64_t, int64_t,
                                           cudaStream_t);

template void launch_japply<float>(const Grid&, const DevParams&, const float*, const dmask_t*,
                                   const float*, float*, cudaStream_t, float*);
template void launch_japply<double>(const Grid&, const DevParams&, const double*, const dmask_t*,
                                     const double*, double*, cudaStream_t, double*);
template void launch_blockdiag<float>(const Grid&, const DevParams&, const float*, const dmask_t*, float*,
                                      float*, cudaStream_t);
template void launch_blockdiag<double>(const Grid&, const DevParams&, const double*, const dmask_t*, double*,
                                       double*, cudaStream_t);
template void launch_block_invert<float>(int64_t, const dmask_t*, float*, int*, cudaStream_t);
template void launch_block_invert<double>(int64_t, const dmask_t*, double*, int*, cudaStream_t);

}  // namespace pfm
