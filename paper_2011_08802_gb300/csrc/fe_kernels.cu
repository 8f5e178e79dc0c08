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
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>

#include "common.cuh"

namespace pfm {
namespace {

template <typename T>
__device__ __forceinline__ T shx(T v, int m) {
  return __shfl_xor_sync(0xffffffffu, v, m);
}

// Nodal value v of this lane's node -> value and gradient at this lane's point.
template <typename T>
__device__ __forceinline__ void q1_gather(T v, int l8, T ihx, T ihy, T ihz, T& val, T& gx, T& gy,
                                          T& gz) {
  const T ga = T(GA), gb = T(GB);
  T s = shx(v, 1);
  T vx = gb * v + ga * s;
  T dx = ((l8 & 1) ? (v - s) : (s - v)) * ihx;
  T s1 = shx(vx, 2), s2 = shx(dx, 2);
  T vxy = gb * vx + ga * s1;
  T vdy = ((l8 & 2) ? (vx - s1) : (s1 - vx)) * ihy;
  T dxy = gb * dx + ga * s2;
  T t1 = shx(vxy, 4), t2 = shx(vdy, 4), t3 = shx(dxy, 4);
  val = gb * vxy + ga * t1;
  gz = ((l8 & 4) ? (vxy - t1) : (t1 - vxy)) * ihz;
  gy = gb * vdy + ga * t2;
  gx = gb * dxy + ga * t3;
}

// Nodal value -> value at this lane's point.
template <typename T>
__device__ __forceinline__ T q1_value(T v) {
  const T ga = T(GA), gb = T(GB);
  v = gb * v + ga * shx(v, 1);
  v = gb * v + ga * shx(v, 2);
  return gb * v + ga * shx(v, 4);
}

// Transpose: point weights (val for N_a, g for grad N_a) -> this lane's node.
template <typename T>
__device__ __forceinline__ T q1_scatter(T val, T gx, T gy, T gz, int l8, T ihx, T ihy, T ihz) {
  const T ga = T(GA), gb = T(GB);
  T sv = shx(val, 4), sz = shx(gz, 4), sx = shx(gx, 4), sy = shx(gy, 4);
  T A = gb * val + ga * sv + ((l8 & 4) ? (gz + sz) : -(gz + sz)) * ihz;
  T Bx = gb * gx + ga * sx;
  T By = gb * gy + ga * sy;
  T sA = shx(A, 2), sBy = shx(By, 2), sBx = shx(Bx, 2);
  T Cc = gb * A + ga * sA + ((l8 & 2) ? (By + sBy) : -(By + sBy)) * ihy;
  T Dx = gb * Bx + ga * sBx;
  T sC = shx(Cc, 1), sD = shx(Dx, 1);
  return gb * Cc + ga * sC + ((l8 & 1) ? (Dx + sD) : -(Dx + sD)) * ihx;
}

template <typename T>
__device__ __forceinline__ T q1_scatter_grad(T gx, T gy, T gz, int l8, T ihx, T ihy, T ihz) {
  const T ga = T(GA), gb = T(GB);
  T sz = shx(gz, 4), sx = shx(gx, 4), sy = shx(gy, 4);
  T A = ((l8 & 4) ? (gz + sz) : -(gz + sz)) * ihz;
  T Bx = gb * gx + ga * sx;
  T By = gb * gy + ga * sy;
  T sA = shx(A, 2), sBy = shx(By, 2), sBx = shx(Bx, 2);
  T Cc = gb * A + ga * sA + ((l8 & 2) ? (By + sBy) : -(By + sBy)) * ihy;
  T Dx = gb * Bx + ga * sBx;
  T sC = shx(Cc, 1), sD = shx(Dx, 1);
  return gb * Cc + ga * sC + ((l8 & 1) ? (Dx + sD) : -(Dx + sD)) * ihx;
}

// Row of packed upper-triangle index idx of a 15x15 matrix, and the packed
// index where row r starts.
__host__ __device__ constexpr int packed_row_start(int r) { return r * NZ - (r * (r - 1)) / 2; }
__host__ __device__ constexpr int packed_row(int idx) {
  int r = 0;
  while (r + 1 < NZ && idx >= packed_row_start(r + 1)) ++r;
  return r;
}
static_assert(packed_row(0) == 0 && packed_row(14) == 0 && packed_row(15) == 1 && packed_row(20) == 1 &&
                  packed_row(119) == 14 && packed_row(117) == 13 && packed_row(116) == 12,
              "packed index decode");

__device__ __forceinline__ int64_t elem_node(const Grid& g, int64_t e, int a) {
  int64_t ei = e % g.nx;
  int64_t r = e / g.nx;
  int64_t ej = r % g.ny;
  int64_t ek = r / g.ny;
  return (ei + (a & 1)) + int64_t(g.nx + 1) * ((ej + ((a >> 1) & 1)) + int64_t(g.ny + 1) * (ek + (a >> 2)));
}

// Gather F = I + grad u, eta_hat and grad eta_hat at this lane's point.
template <typename T, typename Src>
__device__ __forceinline__ void gather_state(const Src* __restrict__ U, int64_t nn, int64_t node,
                                             bool valid, int l8, T ihx, T ihy, T ihz, T F[9],
                                             T eh[6], T ge[18]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T v = valid ? T(U[i * nn + node]) : T(0);
    T val, gx, gy, gz;
    q1_gather(v, l8, ihx, ihy, ihz, val, gx, gy, gz);
    F[3 * i + 0] = gx;
    F[3 * i + 1] = gy;
    F[3 * i + 2] = gz;
  }
  F[0] += T(1);
  F[4] += T(1);
  F[8] += T(1);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    T v = valid ? T(U[(3 + k) * nn + node]) : T(0);
    q1_gather(v, l8, ihx, ihy, ihz, eh[k], ge[3 * k], ge[3 * k + 1], ge[3 * k + 2]);
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_residual(Grid g, DevParams P, const double* __restrict__ U,
                                                  const double* __restrict__ Un,
                                                  const dmask_t* __restrict__ mask,
                                                  double* __restrict__ R, double* energy) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t e = tid >> 3;
  const int l8 = int(tid & 7);
  const bool valid = e < g.ne();
  const int64_t nn = g.nn();
  const int64_t node = valid ? elem_node(g, e, l8) : 0;
  const double ihx = 1.0 / g.hx, ihy = 1.0 / g.hy, ihz = 1.0 / g.hz;
  double F[9], eh[6], ge[18], ehn[6];
  gather_state<double>(U, nn, node, valid, l8, ihx, ihy, ihz, F, eh, ge);
#pragma unroll
  for (int k = 0; k < 6; ++k) ehn[k] = q1_value(valid ? Un[(3 + k) * nn + node] : 0.0);
  double W, gr[NZ];
  qp_local<double, false>(P, F, eh, ehn, &W, gr, nullptr);
  double gf[18];
  double Wg = 0.0;
#pragma unroll
  for (int k = 0; k < 6; ++k)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < 6; ++l) s += P.G[k][l] * ge[3 * l + d];
      gf[3 * k + d] = s;
      Wg += 0.5 * ge[3 * k + d] * s;
    }
  const double w = g.w();
  const dmask_t dm = valid ? mask[node] : dmask_t(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double r = q1_scatter_grad(w * gr[3 * i], w * gr[3 * i + 1], w * gr[3 * i + 2], l8, ihx, ihy, ihz);
    if (valid && !((dm >> i) & 1)) atomicAdd(&R[i * nn + node], r);
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double r = q1_scatter(w * gr[9 + k], w * gf[3 * k], w * gf[3 * k + 1], w * gf[3 * k + 2], l8, ihx,
                          ihy, ihz);
    if (valid && !((dm >> (3 + k)) & 1)) atomicAdd(&R[(3 + k) * nn + node], r);
  }
  if (energy) {
    double en = warp_sum(valid ? w * (W + Wg) : 0.0);
    if ((threadIdx.x & 31) == 0) atomicAdd(energy, en);
  }
}

// Gauss-point Hessians of one level, computed in TC (FP64 for the finest and
// the coarsest level, FP32 for the intermediate levels of an FP32
// preconditioner) and stored in the requested precisions.
template <typename TC>
__global__ void __launch_bounds__(128) k_linearize(Grid g, DevParams P, const double* __restrict__ U,
                                                   const double* __restrict__ Un,
                                                   double* __restrict__ H64, float* __restrict__ H32,
                                                   float* __restrict__ H32lo) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t e = tid >> 3;
  const int l8 = int(tid & 7);
  const int64_t nblk = g.nblk();
  if ((tid >> 5) >= nblk) return;  // whole warps only (padding lanes stay)
  const bool valid = e < g.ne();
  const int64_t nn = g.nn();
  const int64_t node = valid ? elem_node(g, e, l8) : 0;
  const TC ihx = TC(1.0 / g.hx), ihy = TC(1.0 / g.hy), ihz = TC(1.0 / g.hz);
  TC F[9], eh[6], ge[18], ehn[6];
  gather_state<TC>(U, nn, node, valid, l8, ihx, ihy, ihz, F, eh, ge);
#pragma unroll
  for (int k = 0; k < 6; ++k) ehn[k] = q1_value(valid ? TC(Un[(3 + k) * nn + node]) : TC(0));
  TC W, gr[NZ], Hp[NH];
  qp_local<TC, true>(P, F, eh, ehn, &W, gr, Hp);
  const int64_t blk = tid >> 5;
  const int lane = int(tid & 31);
  for (int j = 0; j < NH; ++j) {
    const double h = valid ? double(Hp[j]) : 0.0;
    if (H64) H64[hstore_offset<double>(blk, j, lane)] = h;
    if (H32) H32[hstore_offset<float>(blk, j, lane)] = float(h);
    if (H32lo) H32lo[hstore_offset<float>(blk, j, lane)] = float(h - double(float(h)));
  }
}

// Vector of V = 16/sizeof(T) Hessian entries.
template <typename T> struct Vec16;
template <> struct Vec16<float> {
  using type = float4;
  static __device__ __forceinline__ void unpack(const float4& x, float* o) { o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w; }
};
template <> struct Vec16<double> {
  using type = double2;
  static __device__ __forceinline__ void unpack(const double2& x, double* o) { o[0] = x.x; o[1] = x.y; }
};

template <typename T>
struct JParams {
  T G[6][6];
  T w, ihx, ihy, ihz;
};

// ---- BEGIN tangent application kernel
// Asynchronous bulk prefetch of a contiguous global range into L2 (the
// bulk-copy engine; no registers or shared memory involved). Address 16-byte
// aligned, size a multiple of 16 bytes.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// y += J v over the elements (y initialised by k_japply_init). Persistent
// warps walk the element blocks (4 elements each) with a grid stride; before
// working on a block, lane 0 prefetches the block this warp takes PF strides
// later, so every warp keeps its next 15 KB (FP32) of Hessians in flight.
#ifndef PFM_JAPPLY_MINB
#define PFM_JAPPLY_MINB 2
#endif
template <typename T, int PF>
__global__ void __launch_bounds__(256, PFM_JAPPLY_MINB) k_japply(Grid g, JParams<T> jp, const T* __restrict__ H,
                                                const dmask_t* __restrict__ mask,
                                                const T* __restrict__ v, T* __restrict__ y) {
  constexpr int V = 16 / sizeof(T);
  using VT = typename Vec16<T>::type;
  const int64_t nblk = g.nblk();
  const int64_t wg = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int lane = int(threadIdx.x & 31);
  const int l8 = lane & 7;
  const int64_t nn = g.nn();
  constexpr unsigned BLK_BYTES = unsigned(HBLK * sizeof(T));
  if (lane == 0)
    for (int d = 0; d < PF; ++d)
      if (wg + d * nw < nblk) prefetch_l2(H + (wg + d * nw) * HBLK, BLK_BYTES);
  for (int64_t blk = wg; blk < nblk; blk += nw) {
    if (lane == 0 && blk + PF * nw < nblk) prefetch_l2(H + (blk + PF * nw) * HBLK, BLK_BYTES);
    const int64_t e = blk * 4 + (lane >> 3);
    const bool valid = e < g.ne();
    const int64_t node = valid ? elem_node(g, e, l8) : 0;
    const dmask_t dm = valid ? mask[node] : dmask_t(0x1ff);
    T dz[NZ], ge[18];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T x = ((dm >> i) & 1) ? T(0) : v[i * nn + node];
      T val;
      q1_gather(x, l8, jp.ihx, jp.ihy, jp.ihz, val, dz[3 * i], dz[3 * i + 1], dz[3 * i + 2]);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      T x = ((dm >> (3 + k)) & 1) ? T(0) : v[(3 + k) * nn + node];
      q1_gather(x, l8, jp.ihx, jp.ihy, jp.ihz, dz[9 + k], ge[3 * k], ge[3 * k + 1], ge[3 * k + 2]);
    }
    // sigma = H dz from the packed symmetric store
    T sg[NZ];
#pragma unroll
    for (int r = 0; r < NZ; ++r) sg[r] = T(0);
    const VT* Hv = reinterpret_cast<const VT*>(H) + blk * (NH / V) * 32 + lane;
#pragma unroll
    for (int j = 0; j < NH / V; ++j) {
      T hv[V];
      Vec16<T>::unpack(__ldcs(Hv + j * 32), hv);
#pragma unroll
      for (int t = 0; t < V; ++t) {
        const int idx = j * V + t;
        // (r, c) of packed index idx (constant-folded after unrolling)
        const int r = packed_row(idx);
        const int c = r + (idx - packed_row_start(r));
        sg[r] += hv[t] * dz[c];
        if (c != r) sg[c] += hv[t] * dz[r];
      }
    }
    const T w = jp.w;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T r = q1_scatter_grad(w * sg[3 * i], w * sg[3 * i + 1], w * sg[3 * i + 2], l8, jp.ihx, jp.ihy, jp.ihz);
      if (valid && !((dm >> i) & 1)) atomicAdd(&y[i * nn + node], r);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      T gf[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        T s = T(0);
#pragma unroll
        for (int l = 0; l < 6; ++l) s += jp.G[k][l] * ge[3 * l + d];
        gf[d] = w * s;
      }
      T r = q1_scatter(w * sg[9 + k], gf[0], gf[1], gf[2], l8, jp.ihx, jp.ihy, jp.ihz);
      if (valid && !((dm >> (3 + k)) & 1)) atomicAdd(&y[(3 + k) * nn + node], r);
    }
  }
}

// ---- END tangent application kernel

// ---------------------------------------------------------------------------
// Double-float ("df") arithmetic: a value is an unevaluated sum hi + lo of two
// FP32 numbers (Dekker 1971, "A floating-point technique for extending the
// available precision"; Knuth's TwoSum). Only round-to-nearest FP32 adds,
// multiplies and fused multiply-adds are used (the _rn intrinsics keep the
// compiler from contracting or reassociating them), giving about 48
// significant bits: enough for an outer Krylov operator checked to 1e-8.
struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  const dfl s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ dfl df_shx(dfl v, int m) { return {shx(v.hi, m), shx(v.lo, m)}; }

struct DfConst {
  dfl ga, gb, ihx, ihy, ihz, w;
  dfl G[6][6];
};
inline dfl df_host(double x) {
  const float hi = float(x);
  return {hi, float(x - double(hi))};
}

__device__ __forceinline__ void q1_gather_df(dfl v, int l8, const DfConst& k, dfl& val, dfl& gx, dfl& gy,
                                             dfl& gz) {
  dfl s = df_shx(v, 1);
  dfl vx = df_add(df_mul(k.gb, v), df_mul(k.ga, s));
  dfl dx = df_mul((l8 & 1) ? df_sub(v, s) : df_sub(s, v), k.ihx);
  dfl s1 = df_shx(vx, 2), s2 = df_shx(dx, 2);
  dfl vxy = df_add(df_mul(k.gb, vx), df_mul(k.ga, s1));
  dfl vdy = df_mul((l8 & 2) ? df_sub(vx, s1) : df_sub(s1, vx), k.ihy);
  dfl dxy = df_add(df_mul(k.gb, dx), df_mul(k.ga, s2));
  dfl t1 = df_shx(vxy, 4), t2 = df_shx(vdy, 4), t3 = df_shx(dxy, 4);
  val = df_add(df_mul(k.gb, vxy), df_mul(k.ga, t1));
  gz = df_mul((l8 & 4) ? df_sub(vxy, t1) : df_sub(t1, vxy), k.ihz);
  gy = df_add(df_mul(k.gb, vdy), df_mul(k.ga, t2));
  gx = df_add(df_mul(k.gb, dxy), df_mul(k.ga, t3));
}

__device__ __forceinline__ dfl q1_scatter_df(dfl val, dfl gx, dfl gy, dfl gz, bool has_val, int l8,
                                             const DfConst& k) {
  dfl sz = df_shx(gz, 4), sx = df_shx(gx, 4), sy = df_shx(gy, 4);
  dfl A = df_mul((l8 & 4) ? df_add(gz, sz) : df_neg(df_add(gz, sz)), k.ihz);
  if (has_val) {
    dfl sv = df_shx(val, 4);
    A = df_add(A, df_add(df_mul(k.gb, val), df_mul(k.ga, sv)));
  }
  dfl Bx = df_add(df_mul(k.gb, gx), df_mul(k.ga, sx));
  dfl By = df_add(df_mul(k.gb, gy), df_mul(k.ga, sy));
  dfl sA = df_shx(A, 2), sBy = df_shx(By, 2), sBx = df_shx(Bx, 2);
  dfl Cc = df_add(df_add(df_mul(k.gb, A), df_mul(k.ga, sA)),
                  df_mul((l8 & 2) ? df_add(By, sBy) : df_neg(df_add(By, sBy)), k.ihy));
  dfl Dx = df_add(df_mul(k.gb, Bx), df_mul(k.ga, sBx));
  dfl sC = df_shx(Cc, 1), sD = df_shx(Dx, 1);
  return df_add(df_add(df_mul(k.gb, Cc), df_mul(k.ga, sC)),
                df_mul((l8 & 1) ? df_add(Dx, sD) : df_neg(df_add(Dx, sD)), k.ihx));
}

// y += J v with v in FP32 (exact input), the tangent as Hhi + Hlo (two FP32
// stores of the FP64 Hessians) and double-float arithmetic throughout; the
// element contributions are added to the FP64 output y (initialised by
// k_japply_init_df). Same persistent warp mapping as k_japply.
#ifndef PFM_DF_MINB
#define PFM_DF_MINB 8
#endif
__global__ void __launch_bounds__(256, PFM_DF_MINB) k_japply_df(Grid g, DfConst k, const float* __restrict__ Hhi,
                                                     const float* __restrict__ Hlo,
                                                     const dmask_t* __restrict__ mask,
                                                     const float* __restrict__ v, double* __restrict__ y) {
  const int64_t nblk = g.nblk();
  const int64_t wg = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int lane = int(threadIdx.x & 31);
  const int l8 = lane & 7;
  const int64_t nn = g.nn();
  for (int64_t blk = wg; blk < nblk; blk += nw) {
    const int64_t e = blk * 4 + (lane >> 3);
    const bool valid = e < g.ne();
    const int64_t node = valid ? elem_node(g, e, l8) : 0;
    const dmask_t dm = valid ? mask[node] : dmask_t(0x1ff);
    dfl dz[NZ], ge[18];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float x = ((dm >> i) & 1) ? 0.f : v[i * nn + node];
      dfl val;
      q1_gather_df(dfl{x, 0.f}, l8, k, val, dz[3 * i], dz[3 * i + 1], dz[3 * i + 2]);
    }
#pragma unroll
    for (int kk = 0; kk < 6; ++kk) {
      const float x = ((dm >> (3 + kk)) & 1) ? 0.f : v[(3 + kk) * nn + node];
      q1_gather_df(dfl{x, 0.f}, l8, k, dz[9 + kk], ge[3 * kk], ge[3 * kk + 1], ge[3 * kk + 2]);
    }
    dfl sg[NZ];
#pragma unroll
    for (int r = 0; r < NZ; ++r) sg[r] = dfl{0.f, 0.f};
    const float4* Hh = reinterpret_cast<const float4*>(Hhi) + blk * (NH / 4) * 32 + lane;
    const float4* Hl = reinterpret_cast<const float4*>(Hlo) + blk * (NH / 4) * 32 + lane;
#pragma unroll 2
    for (int j = 0; j < NH / 4; ++j) {
      float hh[4], hl[4];
      Vec16<float>::unpack(__ldcs(Hh + j * 32), hh);
      Vec16<float>::unpack(__ldcs(Hl + j * 32), hl);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int idx = j * 4 + t;
        const int r = packed_row(idx);
        const int c = r + (idx - packed_row_start(r));
        const dfl hv{hh[t], hl[t]};
        sg[r] = df_add(sg[r], df_mul(hv, dz[c]));
        if (c != r) sg[c] = df_add(sg[c], df_mul(hv, dz[r]));
      }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      dfl r = q1_scatter_df(dfl{0.f, 0.f}, df_mul(k.w, sg[3 * i]), df_mul(k.w, sg[3 * i + 1]),
                            df_mul(k.w, sg[3 * i + 2]), false, l8, k);
      if (valid && !((dm >> i) & 1)) atomicAdd(&y[i * nn + node], double(r.hi) + double(r.lo));
    }
#pragma unroll
    for (int kk = 0; kk < 6; ++kk) {
      dfl gf[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        dfl s = dfl{0.f, 0.f};
#pragma unroll
        for (int l = 0; l < 6; ++l) s = df_add(s, df_mul(k.G[kk][l], ge[3 * l + d]));
        gf[d] = df_mul(k.w, s);
      }
      dfl r = q1_scatter_df(df_mul(k.w, sg[9 + kk]), gf[0], gf[1], gf[2], true, l8, k);
      if (valid && !((dm >> (3 + kk)) & 1)) atomicAdd(&y[(3 + kk) * nn + node], double(r.hi) + double(r.lo));
    }
  }
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

// Nodal 9x9 diagonal blocks: thread (element, local node a) sums over the 8
// points B_a(q)^T H_q B_a(q) w plus the gradient-energy block, then adds it
// to the node's block D[(r*9+c)*nn + node].
template <typename T>
__global__ void __launch_bounds__(128) k_blockdiag(Grid g, JParams<T> jp, const T* __restrict__ H,
                                                   T* __restrict__ D) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t e = tid >> 3;
  if (e >= g.ne()) return;
  const int a = int(tid & 7);
  const int64_t blk = e >> 2;
  const int lane0 = int(e & 3) * 8;
  const int64_t nn = g.nn();
  const int64_t node = elem_node(g, e, a);
  T Db[45];
#pragma unroll
  for (int i = 0; i < 45; ++i) Db[i] = T(0);
  const T ih[3] = {jp.ihx, jp.ihy, jp.ihz};
  for (int q = 0; q < 8; ++q) {
    T phi[3], dphi[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int ad = (a >> d) & 1, qd = (q >> d) & 1;
      phi[d] = (ad == qd) ? T(GB) : T(GA);
      dphi[d] = (ad ? T(1) : T(-1)) * ih[d];
    }
    const T N = phi[0] * phi[1] * phi[2];
    const T dN[3] = {dphi[0] * phi[1] * phi[2], phi[0] * dphi[1] * phi[2], phi[0] * phi[1] * dphi[2]};
    // column map: DOF u_i -> z rows 3i+J (coef dN_J); eta_k -> z row 9+k (coef N)
    T Hq[NH];
    for (int j = 0; j < NH; ++j) Hq[j] = H[hstore_offset<T>(blk, j, lane0 + q)];
    auto hget = [&](int r, int c) -> T { return r <= c ? Hq[hidx(r, c)] : Hq[hidx(c, r)]; };
    int idx = 0;
    for (int r = 0; r < 9; ++r)
      for (int c = r; c < 9; ++c) {
        T s = T(0);
        if (r < 3 && c < 3) {
          for (int J = 0; J < 3; ++J)
            for (int L = 0; L < 3; ++L) s += dN[J] * dN[L] * hget(3 * r + J, 3 * c + L);
        } else if (r < 3) {
          for (int J = 0; J < 3; ++J) s += dN[J] * N * hget(3 * r + J, 9 + (c - 3));
        } else {
          s = N * N * hget(9 + (r - 3), 9 + (c - 3)) +
              (dN[0] * dN[0] + dN[1] * dN[1] + dN[2] * dN[2]) * jp.G[r - 3][c - 3];
        }
        Db[idx++] += jp.w * s;
      }
  }
  int idx = 0;
  for (int r = 0; r < 9; ++r)
    for (int c = r; c < 9; ++c) {
      atomicAdd(&D[(r * 9 + c) * nn + node], Db[idx]);
      if (c != r) atomicAdd(&D[(c * 9 + r) * nn + node], Db[idx]);
      ++idx;
    }
}

// In-place inverse of each node's 9x9 block (Dirichlet rows/columns replaced
// by identity first) by Gauss-Jordan elimination with partial pivoting.
template <typename T>
__global__ void k_block_invert(int64_t nn, const dmask_t* __restrict__ mask, T* __restrict__ D,
                               int* singular) {
  const int64_t node = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (node >= nn) return;
  const dmask_t dm = mask[node];
  T a[9][9], x[9][9];
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) {
      T v = D[(r * 9 + c) * nn + node];
      if (((dm >> r) & 1) || ((dm >> c) & 1)) v = (r == c) ? T(1) : T(0);
      a[r][c] = v;
      x[r][c] = (r == c) ? T(1) : T(0);
    }
  bool bad = false;
  for (int k = 0; k < 9; ++k) {
    int p = k;
    T best = fabs(a[k][k]);
    for (int r = k + 1; r < 9; ++r)
      if (fabs(a[r][k]) > best) { best = fabs(a[r][k]); p = r; }
    if (!(best > T(0))) { bad = true; break; }
    if (p != k)
      for (int c = 0; c < 9; ++c) {
        T t = a[k][c]; a[k][c] = a[p][c]; a[p][c] = t;
        t = x[k][c]; x[k][c] = x[p][c]; x[p][c] = t;
      }
    const T ip = T(1) / a[k][k];
    for (int c = 0; c < 9; ++c) { a[k][c] *= ip; x[k][c] *= ip; }
    for (int r = 0; r < 9; ++r) {
      if (r == k) continue;
      const T f = a[r][k];
      if (f == T(0)) continue;
      for (int c = 0; c < 9; ++c) { a[r][c] -= f * a[k][c]; x[r][c] -= f * x[k][c]; }
    }
  }
  if (bad) {
    atomicExch(singular, 1);
    for (int r = 0; r < 9; ++r)
      for (int c = 0; c < 9; ++c) x[r][c] = (r == c) ? T(1) : T(0);
  }
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) D[(r * 9 + c) * nn + node] = x[r][c];
}

__global__ void k_qp_eval(DevParams P, int64_t n, const double* __restrict__ F,
                          const double* __restrict__ eta, const double* __restrict__ eta_n,
                          double* __restrict__ W, double* __restrict__ grad, double* __restrict__ hess) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double Fl[9], e[6], en[6], w, g[NZ], h[NH];
  for (int k = 0; k < 9; ++k) Fl[k] = F[i * 9 + k];
  for (int k = 0; k < 6; ++k) { e[k] = eta[i * 6 + k]; en[k] = eta_n[i * 6 + k]; }
  qp_local<double, true>(P, Fl, e, en, &w, g, h);
  if (W) W[i] = w;
  if (grad)
    for (int k = 0; k < NZ; ++k) grad[i * NZ + k] = g[k];
  if (hess)
    for (int k = 0; k < NH; ++k) hess[i * NH + k] = h[k];
}

template <typename T>
JParams<T> make_jparams(const Grid& g, const DevParams& P) {
  JParams<T> jp;
  for (int k = 0; k < 6; ++k)
    for (int l = 0; l < 6; ++l) jp.G[k][l] = T(P.G[k][l]);
  jp.w = T(g.w());
  jp.ihx = T(1.0 / g.hx);
  jp.ihy = T(1.0 / g.hy);
  jp.ihz = T(1.0 / g.hz);
  return jp;
}

inline unsigned grid_for(int64_t threads, int block) {
  return unsigned((threads + block - 1) / block);
}

// element blocks a warp prefetches ahead of the one it works on
#ifndef PFM_JAPPLY_PF
#define PFM_JAPPLY_PF 0
#endif
constexpr int JAPPLY_PF = PFM_JAPPLY_PF;

}  // namespace

void launch_residual(const Grid& g, const DevParams& P, const double* U, const double* Un,
                     const dmask_t* mask, double* R, double* energy, cudaStream_t s) {
  const int64_t threads = g.nblk() * 32;
  k_residual<<<grid_for(threads, 128), 128, 0, s>>>(g, P, U, Un, mask, R, energy);
  count_launches(1);
}

void launch_linearize(const Grid& g, const DevParams& P, const double* U, const double* Un,
                      double* H64, float* H32, float* H32lo, bool fp32_compute, cudaStream_t s) {
  const int64_t threads = g.nblk() * 32;
  if (fp32_compute)
    k_linearize<float><<<grid_for(threads, 128), 128, 0, s>>>(g, P, U, Un, H64, H32, H32lo);
  else
    k_linearize<double><<<grid_for(threads, 128), 128, 0, s>>>(g, P, U, Un, H64, H32, H32lo);
  count_launches(1);
}

// ---------------------------------------------------------------------------
// Launch-shape autotuner of the tangent application. A launch shape is the
// element tile of one CTA (threads/8 elements: 16 or 32) and the number of
// resident CTAs per SM of the persistent grid. The first application for a
// (precision, size class = floor(log2 element blocks)) key times every
// candidate three times with events and keeps the fastest; the choice is
// cached for the process and, when PFM_AUTOTUNE_FILE names a file, read from
// and appended to it ("prec class threads ctas_per_sm" lines). No tuning runs
// while the stream is being captured into a graph (the default shape is used).
struct JShape {
  int threads = 256;
  int per_sm = 2;
};

std::mutex g_tune_mutex;
std::map<std::pair<int, int>, JShape> g_tuned;
bool g_tune_file_read = false;

void tune_file_read() {
  if (g_tune_file_read) return;
  g_tune_file_read = true;
  const char* path = std::getenv("PFM_AUTOTUNE_FILE");
  if (!path) return;
  std::FILE* f = std::fopen(path, "r");
  if (!f) return;
  int pr, cl, th, ps;
  while (std::fscanf(f, "%d %d %d %d", &pr, &cl, &th, &ps) == 4)
    if ((th == 128 || th == 256) && ps >= 1 && ps <= 16) g_tuned[{pr, cl}] = JShape{th, ps};
  std::fclose(f);
}

void tune_file_append(int pr, int cl, const JShape& js) {
  const char* path = std::getenv("PFM_AUTOTUNE_FILE");
  if (!path) return;
  std::FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%d %d %d %d\n", pr, cl, js.threads, js.per_sm);
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

template <typename T>
void japply_launch_shape(const Grid& g, JParams<T> jp, const T* H, const dmask_t* mask, const T* v, T* y,
                         const JShape& js, cudaStream_t s) {
  const int64_t nn = g.nn();
  k_japply_init<T><<<grid_for(NF * nn, 256) < 4096 ? grid_for(NF * nn, 256) : 4096, 256, 0, s>>>(nn, mask, v, y);
  count_launches(1);
  const int64_t need = (g.nblk() * 32 + js.threads - 1) / js.threads;
  const int64_t full = int64_t(sm_count()) * js.per_sm;
  const unsigned blocks = unsigned(need < full ? need : full);
  k_japply<T, JAPPLY_PF><<<blocks, js.threads, 0, s>>>(g, jp, H, mask, v, y);
  count_launches(1);
}

template <typename T>
JShape japply_tune(const Grid& g, const JParams<T>& jp, const T* H, const dmask_t* mask, const T* v, T* y,
                   cudaStream_t s) {
  const int pr = sizeof(T) == 4 ? 0 : 1;
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
  for (int threads : {256, 128}) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_japply<T, JAPPLY_PF>, threads, 0);
    for (int ps = 1; ps <= occ; ++ps) {
      JShape js{threads, ps};
      japply_launch_shape<T>(g, jp, H, mask, v, y, js, s);  // warm
      cudaEventRecord(a, s);
      for (int r = 0; r < 3; ++r) japply_launch_shape<T>(g, jp, H, mask, v, y, js, s);
      cudaEventRecord(b, s);
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (ms < best_ms) {
        best_ms = ms;
        best = js;
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  g_tuned[{pr, cl}] = best;
  tune_file_append(pr, cl, best);
  return best;
}

template <typename T>
void launch_japply(const Grid& g, const DevParams& P, const T* H, const dmask_t* mask, const T* v,
                   T* y, cudaStream_t s) {
  const JParams<T> jp = make_jparams<T>(g, P);
  const JShape js = japply_tune<T>(g, jp, H, mask, v, y, s);
  japply_launch_shape<T>(g, jp, H, mask, v, y, js, s);
}

void launch_japply_df(const Grid& g, const DevParams& P, const float* Hhi, const float* Hlo, const dmask_t* mask,
                      const float* v, double* y, cudaStream_t s) {
  DfConst k;
  k.ga = df_host(GA);
  k.gb = df_host(GB);
  k.ihx = df_host(1.0 / g.hx);
  k.ihy = df_host(1.0 / g.hy);
  k.ihz = df_host(1.0 / g.hz);
  k.w = df_host(g.w());
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) k.G[a][b] = df_host(P.G[a][b]);
  const int64_t nn = g.nn();
  k_japply_init_df<<<grid_for(NF * nn, 256) < 4096 ? grid_for(NF * nn, 256) : 4096, 256, 0, s>>>(nn, mask, v, y);
  count_launches(1);
  static int per_sm = 0;
  if (per_sm == 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_japply_df, 256, 0);
    if (per_sm < 1) per_sm = 1;
  }
  const int64_t need = (g.nblk() * 32 + 255) / 256;
  const int64_t full = int64_t(sm_count()) * per_sm;
  k_japply_df<<<unsigned(need < full ? need : full), 256, 0, s>>>(g, k, Hhi, Hlo, mask, v, y);
  count_launches(1);
}

template <typename T>
void launch_blockdiag(const Grid& g, const DevParams& P, const T* H, const dmask_t* mask, T* D,
                      cudaStream_t s) {
  (void)mask;
  cudaMemsetAsync(D, 0, sizeof(T) * 81 * g.nn(), s);
  const int64_t threads = g.ne() * 8;
  k_blockdiag<T><<<grid_for(threads, 128), 128, 0, s>>>(g, make_jparams<T>(g, P), H, D);
  count_launches(1);
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

template void launch_japply<float>(const Grid&, const DevParams&, const float*, const dmask_t*,
                                   const float*, float*, cudaStream_t);
template void launch_japply<double>(const Grid&, const DevParams&, const double*, const dmask_t*,
                                     const double*, double*, cudaStream_t);
template void launch_blockdiag<float>(const Grid&, const DevParams&, const float*, const dmask_t*,
                                      float*, cudaStream_t);
template void launch_blockdiag<double>(const Grid&, const DevParams&, const double*, const dmask_t*,
                                       double*, cudaStream_t);
template void launch_block_invert<float>(int64_t, const dmask_t*, float*, int*, cudaStream_t);
template void launch_block_invert<double>(int64_t, const dmask_t*, double*, int*, cudaStream_t);

}  // namespace pfm
