// Device-side building blocks of the element kernels, shared by the
// single-problem kernels (fe_kernels.cu) and the batched kernels (batch.cu):
// Q1 tensor-product gather/scatter by warp shuffles, packed-Hessian index
// decoding, element-node mapping, and the per-element-block bodies of the
// tangent application and the linearisation.
//
// Thread mapping: 8 consecutive lanes form one element; lane l8 = 0..7 plays
// two roles: local node a = l8 (corner (a&1, a>>1&1, a>>2)) when gathering
// nodal data or scattering nodal results, and Gauss point q = l8 (point
// ((1 -+ 1/sqrt 3)/2) per axis) for the point physics. Values and gradients
// at the 8 points are a tensor product of 1-D 2x2 transforms, applied with
// three xor-shuffles (1, 2, 4) per axis; the scatter is the transposed
// transform. A warp holds 4 elements.
#pragma once

#include <cuda_fp16.h>

#include <cstdint>

#include "common.cuh"

namespace pfm {

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
static_assert(packed_row(0) == 0 && packed_row(NZ - 1) == 0 && packed_row(NZ) == 1 &&
                  packed_row(2 * NZ - 2) == 1 && packed_row(NH - 1) == NZ - 1 && packed_row(NH - 2) == NZ - 2 &&
                  packed_row(NH - 3) == NZ - 2 && packed_row(NH - 4) == NZ - 3,
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
                                             T eh[NV], T ge[3 * NV]) {
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
  for (int k = 0; k < NV; ++k) {
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
// binary16 store (FP32 arithmetic): 8 entries per vector
template <> struct Vec16<__half> {
  using type = uint4;
  static __device__ __forceinline__ void unpack(const uint4& x, float* o) {
    const __half2* h = reinterpret_cast<const __half2*>(&x);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float2 f = __half22float2(h[t]);
      o[2 * t] = f.x;
      o[2 * t + 1] = f.y;
    }
  }
};

template <typename T>
struct JParams {
  T G[NV][NV];
  T w, ihx, ihy, ihz;
};

struct NoLinTail {
  template <typename TC>
  __device__ void operator()(const TC*, const TC*, TC, int64_t, bool, int) const {}
};

// Gauss-point Hessians of element block blk (this warp; lane = 8 e + q),
// computed in TC (FP64 for the finest and the coarsest level, FP32 for the
// intermediate levels of an FP32 preconditioner) and stored in the requested
// precisions (null stores are skipped). tail(ge, gr, W, node, valid, l8)
// sees the point's eta gradients, energy gradient and energy density (the
// residual of the same state can be formed from them without a second
// evaluation of the point physics).
template <typename TC, typename Tail = NoLinTail>
__device__ __forceinline__ void linearize_lane(const Grid& g, const DevParams& P, const double* __restrict__ U,
                                               const double* __restrict__ Un, double* __restrict__ H64,
                                               float* __restrict__ H32, float* __restrict__ H32lo, int64_t blk,
                                               int lane, const Tail& tail = Tail{}) {
  const int64_t e = blk * 4 + (lane >> 3);
  const int l8 = lane & 7;
  const bool valid = e < g.ne();
  const int64_t nn = g.nn();
  const int64_t node = valid ? elem_node(g, e, l8) : 0;
  const TC ihx = TC(1.0 / g.hx), ihy = TC(1.0 / g.hy), ihz = TC(1.0 / g.hz);
  TC F[9], eh[NV], ge[3 * NV], ehn[NV];
  gather_state<TC>(U, nn, node, valid, l8, ihx, ihy, ihz, F, eh, ge);
#pragma unroll
  for (int k = 0; k < NV; ++k) ehn[k] = q1_value(valid ? TC(Un[(3 + k) * nn + node]) : TC(0));
  TC W, gr[NZ], Hp[NH];
  qp_local<TC, true>(P, F, eh, ehn, &W, gr, Hp);
  tail(ge, gr, W, node, valid, l8);
  for (int j = 0; j < NHP; ++j) {  // padding entries NH..NHP-1 are stored as zeros
    const double h = (valid && j < NH) ? double(Hp[j < NH ? j : 0]) : 0.0;
    if (H64) H64[hstore_offset<double>(blk, j, lane)] = h;
    if (H32) H32[hstore_offset<float>(blk, j, lane)] = float(h);
    if (H32lo) H32lo[hstore_offset<float>(blk, j, lane)] = float(h - double(float(h)));
  }
}

// Nodal NF x NF diagonal blocks (9 x 9 for N = 6). For local node a of the
// element whose Gauss-point Hessians sit in store block blk at lanes
// lane0..lane0+7, add to Db (upper triangle, row-major, NBD entries) the sum
// over the 8 points of w B_a(q)^T H_q B_a(q) plus the gradient-energy block.
template <typename T>
__device__ __forceinline__ void blockdiag_accumulate(const JParams<T>& jp, const T* __restrict__ H, int64_t blk,
                                                     int lane0, int a, T Db[NBD]) {
  constexpr int V = 16 / sizeof(T);
  using VT = typename Vec16<T>::type;
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
    T Hq[NHP];
    const VT* Hv = reinterpret_cast<const VT*>(H) + blk * (NHP / V) * 32 + lane0 + q;
#pragma unroll
    for (int jj = 0; jj < NHP / V; ++jj) Vec16<T>::unpack(Hv[jj * 32], Hq + jj * V);
    const T g2 = dN[0] * dN[0] + dN[1] * dN[1] + dN[2] * dN[2];
    int idx = 0;
#pragma unroll
    for (int r = 0; r < NF; ++r)
#pragma unroll
      for (int c = r; c < NF; ++c) {
        T s = T(0);
        if (r < 3 && c < 3) {
#pragma unroll
          for (int J = 0; J < 3; ++J)
#pragma unroll
            for (int L = 0; L < 3; ++L) {
              const int rr = 3 * r + J, cc = 3 * c + L;
              s += dN[J] * dN[L] * Hq[rr <= cc ? hidx(rr, cc) : hidx(cc, rr)];
            }
        } else if (r < 3) {
#pragma unroll
          for (int J = 0; J < 3; ++J) s += dN[J] * N * Hq[hidx(3 * r + J, 9 + (c - 3))];
        } else {
          s = N * N * Hq[hidx(9 + (r - 3), 9 + (c - 3))] + g2 * jp.G[r - 3][c - 3];
        }
        Db[idx++] += jp.w * s;
      }
  }
}

// (element e, local node a): its element's contribution added to the node's
// block D[(r*NF+c)*nn + node] with atomics (batched engine).
template <typename T>
__device__ __forceinline__ void blockdiag_elem_node(const Grid& g, const JParams<T>& jp, const T* __restrict__ H,
                                                    T* __restrict__ D, int64_t e, int a) {
  const int64_t nn = g.nn();
  const int64_t node = elem_node(g, e, a);
  T Db[NBD];
#pragma unroll
  for (int i = 0; i < NBD; ++i) Db[i] = T(0);
  blockdiag_accumulate<T>(jp, H, e >> 2, int(e & 3) * 8, a, Db);
  int idx = 0;
  for (int r = 0; r < NF; ++r)
    for (int c = r; c < NF; ++c) {
      atomicAdd(&D[(r * NF + c) * nn + node], Db[idx]);
      if (c != r) atomicAdd(&D[(c * NF + r) * nn + node], Db[idx]);
      ++idx;
    }
}

// In-place inverse of one node's NF x NF block (Dirichlet rows/columns replaced
// by identity first) by Gauss-Jordan elimination with partial pivoting; a
// singular block sets *singular and is replaced by the identity.
template <typename T>
__device__ __forceinline__ void block_invert_node(int64_t nn, const dmask_t* __restrict__ mask, T* __restrict__ D,
                                                  int* singular, int64_t node) {
  const dmask_t dm = mask[node];
  T a[NF][NF], x[NF][NF];
  for (int r = 0; r < NF; ++r)
    for (int c = 0; c < NF; ++c) {
      T v = D[(r * NF + c) * nn + node];
      if (((dm >> r) & 1) || ((dm >> c) & 1)) v = (r == c) ? T(1) : T(0);
      a[r][c] = v;
      x[r][c] = (r == c) ? T(1) : T(0);
    }
  bool bad = false;
  for (int k = 0; k < NF; ++k) {
    int p = k;
    T best = fabs(a[k][k]);
    for (int r = k + 1; r < NF; ++r)
      if (fabs(a[r][k]) > best) { best = fabs(a[r][k]); p = r; }
    if (!(best > T(0))) { bad = true; break; }
    if (p != k)
      for (int c = 0; c < NF; ++c) {
        T t = a[k][c]; a[k][c] = a[p][c]; a[p][c] = t;
        t = x[k][c]; x[k][c] = x[p][c]; x[p][c] = t;
      }
    const T ip = T(1) / a[k][k];
    for (int c = 0; c < NF; ++c) { a[k][c] *= ip; x[k][c] *= ip; }
    for (int r = 0; r < NF; ++r) {
      if (r == k) continue;
      const T f = a[r][k];
      if (f == T(0)) continue;
      for (int c = 0; c < NF; ++c) { a[r][c] -= f * a[k][c]; x[r][c] -= f * x[k][c]; }
    }
  }
  if (bad) {
    atomicExch(singular, 1);
    for (int r = 0; r < NF; ++r)
      for (int c = 0; c < NF; ++c) x[r][c] = (r == c) ? T(1) : T(0);
  }
  for (int r = 0; r < NF; ++r)
    for (int c = 0; c < NF; ++c) D[(r * NF + c) * nn + node] = x[r][c];
}

// Element constants of a level: gradient-energy matrix, quadrature weight and
// inverse spacings (host-side construction).
template <typename T>
inline JParams<T> make_jparams(const Grid& g, const DevParams& P) {
  JParams<T> jp;
  for (int k = 0; k < NV; ++k)
    for (int l = 0; l < NV; ++l) jp.G[k][l] = T(P.G[k][l]);
  jp.w = T(g.w());
  jp.ihx = T(1.0 / g.hx);
  jp.ihy = T(1.0 / g.hy);
  jp.ihz = T(1.0 / g.hz);
  return jp;
}

// Nodal result r of this lane (element e = 4 blk + lane/8, local node
// lane%8) for DOF row idx = f nn + node: added to y with an atomic (DET
// false), or (DET true, atomic-free) stored to the per-(element, node)
// scratch W[f ws + 32 blk + lane], 0 where the row is skipped; a node pass
// then sums each node's contributions in a fixed order.
template <bool DET, typename TY, typename TW, typename TR>
__device__ __forceinline__ void scatter_row(TY* __restrict__ y, TW* __restrict__ W, int64_t ws, int f, int64_t blk,
                                            int lane, int64_t idx, TR r, bool on) {
  if constexpr (DET) {
    W[f * ws + blk * 32 + lane] = on ? TW(r) : TW(0);
  } else {
    if (on) atomicAdd(&y[idx], TY(r));
  }
}

// ---- BEGIN tangent application kernel
// y += J v on the 4 elements of block blk (this warp; lane = 0..31): gather v
// at the element nodes (Dirichlet DOFs read as 0), dz = (grad du, d eta_hat)
// at the Gauss points, sigma = H dz from the packed symmetric store, plus the
// constant gradient-energy term, scattered back with atomics.
template <typename T>
__device__ __forceinline__ void japply_block(const Grid& g, const JParams<T>& jp, const T* __restrict__ H,
                                             const dmask_t* __restrict__ mask, const T* __restrict__ v,
                                             T* __restrict__ y, int64_t blk, int lane) {
  constexpr int V = 16 / sizeof(T);
  using VT = typename Vec16<T>::type;
  const int l8 = lane & 7;
  const int64_t nn = g.nn();
  const int64_t e = blk * 4 + (lane >> 3);
  const bool valid = e < g.ne();
  const int64_t node = valid ? elem_node(g, e, l8) : 0;
  const dmask_t dm = valid ? mask[node] : MASK_ALL;
  T dz[NZ], ge[3 * NV];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T x = ((dm >> i) & 1) ? T(0) : v[i * nn + node];
    T val;
    q1_gather(x, l8, jp.ihx, jp.ihy, jp.ihz, val, dz[3 * i], dz[3 * i + 1], dz[3 * i + 2]);
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    T x = ((dm >> (3 + k)) & 1) ? T(0) : v[(3 + k) * nn + node];
    q1_gather(x, l8, jp.ihx, jp.ihy, jp.ihz, dz[9 + k], ge[3 * k], ge[3 * k + 1], ge[3 * k + 2]);
  }
  // sigma = H dz from the packed symmetric store
  T sg[NZ];
#pragma unroll
  for (int r = 0; r < NZ; ++r) sg[r] = T(0);
  const VT* Hv = reinterpret_cast<const VT*>(H) + blk * (NHP / V) * 32 + lane;
#pragma unroll
  for (int j = 0; j < NHP / V; ++j) {
    T hv[V];
    Vec16<T>::unpack(__ldcs(Hv + j * 32), hv);
#pragma unroll
    for (int t = 0; t < V; ++t) {
      const int idx = j * V + t;
      if (idx >= NH) continue;  // zero padding of the store
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
  for (int k = 0; k < NV; ++k) {
    T gf[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      T s = T(0);
#pragma unroll
      for (int l = 0; l < NV; ++l) s += jp.G[k][l] * ge[3 * l + d];
      gf[d] = w * s;
    }
    T r = q1_scatter(w * sg[9 + k], gf[0], gf[1], gf[2], l8, jp.ihx, jp.ihy, jp.ihz);
    if (valid && !((dm >> (3 + k)) & 1)) atomicAdd(&y[(3 + k) * nn + node], r);
  }
}
// ---- END tangent application kernel

// The same body in the atomic-free form (deterministic mode): the lane's
// nodal results go to the scratch W for the node pass (scatter_row).
// y += J v on the 4 elements of block blk (this warp; lane = 0..31): gather v
// at the element nodes (Dirichlet DOFs read as 0), dz = (grad du, d eta_hat)
// at the Gauss points, sigma = H dz from the packed symmetric store, plus the
// constant gradient-energy term, scattered back with atomics.
template <typename T>
__device__ __forceinline__ void japply_block_det(const Grid& g, const JParams<T>& jp, const T* __restrict__ H,
                                                 const dmask_t* __restrict__ mask, const T* __restrict__ v,
                                                 T* __restrict__ W, int64_t ws, int64_t blk, int lane) {
  constexpr int V = 16 / sizeof(T);
  using VT = typename Vec16<T>::type;
  const int l8 = lane & 7;
  const int64_t nn = g.nn();
  const int64_t e = blk * 4 + (lane >> 3);
  const bool valid = e < g.ne();
  const int64_t node = valid ? elem_node(g, e, l8) : 0;
  const dmask_t dm = valid ? mask[node] : MASK_ALL;
  T dz[NZ], ge[3 * NV];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T x = ((dm >> i) & 1) ? T(0) : v[i * nn + node];
    T val;
    q1_gather(x, l8, jp.ihx, jp.ihy, jp.ihz, val, dz[3 * i], dz[3 * i + 1], dz[3 * i + 2]);
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    T x = ((dm >> (3 + k)) & 1) ? T(0) : v[(3 + k) * nn + node];
    q1_gather(x, l8, jp.ihx, jp.ihy, jp.ihz, dz[9 + k], ge[3 * k], ge[3 * k + 1], ge[3 * k + 2]);
  }
  // sigma = H dz from the packed symmetric store
  T sg[NZ];
#pragma unroll
  for (int r = 0; r < NZ; ++r) sg[r] = T(0);
  const VT* Hv = reinterpret_cast<const VT*>(H) + blk * (NHP / V) * 32 + lane;
#pragma unroll
  for (int j = 0; j < NHP / V; ++j) {
    T hv[V];
    Vec16<T>::unpack(__ldcs(Hv + j * 32), hv);
#pragma unroll
    for (int t = 0; t < V; ++t) {
      const int idx = j * V + t;
      if (idx >= NH) continue;  // zero padding of the store
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
    scatter_row<true>(static_cast<T*>(nullptr), W, ws, i, blk, lane, i * nn + node, r, valid && !((dm >> i) & 1));
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    T gf[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      T s = T(0);
#pragma unroll
      for (int l = 0; l < NV; ++l) s += jp.G[k][l] * ge[3 * l + d];
      gf[d] = w * s;
    }
    T r = q1_scatter(w * sg[9 + k], gf[0], gf[1], gf[2], l8, jp.ihx, jp.ihy, jp.ihz);
    scatter_row<true>(static_cast<T*>(nullptr), W, ws, 3 + k, blk, lane, (3 + k) * nn + node, r, valid && !((dm >> (3 + k)) & 1));
  }
}


// y += J v on element block blk from a binary16 copy of the store holding
// s H (FP32 arithmetic): the same gather, contraction and scatter as
// japply_block, with the Hessian part weighted by wh = w / s. The FP32 and
// FP64 applications keep their own body above.
template <bool DET = false>
__device__ __forceinline__ void japply_block_h16(const Grid& g, const JParams<float>& jp, float wh,
                                                 const __half* __restrict__ H, const dmask_t* __restrict__ mask,
                                                 const float* __restrict__ v, float* __restrict__ y, int64_t blk,
                                                 int lane, float* __restrict__ W = nullptr, int64_t ws = 0) {
  constexpr int V = 8;
  const int l8 = lane & 7;
  const int64_t nn = g.nn();
  const int64_t e = blk * 4 + (lane >> 3);
  const bool valid = e < g.ne();
  const int64_t node = valid ? elem_node(g, e, l8) : 0;
  const dmask_t dm = valid ? mask[node] : MASK_ALL;
  float dz[NZ], ge[3 * NV];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float x = ((dm >> i) & 1) ? 0.f : v[i * nn + node];
    float val;
    q1_gather(x, l8, jp.ihx, jp.ihy, jp.ihz, val, dz[3 * i], dz[3 * i + 1], dz[3 * i + 2]);
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    float x = ((dm >> (3 + k)) & 1) ? 0.f : v[(3 + k) * nn + node];
    q1_gather(x, l8, jp.ihx, jp.ihy, jp.ihz, dz[9 + k], ge[3 * k], ge[3 * k + 1], ge[3 * k + 2]);
  }
  float sg[NZ];
#pragma unroll
  for (int r = 0; r < NZ; ++r) sg[r] = 0.f;
  const uint4* Hv = reinterpret_cast<const uint4*>(H) + blk * (NHP / V) * 32 + lane;
#pragma unroll
  for (int j = 0; j < NHP / V; ++j) {
    float hv[V];
    Vec16<__half>::unpack(__ldcs(Hv + j * 32), hv);
#pragma unroll
    for (int t = 0; t < V; ++t) {
      const int idx = j * V + t;
      if (idx >= NH) continue;  // zero padding of the store
      const int r = packed_row(idx);
      const int c = r + (idx - packed_row_start(r));
      sg[r] += hv[t] * dz[c];
      if (c != r) sg[c] += hv[t] * dz[r];
    }
  }
  const float w = jp.w;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float r = q1_scatter_grad(wh * sg[3 * i], wh * sg[3 * i + 1], wh * sg[3 * i + 2], l8, jp.ihx, jp.ihy, jp.ihz);
    scatter_row<DET>(y, W, ws, i, blk, lane, i * nn + node, r, valid && !((dm >> i) & 1));
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    float gf[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float s = 0.f;
#pragma unroll
      for (int l = 0; l < NV; ++l) s += jp.G[k][l] * ge[3 * l + d];
      gf[d] = w * s;
    }
    float r = q1_scatter(wh * sg[9 + k], gf[0], gf[1], gf[2], l8, jp.ihx, jp.ihy, jp.ihz);
    scatter_row<DET>(y, W, ws, 3 + k, blk, lane, (3 + k) * nn + node, r, valid && !((dm >> (3 + k)) & 1));
  }
}


// Output vector i of the binary16 copy s H of an FP32 store: vector i =
// (blk*(NHP/8) + j)*32 + lane holds entries 8j..8j+7 of that lane, which the
// FP32 store keeps in its vectors (blk*(NHP/4) + 2j)*32 + lane and the one 32
// vectors later.
__device__ __forceinline__ uint4 half_vector(const float4* __restrict__ H32, float s, int64_t i) {
  const int64_t lane = i & 31, bj = i >> 5;
  const int64_t blk = bj / (NHP / 8), j = bj % (NHP / 8);
  const int64_t src = (blk * (NHP / 4) + 2 * j) * 32 + lane;
  const float4 a = H32[src], b = H32[src + 32];
  uint4 o;
  __half2* h = reinterpret_cast<__half2*>(&o);
  h[0] = __floats2half2_rn(a.x * s, a.y * s);
  h[1] = __floats2half2_rn(a.z * s, a.w * s);
  h[2] = __floats2half2_rn(b.x * s, b.y * s);
  h[3] = __floats2half2_rn(b.z * s, b.w * s);
  return o;
}

// running max of |x| in which a NaN counts as +infinity (so that a
// non-finite store is always detected)
__device__ __forceinline__ float absmax_step(float m, float x) {
  const float a = fabsf(x);
  return a == a ? fmaxf(m, a) : __int_as_float(0x7f800000);
}

// ---------------------------------------------------------------------------
// Bulk copies from global to shared memory by the tensor memory accelerator
// (cp.async.bulk, completion counted in bytes on an mbarrier), and bounded
// waits on those barriers.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make barrier initialisations visible to the asynchronous (TMA) proxy
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// order this CTA's generic-proxy accesses of shared memory before later
// asynchronous-proxy writes into it
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// L2 policy for data read once (the Hessian store): evicted first, so the
// nodal vectors that every element reads stay resident
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// bytes (a multiple of 16) from global src to shared dst (both 16-byte
// aligned); completion adds to the barrier's transaction count
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Warp-uniform bounded wait for the completion of the barrier phase with the
// given parity: true once every lane has seen it, false after about
// limit_ns nanoseconds (the decision is lane 0's clock, broadcast).
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* bar, unsigned parity, uint64_t limit_ns) {
  if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
  const uint64_t t0 = global_ns();
  for (unsigned it = 1;; ++it) {
    if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
    if ((it & 63u) == 0u) {
      const uint64_t dt = __shfl_sync(0xffffffffu, global_ns() - t0, 0);
      if (dt > limit_ns) return false;
    }
  }
}

// Element constants of the staged tangent application. The Hessian part is
// weighted through the input: the gathered vector is x' = wh x (wh = w for an
// FP32 store, w / s for a binary16 copy holding s H), so sigma = H dz' is
// already weighted, and the gradient-energy matrix carries w / wh.
struct JStaged {
  float Gs[NV][NV];  // (w / wh) G
  float wh, ihx, ihy, ihz;
  FastDiv dx, dy;    // element index -> (i, j, k): e = i + nx (j + ny k)
#if PFM_NV == 6
  // G = g_alpha I + g_beta 1 1^T (both times w / wh) when g_diag_plus_ones:
  // the form G takes when every austenite-variant pair shares one interface
  // energy and every variant-variant pair another (Sec. 5.1 data); the
  // twelve-variant build keeps the general product only (with both forms its
  // fully unrolled body takes nvcc more than 60 GB and 15 minutes)
  int g_diag_plus_ones;
  float g_alpha, g_beta;
#endif
};

// First half of the staged body, in two steps so that a warp can issue the
// loads of its next element block before the arithmetic of the current one:
// staged_load finds this lane's element node and loads its Dirichlet mask
// and the NF input values (no load depends on another); staged_shuffle then
// forms dz' = wh (grad du, d eta_hat) and the gradients ge' of the
// order-parameter increments at this lane's Gauss point.
struct StagedLane {
  int64_t node;
  dmask_t dm;
  bool valid;
  float x[NF];
};
__device__ __forceinline__ void staged_load(const Grid& g, const JStaged& jp, const dmask_t* __restrict__ mask,
                                            const float* __restrict__ v, int64_t blk, int lane, StagedLane& s) {
  const int l8 = lane & 7;
  const uint32_t e = uint32_t(blk) * 4u + uint32_t(lane >> 3);  // ne < 2^31 (checked by the launcher)
  s.valid = e < uint32_t(g.ne());
  s.node = 0;  // padding lanes read node 0 (in bounds) and use none of it
  if (s.valid) {
    const uint32_t r = jp.dx.div(e);
    const uint32_t ei = e - r * uint32_t(g.nx);
    const uint32_t ek = jp.dy.div(r);
    const uint32_t ej = r - ek * uint32_t(g.ny);
    s.node = int64_t(ei + (l8 & 1)) +
             int64_t(g.nx + 1) * (int64_t(ej + ((l8 >> 1) & 1)) + int64_t(g.ny + 1) * int64_t(ek + (l8 >> 2)));
  }
  s.dm = mask[s.node];
  const int64_t nn = g.nn();
  const float* vp = v + s.node;
#pragma unroll
  for (int f = 0; f < NF; ++f) s.x[f] = vp[f * nn];
}
__device__ __forceinline__ void staged_shuffle(const JStaged& jp, StagedLane& s, int lane, float dz[NZ],
                                               float ge[3 * NV]) {
  const int l8 = lane & 7;
  if (!s.valid) s.dm = MASK_ALL;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float x = ((s.dm >> i) & 1) ? 0.f : jp.wh * s.x[i];
    float val;
    q1_gather(x, l8, jp.ihx, jp.ihy, jp.ihz, val, dz[3 * i], dz[3 * i + 1], dz[3 * i + 2]);
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const float x = ((s.dm >> (3 + k)) & 1) ? 0.f : jp.wh * s.x[3 + k];
    q1_gather(x, l8, jp.ihx, jp.ihy, jp.ihz, dz[9 + k], ge[3 * k], ge[3 * k + 1], ge[3 * k + 2]);
  }
}

// Second half: sigma = H dz' from the element block's Hessians staged in
// shared memory (lane-interleaved 16-byte vectors, the layout of the global
// store), the gradient-energy term, and the scatter with atomics.
template <typename S>
__device__ __forceinline__ void staged_contract_scatter(const Grid& g, const JStaged& jp, const unsigned char* Hs,
                                                        const StagedLane& s, float* __restrict__ y, int lane,
                                                        const float dz[NZ],
                                                        const float ge[3 * NV]) {
  constexpr int V = 16 / sizeof(S);
  using VT = typename Vec16<S>::type;
  const int l8 = lane & 7;
  const int64_t nn = g.nn();
  float sg[NZ];
#pragma unroll
  for (int r = 0; r < NZ; ++r) sg[r] = 0.f;
  const VT* Hv = reinterpret_cast<const VT*>(Hs) + lane;
#pragma unroll
  for (int j = 0; j < NHP / V; ++j) {
    float hv[V];
    Vec16<S>::unpack(Hv[j * 32], hv);
#pragma unroll
    for (int t = 0; t < V; ++t) {
      const int idx = j * V + t;
      if (idx >= NH) continue;  // zero padding of the store
      const int r = packed_row(idx);
      const int c = r + (idx - packed_row_start(r));
      sg[r] += hv[t] * dz[c];
      if (c != r) sg[c] += hv[t] * dz[r];
    }
  }
  float* yp = y + s.node;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float r = q1_scatter_grad(sg[3 * i], sg[3 * i + 1], sg[3 * i + 2], l8, jp.ihx, jp.ihy, jp.ihz);
    if (s.valid && !((s.dm >> i) & 1)) atomicAdd(yp + i * nn, r);
  }
#if PFM_NV == 6
  // gradient-energy term G ge per direction: with G = alpha I + beta 1 1^T
  // it is alpha ge_k + beta sum_l ge_l (12 operations instead of 36)
  float bsum[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float t = 0.f;
#pragma unroll
    for (int l = 0; l < NV; ++l) t += ge[3 * l + d];
    bsum[d] = jp.g_beta * t;
  }
#endif
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    float gf[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#if PFM_NV == 6
      if (jp.g_diag_plus_ones) {
        gf[d] = fmaf(jp.g_alpha, ge[3 * k + d], bsum[d]);
        continue;
      }
#endif
      float a = 0.f;
#pragma unroll
      for (int l = 0; l < NV; ++l) a += jp.Gs[k][l] * ge[3 * l + d];
      gf[d] = a;
    }
    const float r = q1_scatter(sg[9 + k], gf[0], gf[1], gf[2], l8, jp.ihx, jp.ihy, jp.ihz);
    if (s.valid && !((s.dm >> (3 + k)) & 1)) atomicAdd(yp + (3 + k) * nn, r);
  }
}

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
  dfl G[NV][NV];
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

inline DfConst make_dfconst(const Grid& g, const DevParams& P) {
  DfConst k;
  k.ga = df_host(GA);
  k.gb = df_host(GB);
  k.ihx = df_host(1.0 / g.hx);
  k.ihy = df_host(1.0 / g.hy);
  k.ihz = df_host(1.0 / g.hz);
  k.w = df_host(g.w());
  for (int a = 0; a < NV; ++a)
    for (int b = 0; b < NV; ++b) k.G[a][b] = df_host(P.G[a][b]);
  return k;
}

// Compensated accumulator s + c for sums of products h * z with h = hh + hl
// (two FP32 parts) and z a double-float number (the compensated dot product
// of Ogita, Rump and Oishi 2005): the leading product hh * z.hi is split
// exactly by a fused multiply-add, its sum into s by TwoSum, and every
// rounding error and the two small cross products go into c. Twelve FP32
// operations per term instead of eighteen for a double-float multiply-add,
// with the same (twice FP32) working accuracy.
struct cacc {
  float s, c;
};
__device__ __forceinline__ void cacc_add(cacc& a, float hh, float hl, dfl z) {
  const float p = __fmul_rn(hh, z.hi);
  const float e = __fmaf_rn(hh, z.hi, -p);
  const float s = __fadd_rn(a.s, p);
  const float bb = __fsub_rn(s, a.s);
  const float q = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  float c = __fmaf_rn(hh, z.lo, a.c);
  c = __fmaf_rn(hl, z.hi, c);
  a.c = __fadd_rn(c, __fadd_rn(q, e));
  a.s = s;
}
__device__ __forceinline__ dfl cacc_value(const cacc& a) { return df_two_sum(a.s, a.c); }

// y += J v on element block blk in double-float arithmetic: v in FP32
// (exact input), the tangent as Hhi + Hlo (two FP32 stores of the FP64
// Hessians), element contributions added to the FP64 output y.
// Unroll factor of the double-float contraction loop: fully unrolled (every
// accumulator index known at compile time, so the accumulators stay in
// registers) for six variants; the twelve-variant body keeps a factor of 2
// (its fully unrolled form is twice as large). Measured at 128^3 with six
// variants: 7.72 ms per application fully unrolled at 2 CTAs of 256 threads per
// SM (128 registers) against 11.58 ms unrolled by 2 at 8 CTAs (32 registers).
#ifndef PFM_DF_UNROLL
#define PFM_DF_UNROLL (PFM_NV == 6 ? NHP / 4 : 2)
#endif
constexpr int kDfUnroll = PFM_DF_UNROLL;

template <bool DET = false>
__device__ __forceinline__ void japply_df_block(const Grid& g, const DfConst& k, const float* __restrict__ Hhi,
                                                const float* __restrict__ Hlo, const dmask_t* __restrict__ mask,
                                                const float* __restrict__ v, double* __restrict__ y, int64_t blk,
                                                int lane, double* __restrict__ W = nullptr, int64_t ws = 0) {
  const int l8 = lane & 7;
  const int64_t nn = g.nn();
  const int64_t e = blk * 4 + (lane >> 3);
  const bool valid = e < g.ne();
  const int64_t node = valid ? elem_node(g, e, l8) : 0;
  const dmask_t dm = valid ? mask[node] : MASK_ALL;
  dfl dz[NZ], ge[3 * NV];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float x = ((dm >> i) & 1) ? 0.f : v[i * nn + node];
    dfl val;
    q1_gather_df(dfl{x, 0.f}, l8, k, val, dz[3 * i], dz[3 * i + 1], dz[3 * i + 2]);
  }
#pragma unroll
  for (int kk = 0; kk < NV; ++kk) {
    const float x = ((dm >> (3 + kk)) & 1) ? 0.f : v[(3 + kk) * nn + node];
    q1_gather_df(dfl{x, 0.f}, l8, k, dz[9 + kk], ge[3 * kk], ge[3 * kk + 1], ge[3 * kk + 2]);
  }
  cacc acc[NZ];
#pragma unroll
  for (int r = 0; r < NZ; ++r) acc[r] = cacc{0.f, 0.f};
  const float4* Hh = reinterpret_cast<const float4*>(Hhi) + blk * (NHP / 4) * 32 + lane;
  const float4* Hl = reinterpret_cast<const float4*>(Hlo) + blk * (NHP / 4) * 32 + lane;
#pragma unroll kDfUnroll
  for (int j = 0; j < NHP / 4; ++j) {
    float hh[4], hl[4];
    Vec16<float>::unpack(__ldcs(Hh + j * 32), hh);
    Vec16<float>::unpack(__ldcs(Hl + j * 32), hl);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int idx = j * 4 + t;
      if (idx >= NH) continue;  // zero padding of the store
      const int r = packed_row(idx);
      const int c = r + (idx - packed_row_start(r));
      cacc_add(acc[r], hh[t], hl[t], dz[c]);
      if (c != r) cacc_add(acc[c], hh[t], hl[t], dz[r]);
    }
  }
  dfl sg[NZ];
#pragma unroll
  for (int r = 0; r < NZ; ++r) sg[r] = cacc_value(acc[r]);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    dfl r = q1_scatter_df(dfl{0.f, 0.f}, df_mul(k.w, sg[3 * i]), df_mul(k.w, sg[3 * i + 1]),
                          df_mul(k.w, sg[3 * i + 2]), false, l8, k);
    scatter_row<DET>(y, W, ws, i, blk, lane, i * nn + node, double(r.hi) + double(r.lo), valid && !((dm >> i) & 1));
  }
#pragma unroll
  for (int kk = 0; kk < NV; ++kk) {
    dfl gf[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      cacc s = cacc{0.f, 0.f};
#pragma unroll
      for (int l = 0; l < NV; ++l) cacc_add(s, k.G[kk][l].hi, k.G[kk][l].lo, ge[3 * l + d]);
      gf[d] = df_mul(k.w, cacc_value(s));
    }
    dfl r = q1_scatter_df(df_mul(k.w, sg[9 + kk]), gf[0], gf[1], gf[2], true, l8, k);
    scatter_row<DET>(y, W, ws, 3 + kk, blk, lane, (3 + kk) * nn + node, double(r.hi) + double(r.lo),
                     valid && !((dm >> (3 + kk)) & 1));
  }
}

// Node pass of the atomic-free scatter: node n of grid g sums, for every
// field f, the contributions W[f ws + 32 (e/4) + 8 (e%4) + a] of its (up to 8)
// adjacent elements e (local node a) in a fixed order (z, then y, then x),
// and writes y[f nn + n]; a Dirichlet row gets v[f nn + n] (identity row of
// the tangent) or 0 when v is null (residual).
template <typename TW, typename TV, typename TY>
__device__ __forceinline__ void node_gather(const Grid& g, const TW* __restrict__ W, int64_t ws,
                                            const dmask_t* __restrict__ mask, const TV* __restrict__ v,
                                            TY* __restrict__ y, int64_t n) {
  const int64_t nn = g.nn();
  const int i = int(n % (g.nx + 1));
  const int j = int((n / (g.nx + 1)) % (g.ny + 1));
  const int k = int(n / (int64_t(g.nx + 1) * (g.ny + 1)));
  int64_t col[8];
  int cnt = 0;
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
        col[cnt++] = (e >> 2) * 32 + (e & 3) * 8 + a;
      }
    }
  }
  const dmask_t dm = mask[n];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    if ((dm >> f) & 1) {
      y[f * nn + n] = v ? TY(v[f * nn + n]) : TY(0);
      continue;
    }
    TW s = TW(0);
    for (int c = 0; c < cnt; ++c) s += W[f * ws + col[c]];
    y[f * nn + n] = TY(s);
  }
}

}  // namespace pfm
