// Building blocks of the multigrid kernels (the transfers also compile for
// the host, where a test checks them against the oracle), shared by the
// single-problem kernels (mg_kernels.cu) and the batched kernels (batch.cu):
// integer-exact 1-D interpolation between structured grids on the same box,
// state injection, prolongation and restriction at one node, the Chebyshev
// smoothing updates at one node, the power-iteration start vector and one
// Gauss-Jordan elimination step of the dense coarse operator.
//
// Grid transfer in 1-D: fine node i sits at coarse coordinate i*nc/nf; with
// i*nc = I0*nf + rem, its interpolation weights are (1 - rem/nf) on coarse
// node I0 and rem/nf on I0+1. All index arithmetic is integer, so P and
// R = P^T use identical weights on nested (nf = 2 nc) and non-nested grids.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace pfm {

struct Interp1 {
  int i0;
  double t;  // weight of i0+1
};

__host__ __device__ __forceinline__ Interp1 interp1(int i, int nf, int nc) {
  // coarse coordinate of fine node i: i*nc/nf
  long long num = (long long)i * nc;
  int I0 = int(num / nf);
  long long rem = num - (long long)I0 * nf;
  if (I0 >= nc) { I0 = nc - 1; rem = nf; }
  return {I0, double(rem) / double(nf)};
}

// Value of the nodal field X (grid nx,ny,nz; field stride n) at the point with
// per-axis element index i0 and local coordinate t (trilinear).
template <typename T>
__host__ __device__ __forceinline__ double trilinear(const T* X, int nx, int ny, const int i0[3], const double t[3]) {
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int a0 = c & 1, a1 = (c >> 1) & 1, a2 = (c >> 2) & 1;
    double w = (a0 ? t[0] : 1.0 - t[0]) * (a1 ? t[1] : 1.0 - t[1]) * (a2 ? t[2] : 1.0 - t[2]);
    if (w == 0.0) continue;
    int64_t node = (i0[0] + a0) + int64_t(nx + 1) * ((i0[1] + a1) + int64_t(ny + 1) * (i0[2] + a2));
    s += w * double(X[node]);
  }
  return s;
}

// Coarse node idx: the fine Q1 field evaluated at its position, all fields.
__host__ __device__ __forceinline__ void inject_node(const Grid& f, const Grid& c, const double* __restrict__ Uf,
                                            double* __restrict__ Uc, int64_t idx) {
  const int64_t nnc = c.nn();
  const int64_t nnf = f.nn();
  int I = int(idx % (c.nx + 1));
  int J = int((idx / (c.nx + 1)) % (c.ny + 1));
  int K = int(idx / (int64_t(c.nx + 1) * (c.ny + 1)));
  // fine coordinate of coarse node: I*nf/nc
  int i0[3];
  double t[3];
  const int Ic[3] = {I, J, K}, nfv[3] = {f.nx, f.ny, f.nz}, ncv[3] = {c.nx, c.ny, c.nz};
  for (int d = 0; d < 3; ++d) {
    Interp1 p = interp1(Ic[d], ncv[d], nfv[d]);  // coarse node in fine coordinates
    i0[d] = p.i0;
    t[d] = p.t;
  }
  for (int fld = 0; fld < NF; ++fld) Uc[fld * nnc + idx] = trilinear(Uf + fld * nnf, f.nx, f.ny, i0, t);
}

// Fine node idx: xf += P xc at its free DOFs.
template <typename T>
__host__ __device__ __forceinline__ void prolong_node(const Grid& f, const Grid& c, const T* __restrict__ xc,
                                             const dmask_t* __restrict__ mf, T* __restrict__ xf, int64_t idx) {
  const int64_t nnf = f.nn();
  const int64_t nnc = c.nn();
  int i = int(idx % (f.nx + 1));
  int j = int((idx / (f.nx + 1)) % (f.ny + 1));
  int k = int(idx / (int64_t(f.nx + 1) * (f.ny + 1)));
  Interp1 px = interp1(i, f.nx, c.nx), py = interp1(j, f.ny, c.ny), pz = interp1(k, f.nz, c.nz);
  const int i0[3] = {px.i0, py.i0, pz.i0};
  const double t[3] = {px.t, py.t, pz.t};
  const dmask_t dm = mf[idx];
  for (int fld = 0; fld < NF; ++fld) {
    if ((dm >> fld) & 1) continue;
    xf[fld * nnf + idx] += T(trilinear(xc + fld * nnc, c.nx, c.ny, i0, t));
  }
}

// Coarse node idx: rc = (P^T rf) there, zero at its Dirichlet DOFs. Coarse
// node I collects fine nodes i with |i*nc - I*nf| < nf, weight
// 1 - |i*nc - I*nf|/nf (per axis).
template <typename T>
__host__ __device__ __forceinline__ void restrict_node(const Grid& f, const Grid& c, const T* __restrict__ rf,
                                              const dmask_t* __restrict__ mc, T* __restrict__ rc, int64_t idx) {
  const int64_t nnf = f.nn();
  const int64_t nnc = c.nn();
  const int Ic[3] = {int(idx % (c.nx + 1)), int((idx / (c.nx + 1)) % (c.ny + 1)),
                     int(idx / (int64_t(c.nx + 1) * (c.ny + 1)))};
  const int nfv[3] = {f.nx, f.ny, f.nz}, ncv[3] = {c.nx, c.ny, c.nz};
  int lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    long long center = (long long)Ic[d] * nfv[d];  // in units of 1/(nf*nc) ... i*nc vs I*nf
    // i*nc > I*nf - nf  and  i*nc < I*nf + nf
    long long a = center - nfv[d];
    long long b = center + nfv[d];
    int l = int(a >= 0 ? a / ncv[d] + 1 : 0);
    int h = int(b % ncv[d] == 0 ? b / ncv[d] - 1 : b / ncv[d]);
    if (l < 0) l = 0;
    if (h > nfv[d]) h = nfv[d];
    lo[d] = l;
    hi[d] = h;
  }
  const dmask_t dm = mc[idx];
  double acc[NF];
  for (int fld = 0; fld < NF; ++fld) acc[fld] = 0.0;
  for (int k = lo[2]; k <= hi[2]; ++k) {
    double wz = 1.0 - fabs(double((long long)k * ncv[2] - (long long)Ic[2] * nfv[2])) / nfv[2];
    for (int j = lo[1]; j <= hi[1]; ++j) {
      double wy = 1.0 - fabs(double((long long)j * ncv[1] - (long long)Ic[1] * nfv[1])) / nfv[1];
      for (int i = lo[0]; i <= hi[0]; ++i) {
        double wx = 1.0 - fabs(double((long long)i * ncv[0] - (long long)Ic[0] * nfv[0])) / nfv[0];
        const double w = wx * wy * wz;
        const int64_t fn = i + int64_t(f.nx + 1) * (j + int64_t(f.ny + 1) * k);
        for (int fld = 0; fld < NF; ++fld) acc[fld] += w * double(rf[fld * nnf + fn]);
      }
    }
  }
  for (int fld = 0; fld < NF; ++fld) rc[fld * nnc + idx] = ((dm >> fld) & 1) ? T(0) : T(acc[fld]);
}

// Nested grids (nf = 2 nc on every axis), the case of every level of a
// power-of-two hierarchy: fine node i of an axis coincides with coarse node
// i/2 (even i, weight 1) or lies midway between coarse nodes (i-1)/2 and
// (i+1)/2 (odd i, weights 1/2). These are the weights of the general
// transfers above on such grids; being powers of two they are exact in
// binary arithmetic, so the node bodies below form their sums in T (FP32 in
// the FP32 preconditioner) and take the node from its (i, j, k) position.

// Fine node (i, j, k): xf += P xc at its free DOFs.
template <typename T>
__host__ __device__ __forceinline__ void prolong_node_nested(const Grid& f, const Grid& c, const T* __restrict__ xc,
                                                    const dmask_t* __restrict__ mf, T* __restrict__ xf, int i,
                                                    int j, int k) {
  const int64_t nnf = f.nn(), nnc = c.nn();
  const int64_t idx = i + int64_t(f.nx + 1) * (j + int64_t(f.ny + 1) * k);
  const dmask_t dm = mf[idx];
  if (dm == MASK_ALL) return;
  const int ni = (i & 1) + 1, nj = (j & 1) + 1, nk = (k & 1) + 1;
  const T w = ((i & 1) ? T(0.5) : T(1)) * ((j & 1) ? T(0.5) : T(1)) * ((k & 1) ? T(0.5) : T(1));
  const int64_t c0 = (i >> 1) + int64_t(c.nx + 1) * ((j >> 1) + int64_t(c.ny + 1) * (k >> 1));
  const int64_t sy = c.nx + 1, sz = int64_t(c.nx + 1) * (c.ny + 1);
  for (int fld = 0; fld < NF; ++fld) {
    if ((dm >> fld) & 1) continue;
    const T* X = xc + fld * nnc + c0;
    T s = T(0);
    for (int a2 = 0; a2 < nk; ++a2)
      for (int a1 = 0; a1 < nj; ++a1)
        for (int a0 = 0; a0 < ni; ++a0) s += X[a0 + a1 * sy + a2 * sz];
    xf[fld * nnf + idx] += w * s;
  }
}

// Coarse node (I, J, K): rc = (P^T rf) there, zero at its Dirichlet DOFs;
// it collects fine nodes 2I-1, 2I, 2I+1 per axis with weights 1/2, 1, 1/2.
template <typename T>
__host__ __device__ __forceinline__ void restrict_node_nested(const Grid& f, const Grid& c, const T* __restrict__ rf,
                                                     const dmask_t* __restrict__ mc, T* __restrict__ rc, int I,
                                                     int J, int K) {
  const int64_t nnf = f.nn(), nnc = c.nn();
  const int64_t idx = I + int64_t(c.nx + 1) * (J + int64_t(c.ny + 1) * K);
  const dmask_t dm = mc[idx];
  const int64_t sy = f.nx + 1, sz = int64_t(f.nx + 1) * (f.ny + 1);
  for (int fld = 0; fld < NF; ++fld) {
    if ((dm >> fld) & 1) {
      rc[fld * nnc + idx] = T(0);
      continue;
    }
    const T* X = rf + fld * nnf;
    T acc = T(0);
    for (int dk = -1; dk <= 1; ++dk) {
      const int k = 2 * K + dk;
      if (k < 0 || k > f.nz) continue;
      T sj = T(0);
      for (int dj = -1; dj <= 1; ++dj) {
        const int j = 2 * J + dj;
        if (j < 0 || j > f.ny) continue;
        const T* row = X + j * sy + k * sz;
        T si = row[2 * I];
        if (I > 0) si += T(0.5) * row[2 * I - 1];
        if (2 * I + 1 <= f.nx) si += T(0.5) * row[2 * I + 1];
        sj += (dj ? T(0.5) : T(1)) * si;
      }
      acc += (dk ? T(0.5) : T(1)) * sj;
    }
    rc[fld * nnc + idx] = acc;
  }
}

inline __host__ __device__ bool nested(const Grid& f, const Grid& c) {
  return f.nx == 2 * c.nx && f.ny == 2 * c.ny && f.nz == 2 * c.nz;
}

// Chebyshev-accelerated point-block Jacobi at one node (Saad, Iterative
// Methods, Alg. 12.1 applied to D^-1 J). First step: d = c D^-1 r0 with
// r0 = src (also stored in r when copy_r), x = d (zero_x) or x += d.
template <typename T>
__device__ __forceinline__ void cheb_first_node(int64_t nn, const T* __restrict__ D, const T* src, T c, bool copy_r,
                                                bool zero_x, T* r, T* __restrict__ d, T* __restrict__ x,
                                                int64_t node) {
  T rv[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    rv[f] = src[f * nn + node];
    if (copy_r) r[f * nn + node] = rv[f];
  }
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    T s = T(0);
#pragma unroll
    for (int cc = 0; cc < NF; ++cc) s += D[(f * NF + cc) * nn + node] * rv[cc];
    const T dv = c * s;
    d[f * nn + node] = dv;
    x[f * nn + node] = zero_x ? dv : x[f * nn + node] + dv;
  }
}

// Later steps: r -= y; d = a d + c D^-1 r; x += d.
template <typename T>
__device__ __forceinline__ void cheb_step_node(int64_t nn, const T* __restrict__ D, const T* __restrict__ y, T a,
                                               T c, T* __restrict__ r, T* __restrict__ d, T* __restrict__ x,
                                               int64_t node) {
  T rv[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    rv[f] = r[f * nn + node] - y[f * nn + node];
    r[f * nn + node] = rv[f];
  }
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    T s = T(0);
#pragma unroll
    for (int cc = 0; cc < NF; ++cc) s += D[(f * NF + cc) * nn + node] * rv[cc];
    const T dv = a * d[f * nn + node] + c * s;
    d[f * nn + node] = dv;
    x[f * nn + node] += dv;
  }
}

// Deterministic start value of the power iteration at DOF index i of a level
// with nn nodes: in [-1, 1) from an integer hash of i, zero at Dirichlet DOFs.
__device__ __forceinline__ double power_init_value(int64_t i, int64_t nn, const dmask_t* __restrict__ mask) {
  uint64_t z = uint64_t(i) + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const double u = double(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  const int f = int(i / nn);
  return ((mask[i % nn] >> f) & 1) ? 0.0 : u;
}

// Gauss-Jordan elimination with partial pivoting on the augmented n x 2n
// matrix [K | I], with the row permutation kept implicit: step k takes the
// pivot row p chosen by step k-1 (largest |M[i][k]| over rows not yet used as
// pivots), eliminates column k from every other row (columns > k of the left
// half and the whole right half; column k itself is never read again), and in
// the same launch votes the pivot of step k+1 with a 64-bit atomicMax on
// (|value| as FP32 bits, row). Row p is left unscaled; at the end inverse row
// k is row piv[k] of the right half divided by M[piv[k]][k].
__device__ __forceinline__ unsigned long long pivot_key(double v, int row) {
  return (static_cast<unsigned long long>(__float_as_uint(float(fabs(v)))) << 32) | unsigned(row);
}

// Step k of the elimination for row i (one thread block; threads stride over
// the columns); the block with lead == true records the pivot.
__device__ __forceinline__ void gj_step_row(double* __restrict__ M, int n, int ld, int k,
                                            unsigned long long* __restrict__ keys, int* __restrict__ used,
                                            int* __restrict__ piv, int* singular, int i, bool lead) {
  const int p = int(keys[k] & 0xffffffffu);
  const double pk = M[int64_t(p) * ld + k];
  if (!(fabs(pk) > 0.0)) {
    if (lead && threadIdx.x == 0) *singular = 1;
    return;
  }
  if (lead && threadIdx.x == 0) piv[k] = p;
  if (i >= n) return;
  if (i == p) {
    if (threadIdx.x == 0) used[p] = 1;
    return;
  }
  const double f = M[int64_t(i) * ld + k] / pk;
  const bool candidate = (k + 1 < n) && !used[i];
  double* Mi = M + int64_t(i) * ld;
  const double* Mp = M + int64_t(p) * ld;
  if (f != 0.0) {
    for (int j = k + 1 + threadIdx.x; j < 2 * n; j += blockDim.x) {
      const double v = Mi[j] - f * Mp[j];
      Mi[j] = v;
      if (j == k + 1 && candidate) atomicMax(&keys[k + 1], pivot_key(v, i));
    }
  } else if (candidate && threadIdx.x == 0) {
    atomicMax(&keys[k + 1], pivot_key(Mi[k + 1], i));
  }
}

}  // namespace pfm
