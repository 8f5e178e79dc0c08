// Quadrature-point physics of the multivariant finite-strain phase-field
// model: local energy density, its gradient and its exact 15x15 Hessian with
// respect to z = (F_iJ row-major, eta_1..eta_6).
//
// Model (Sec. 2.1-2.3, Sec. 3.1): eta_0 = 1 - sum eta_k; F^t = sum_i eta_i U_i
// (Eq. LinMix); F^e = F (F^t)^-1, C^e = F^eT F^e, H^e = 1/2 log C^e and
// F_el = 1/2 det(F^t) H^e . L(eta) H^e with L = sum_i eta_i L_i
// (Eq. elasticEn); chemical sum eta_i F_i^0; local part of the double
// obstacle sum_{i<j} 4 gamma_ij/(pi ell_ij) eta_i eta_j (Eq. IntEnergy);
// backward-Euler dissipation sum (eta_i - eta_i,n)^2/(2 m_i tau) (Sec. 2.3);
// penalty sum 1/2 eps <eta_i>_-^2 (Eq. PenPot). The gradient part of the
// interface energy is a constant quadratic form handled by the element
// kernels.
//
// Derivatives. With A = (F^t)^-1, M = F A, E = C^e = M^T M and the energy
// written as g(E, eta) = 1/2 J_t h(E):L(eta):h(E), J_t = det F^t, the chain
// rule gives first and second derivatives from those of E and of h = 1/2 log.
// The derivatives of the matrix logarithm use the spectral decomposition of
// E (cyclic Jacobi) and the Daleckii-Krein formulas: in the eigenbasis,
// Dlog[X]_ab = f1(l_a,l_b) X_ab and
// D2log[X,Y]_ab = sum_c f2(l_a,l_c,l_b) (X_ac Y_cb + Y_ac X_cb), with f1, f2
// the first and second divided differences of log. These are exact for
// repeated eigenvalues as long as the divided differences are evaluated
// without cancellation, which dd1_log / dd2_log do (log1p quotient; Taylor
// series of the second divided difference about the mean when all three
// arguments are close).
//
// Pade modes (Sec. 2.4, Eqs. pade11, pade22, pade33). The paper's (m,m)
// approximant of H^e is the primary matrix function h = 1/2 r_m(C^e), r_m the
// [m/m] Pade approximant of log about 1. The m-point Gauss-Legendre rule on
// log x = int_0^1 (x - 1)/(1 + s (x - 1)) ds is that approximant (Dieci,
// Morini and Papini, 1996): r_m(x) = sum_k w_k (x - 1) p_k(x)^-1 with
// p_k(x) = 1 + s_k (x - 1). The same spectral route then applies with
// divided differences that are products of the reciprocals 1/p_k, free of
// cancellation for any eigenvalue spread:
// r_m[a,b] = sum_k w_k / (p_k(a) p_k(b)),
// r_m[a,b,c] = -sum_k w_k s_k / (p_k(a) p_k(b) p_k(c)).
#pragma once

#ifdef __CUDACC__
#define PFM_HD __host__ __device__ __forceinline__
#define PFM_HD_BIG __host__ __device__
#else
#define PFM_HD_BIG inline
#include <cmath>
#define PFM_HD inline
using std::sqrt;
using std::log;
using std::log1p;
using std::fabs;
#endif

namespace pfm {

#ifdef __CUDACC__
// keep the C math functions visible next to the double-float overloads below
using ::fabs;
using ::log;
using ::log1p;
using ::sqrt;

// ---------------------------------------------------------------------------
// Double-float number hi + lo (two FP32 values, |lo| <= ulp(hi)/2): about 48
// significant bits from FP32 adds, multiplies and fused multiply-adds only
// (Dekker 1971; Knuth's TwoSum), so the point physics can run on the FP32
// pipes. Division, square root and the logarithms go through FP64 (a handful
// per Gauss point). The _rn intrinsics keep the compiler from contracting or
// reassociating the error-free transformations.
struct df64 {
  float hi, lo;
  df64() = default;
  __device__ __forceinline__ df64(double x) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - double(hi));
  }
  __device__ __forceinline__ explicit operator double() const { return double(hi) + double(lo); }
  __device__ __forceinline__ static df64 make(float h, float l) {
    df64 r;
    r.hi = h;
    r.lo = l;
    return r;
  }
};

__device__ __forceinline__ df64 df64_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return df64::make(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return df64_fast_two_sum(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64::make(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df64_fast_two_sum(p, e);
}
__device__ __forceinline__ df64 operator/(df64 a, df64 b) { return df64(double(a) / double(b)); }
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }
__device__ __forceinline__ df64& operator/=(df64& a, df64 b) { return a = a / b; }
__device__ __forceinline__ bool operator<(df64 a, df64 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(df64 a, df64 b) { return b < a; }
__device__ __forceinline__ bool operator<=(df64 a, df64 b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(df64 a, df64 b) { return !(a < b); }
__device__ __forceinline__ bool operator==(df64 a, df64 b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(df64 a, df64 b) { return !(a == b); }
__device__ __forceinline__ df64 fabs(df64 a) { return a.hi < 0.f ? -a : a; }
__device__ __forceinline__ df64 sqrt(df64 a) { return df64(::sqrt(double(a))); }
__device__ __forceinline__ df64 log(df64 a) { return df64(::log(double(a))); }
__device__ __forceinline__ df64 log1p(df64 a) { return df64(::log1p(double(a))); }
__device__ __forceinline__ df64 shx(df64 v, int m) {
  return df64::make(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}
#endif

// Number of martensite variants N, fixed at compile time: 6 for the CuAlNi
// data of Sec. 5.1 (the default build), 12 for a NiTi-type monoclinic set
// (15 unknowns per node, the footnote of Sec. 5.4); the library is built once
// per value (libpfm.so, libpfm_nv12.so).
#ifndef PFM_NV
#define PFM_NV 6
#endif
constexpr int NV = PFM_NV;
constexpr int NPH = NV + 1;           // phases: austenite + N variants
constexpr int NZ = 9 + NV;            // local unknowns at a point: F (9) + eta_hat (N)
constexpr int NH = NZ * (NZ + 1) / 2; // packed upper triangle of the NZ x NZ Hessian (120 for N = 6)
// entries stored per Gauss point: NH rounded up to a multiple of 8, so that
// 16-byte vectors of binary16, FP32 or FP64 entries tile it (120 and 232)
constexpr int NHP = (NH + 7) / 8 * 8;

// Physical parameters, passed by value to kernels (constant bank).
struct DevParams {
  double U[NPH][3][3];      // transformation stretches U_i (U_0 = I)
  double Lv[NPH][6][6];     // stiffness L_i in Voigt form (engineering shear)
  double F0[NPH];           // chemical energies F_i^0
  double inv_mtau[NPH];     // 1 / (m_i tau)
  double cobst[NPH][NPH];   // 4 gamma_ij / (pi ell_ij), zero diagonal
  double G[NV][NV];         // gradient-energy matrix in eta_hat (per direction)
  double eps_eta;           // penalty parameter
  int same_L;               // 1 when every phase has the same stiffness (then L(eta) = L sum eta)
  int cubic;                // 1 when that stiffness is cubic in the frame of the data:
  double cub_lambda, cub_mu, cub_delta;  // L = lambda I x I + 2 mu I_sym + delta sum_n e_n^4
  int hencky;               // 0: exact log; m = 1, 2, 3: Pade (m,m) (Gauss-Legendre form below)
  double pade_s[3], pade_w[3];  // m-point Gauss-Legendre nodes and weights on [0, 1]
};

// Packed index of (r, c), r <= c, in the row-major upper triangle.
PFM_HD int hidx(int r, int c) { return r * NZ - (r * (r - 1)) / 2 + (c - r); }

template <typename T> struct Tol;
template <> struct Tol<double> {
  static constexpr double dd2_gap = 1e-3;    // relative spread below which f2 uses its Taylor series
  static constexpr double jacobi_off = 1e-17;
};
#ifdef __CUDACC__
template <> struct Tol<df64> {
  static constexpr double dd2_gap = 1e-3;
  static constexpr double jacobi_off = 1e-14;  // the double-float resolution
};
#endif
template <> struct Tol<float> {
  static constexpr float dd2_gap = 3e-2f;
  static constexpr float jacobi_off = 1e-8f;
};

template <typename T> PFM_HD T tmin(T a, T b) { return a < b ? a : b; }

// ---------------------------------------------------------------------------
// 3x3 helpers (full storage)

template <typename T>
PFM_HD void mm3(const T a[3][3], const T b[3][3], T c[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) c[i][k] = a[i][0] * b[0][k] + a[i][1] * b[1][k] + a[i][2] * b[2][k];
}

// c = a^T b
template <typename T>
PFM_HD void mtm3(const T a[3][3], const T b[3][3], T c[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) c[i][k] = a[0][i] * b[0][k] + a[1][i] * b[1][k] + a[2][i] * b[2][k];
}

// c = Q^T a Q (rotate a symmetric matrix into the basis of Q's columns)
template <typename T>
PFM_HD void rot_in(const T Q[3][3], const T a[3][3], T c[3][3]) {
  T t[3][3];
  mm3(a, Q, t);
  mtm3(Q, t, c);
}

template <typename T>
PFM_HD T tr_ab(const T a[3][3], const T b[3][3]) {  // tr(a b)
  T s = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) s += a[i][j] * b[j][i];
  return s;
}

template <typename T>
PFM_HD T ddot3(const T a[3][3], const T b[3][3]) {  // a : b
  T s = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) s += a[i][j] * b[i][j];
  return s;
}

// Inverse and determinant of a symmetric positive-definite 3x3 matrix.
template <typename T>
PFM_HD T inv_sym3(const T a[3][3], T r[3][3]) {
  T c00 = a[1][1] * a[2][2] - a[1][2] * a[2][1];
  T c01 = a[1][2] * a[2][0] - a[1][0] * a[2][2];
  T c02 = a[1][0] * a[2][1] - a[1][1] * a[2][0];
  T det = a[0][0] * c00 + a[0][1] * c01 + a[0][2] * c02;
  T id = T(1) / det;
  r[0][0] = c00 * id;
  r[0][1] = r[1][0] = c01 * id;
  r[0][2] = r[2][0] = c02 * id;
  r[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) * id;
  r[1][2] = r[2][1] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) * id;
  r[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) * id;
  return det;
}

// Voigt vector with engineering shear: (a00, a11, a22, 2a12, 2a02, 2a01).
template <typename T>
PFM_HD void voigt_strain(const T a[3][3], T v[6]) {
  v[0] = a[0][0]; v[1] = a[1][1]; v[2] = a[2][2];
  v[3] = a[1][2] + a[2][1]; v[4] = a[0][2] + a[2][0]; v[5] = a[0][1] + a[1][0];
}
// Symmetric tensor from a Voigt stress vector (no shear factor).
template <typename T>
PFM_HD void from_voigt_stress(const T v[6], T a[3][3]) {
  a[0][0] = v[0]; a[1][1] = v[1]; a[2][2] = v[2];
  a[1][2] = a[2][1] = v[3]; a[0][2] = a[2][0] = v[4]; a[0][1] = a[1][0] = v[5];
}


// Packed symmetric 3x3 storage (00, 11, 22, 12, 02, 01), the Voigt order.
PFM_HD int sym_i(int v) { return v < 3 ? v : (v == 3 ? 1 : 0); }
PFM_HD int sym_j(int v) { return v < 3 ? v : (v == 5 ? 1 : 2); }
template <typename T>
PFM_HD T symget(const T* X, int a, int b) {
  if (a == b) return X[a];
  const int s = a + b;  // (1,2) -> 3, (0,2) -> 2, (0,1) -> 1
  return X[s == 3 ? 3 : (s == 2 ? 4 : 5)];
}
// Voigt slot (00, 11, 22, 12, 02, 01) of the symmetric pair (a, c).
PFM_HD int voigt_slot(int a, int c) { return a == c ? a : 6 - a - c; }

template <typename T>
PFM_HD void load_U(const DevParams& P, int p, T U[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) U[i][j] = T(P.U[p][i][j]);
}

// ---------------------------------------------------------------------------
// Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations:
// a = Q diag(lam) Q^T, Q orthonormal (columns are eigenvectors).

template <typename T>
PFM_HD void jacobi_eig3(T a[3][3], T lam[3], T Q[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Q[i][j] = (i == j) ? T(1) : T(0);
  for (int sweep = 0; sweep < 16; ++sweep) {
    T off = fabs(a[0][1]) + fabs(a[0][2]) + fabs(a[1][2]);
    T dia = fabs(a[0][0]) + fabs(a[1][1]) + fabs(a[2][2]);
    if (off <= Tol<T>::jacobi_off * dia) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = (pq == 2) ? 1 : 0;
      const int q = (pq == 0) ? 1 : 2;
      const int r = 3 - p - q;
      T apq = a[p][q];
      if (fabs(apq) <= Tol<T>::jacobi_off * (fabs(a[p][p]) + fabs(a[q][q]))) {
        a[p][q] = a[q][p] = T(0);
        continue;
      }
      // rotation angle phi with cot(2 phi) = theta zeroes a_pq; t = tan(phi)
      T theta = (a[q][q] - a[p][p]) / (T(2) * apq);
      T t = T(1) / (fabs(theta) + sqrt(theta * theta + T(1)));
      if (theta < T(0)) t = -t;
      T c = T(1) / sqrt(t * t + T(1));
      T s = t * c;
      T tau = s / (T(1) + c);
      a[p][p] -= t * apq;
      a[q][q] += t * apq;
      a[p][q] = a[q][p] = T(0);
      T arp = a[r][p], arq = a[r][q];
      a[r][p] = a[p][r] = arp - s * (arq + tau * arp);
      a[r][q] = a[q][r] = arq + s * (arp - tau * arq);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        T qkp = Q[k][p], qkq = Q[k][q];
        Q[k][p] = qkp - s * (qkq + tau * qkp);
        Q[k][q] = qkq + s * (qkp - tau * qkq);
      }
    }
  }
  lam[0] = a[0][0]; lam[1] = a[1][1]; lam[2] = a[2][2];
}


// Eigen-decomposition used by the point physics: in FP32 directly; in FP64
// the Jacobi rotations are first run in FP32 (cheap square roots and
// divisions), the matrix is rotated into that approximate eigenbasis in FP64
// and FP64 Jacobi sweeps finish it (quadratic convergence from ~1e-7).
template <typename T>
PFM_HD void eig_sym3(T a[3][3], T lam[3], T Q[3][3]) {
  jacobi_eig3(a, lam, Q);
}
template <>
PFM_HD void eig_sym3<double>(double a[3][3], double lam[3], double Q[3][3]) {
  float af[3][3], lf[3], Qf[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) af[i][j] = float(a[i][j]);
  jacobi_eig3(af, lf, Qf);
  double Q0[3][3], b[3][3], Q1[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Q0[i][j] = double(Qf[i][j]);
  // re-orthonormalise the FP32 eigenvectors in FP64 (modified Gram-Schmidt)
  for (int c = 0; c < 3; ++c) {
    for (int pc = 0; pc < c; ++pc) {
      double d = Q0[0][c] * Q0[0][pc] + Q0[1][c] * Q0[1][pc] + Q0[2][c] * Q0[2][pc];
      for (int i = 0; i < 3; ++i) Q0[i][c] -= d * Q0[i][pc];
    }
    double nrm = sqrt(Q0[0][c] * Q0[0][c] + Q0[1][c] * Q0[1][c] + Q0[2][c] * Q0[2][c]);
    const double inrm = 1.0 / nrm;
    for (int i = 0; i < 3; ++i) Q0[i][c] *= inrm;
  }
  rot_in(Q0, a, b);
  jacobi_eig3(b, lam, Q1);
  mm3(Q0, Q1, Q);
}

#ifdef __CUDACC__
// Double-float version of the FP64 eigen-decomposition: FP32 Jacobi seed,
// re-orthonormalisation and the finishing sweeps in double-float.
__device__ __forceinline__ void eig_sym3(df64 a[3][3], df64 lam[3], df64 Q[3][3]) {
  float af[3][3], lf[3], Qf[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) af[i][j] = a[i][j].hi;
  jacobi_eig3(af, lf, Qf);
  df64 Q0[3][3], b[3][3], Q1[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Q0[i][j] = df64(double(Qf[i][j]));
  for (int c = 0; c < 3; ++c) {
    for (int pc = 0; pc < c; ++pc) {
      df64 d = Q0[0][c] * Q0[0][pc] + Q0[1][c] * Q0[1][pc] + Q0[2][c] * Q0[2][pc];
      for (int i = 0; i < 3; ++i) Q0[i][c] -= d * Q0[i][pc];
    }
    df64 inrm = df64(1.0 / ::sqrt(double(Q0[0][c] * Q0[0][c] + Q0[1][c] * Q0[1][c] + Q0[2][c] * Q0[2][c])));
    for (int i = 0; i < 3; ++i) Q0[i][c] *= inrm;
  }
  rot_in(Q0, a, b);
  jacobi_eig3(b, lam, Q1);
  mm3(Q0, Q1, Q);
}
#endif

// First divided difference of log: (log a - log b)/(a - b), 1/a if a == b.
template <typename T>
PFM_HD T dd1_log(T a, T b) {
  if (a < b) { T t = a; a = b; b = t; }
  T d = a - b;
  if (d == T(0)) return T(1) / a;
  return log1p(d / b) / d;
}

// Second divided difference of log, symmetric in its arguments.
template <typename T>
PFM_HD T dd2_log(T x0, T x1, T x2) {
  // sort descending: a >= b >= c
  T a = x0, b = x1, c = x2, t;
  if (a < b) { t = a; a = b; b = t; }
  if (b < c) { t = b; b = c; c = t; }
  if (a < b) { t = a; a = b; b = t; }
  T gap = a - c;
  if (gap > Tol<T>::dd2_gap * a) return (dd1_log(a, b) - dd1_log(b, c)) / gap;
  // f[x0,x1,x2] = sum_j f^(2+j)(m)/(2+j)! h_j(x - m); for log this is
  // (1/m^2) sum_j (-1)^(j+1) h_j(u)/(j+2), u = (x - m)/m, h_j the complete
  // homogeneous symmetric polynomial of degree j, built one variable at a
  // time: h_j(u_0..u_i) = h_j(u_0..u_(i-1)) + u_i h_(j-1)(u_0..u_i).
  const T m = (a + b + c) / T(3);
  const T im = T(1) / m;
  const T u[3] = {(a - m) * im, (b - m) * im, (c - m) * im};
  T hh[6] = {T(1), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 1; j < 6; ++j) hh[j] = (i == 0 ? T(0) : hh[j]) + u[i] * hh[j - 1];
  // alternating weights -1/2, 1/3, -1/4, 1/5, -1/6, 1/7
  const T wj[6] = {T(-0.5), T(1.0 / 3.0), T(-0.25), T(0.2), T(-1.0 / 6.0), T(1.0 / 7.0)};
  T sum = T(0);
#pragma unroll
  for (int j = 0; j < 6; ++j) sum += wj[j] * hh[j];
  return sum * im * im;
}

// Second divided difference of log at (x, y, z) from the first ones
// fxy = f[x,y], fyz = f[y,z], fxz = f[x,z]. On a wide spread it is the
// quotient over the largest gap with the middle value as pivot, which is the
// quotient dd2_log forms after sorting (the same operands up to signs, so the
// same result); on a narrow spread, dd2_log's series.
template <typename T>
PFM_HD T dd2_log_f1(T x, T y, T z, T fxy, T fyz, T fxz) {
  const T dxz = x - z, dxy = x - y, dyz = y - z;
  const T axz = fabs(dxz), axy = fabs(dxy), ayz = fabs(dyz);
  T num, den, gap;
  if (axz >= axy && axz >= ayz) {  // y in the middle
    num = fxy - fyz;
    den = dxz;
    gap = axz;
  } else if (axy >= ayz) {  // z in the middle
    num = fxz - fyz;
    den = dxy;
    gap = axy;
  } else {  // x in the middle
    num = fxy - fxz;
    den = dyz;
    gap = ayz;
  }
  const T top = x > y ? (x > z ? x : z) : (y > z ? y : z);
  if (gap > Tol<T>::dd2_gap * top) return num / den;
  return dd2_log(x, y, z);
}

// ---------------------------------------------------------------------------
// Local energy density with gradient and (optionally) packed Hessian.
//
// Fin: F row-major; eh, ehn: eta_1..eta_6 at t_{n+1} and t_n.
// Outputs: *W, g[15] = dW/dz, Hp[120] = packed d^2W/dz^2 (if Hp != nullptr).
template <typename T, bool WANT_HESS>
PFM_HD_BIG void qp_local(const DevParams& P, const T Fin[9], const T eh[NV], const T ehn[NV], T* W,
                     T g[NZ], T* Hp) {
  T eta[NPH], etan[NPH];
  {
    T s = 0, sn = 0;
#pragma unroll
    for (int k = 0; k < NV; ++k) { eta[k + 1] = eh[k]; etan[k + 1] = ehn[k]; s += eh[k]; sn += ehn[k]; }
    eta[0] = T(1) - s;
    etan[0] = T(1) - sn;
  }
  // sum of the eta_i as the same floating-point sum the per-phase loops form
  T esum = T(0);
#pragma unroll
  for (int p = 0; p < NPH; ++p) esum += eta[p];
  T F[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) F[i][j] = Fin[3 * i + j];

  // transformation stretch, its inverse and determinant
  T Ft[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
  for (int p = 0; p < NPH; ++p)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Ft[i][j] += eta[p] * T(P.U[p][i][j]);
  T A[3][3];
  const T Jt = inv_sym3(Ft, A);
  T M[3][3];  // F^e = F A
  mm3(F, A, M);
  T E[3][3];  // C^e = M^T M
  mtm3(M, M, E);

  // spectral decomposition of C^e and the Hencky strain h = 1/2 log C^e
  T lam[3], Q[3][3];
  {
    T tmp[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) tmp[i][j] = E[i][j];
    eig_sym3(tmp, lam, Q);
  }
  // f = log (exact mode) or the Pade approximant r_m, at the eigenvalues, and
  // its first divided differences
  T loglam[3];
  T f1[3][3];
  T rp[3][3];  // Pade modes: rp[k][a] = 1 / p_k(lam_a)
  const int npade = P.hencky;
  if (npade == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) loglam[a] = log(lam[a]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = a; b < 3; ++b) f1[a][b] = f1[b][a] = (a == b) ? T(1) / lam[a] : dd1_log(lam[a], lam[b]);
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      loglam[a] = T(0);
#pragma unroll
      for (int b = 0; b < 3; ++b) f1[a][b] = T(0);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (k < npade) {
        const T sk = T(P.pade_s[k]), wk = T(P.pade_w[k]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          rp[k][a] = T(1) / (T(1) + sk * (lam[a] - T(1)));
          loglam[a] += wk * (lam[a] - T(1)) * rp[k][a];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) f1[a][b] += wk * rp[k][a] * rp[k][b];
      }
    }
  }
  T h[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      h[i][j] = T(0.5) * (Q[i][0] * loglam[0] * Q[j][0] + Q[i][1] * loglam[1] * Q[j][1] +
                          Q[i][2] * loglam[2] * Q[j][2]);

  // stress-like T = L(eta) : h and the per-phase L_i : h
  T hv[6];
  voigt_strain(h, hv);
  T Tv[6] = {0, 0, 0, 0, 0, 0};
  T hLh[NPH];  // h : L_i : h
  if (P.same_L) {
    T s = 0;
#pragma unroll
    for (int I = 0; I < 6; ++I) {
      T li = 0;
#pragma unroll
      for (int J = 0; J < 6; ++J) li += T(P.Lv[0][I][J]) * hv[J];
      Tv[I] = esum * li;
      s += hv[I] * li;
    }
#pragma unroll
    for (int p = 0; p < NPH; ++p) hLh[p] = s;
  } else {
#pragma unroll
    for (int p = 0; p < NPH; ++p) {
      T s = 0;
#pragma unroll
      for (int I = 0; I < 6; ++I) {
        T li = 0;
#pragma unroll
        for (int J = 0; J < 6; ++J) li += T(P.Lv[p][I][J]) * hv[J];
        Tv[I] += eta[p] * li;
        s += hv[I] * li;
      }
      hLh[p] = s;
    }
  }
  T hT = 0;
#pragma unroll
  for (int I = 0; I < 6; ++I) hT += hv[I] * Tv[I];
  T Tm[3][3];
  from_voigt_stress(Tv, Tm);

  // S = dW_el/dE = J_t Dh[T] = 1/2 J_t Dlog[T]; in the eigenbasis S~ = 1/2 J_t f1 o T~
  T Tt[3][3];
  rot_in(Q, Tm, Tt);
  T St[3][3], S[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) St[a][b] = T(0.5) * Jt * f1[a][b] * Tt[a][b];
  {
    T t[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int b = 0; b < 3; ++b) t[i][b] = Q[i][0] * St[0][b] + Q[i][1] * St[1][b] + Q[i][2] * St[2][b];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) S[i][j] = t[i][0] * Q[j][0] + t[i][1] * Q[j][1] + t[i][2] * Q[j][2];
  }

  // energy
  T Wloc = T(0.5) * Jt * hT;
  // With eta_0 = 1 - sum eta_hat (Sec. 3.1) the elastic energy depends on
  // eta_hat_k through U(eta) = sum eta_i U_i and L(eta) = sum eta_i L_i, i.e.
  // along dU_k = U_k - U_0 and dL_k = L_k - L_0.
  // dU_k is symmetric (a difference of stretches), so tr(X dU_k) = <X^T, dU_k>.
  T trAdU[NV];  // tr(A dU_k) = (d J_t / d eta_hat_k) / J_t
  T gel[NV];    // dW_el / d eta_hat_k
  {
    T ES[3][3], ESA[3][3];  // E S, E S A
    mm3(E, S, ES);
    mm3(ES, A, ESA);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      T ta = 0, te = 0;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const T d = T(P.U[k + 1][i][j]) - T(P.U[0][i][j]);
          ta += A[i][j] * d;
          te += ESA[j][i] * d;
        }
      trAdU[k] = ta;
      // S : dE/d eta_hat_k = -2 tr(S A dU_k E) = -2 tr(E S A dU_k)
      gel[k] = T(0.5) * Jt * trAdU[k] * hT + T(0.5) * Jt * (hLh[k + 1] - hLh[0]) + T(-2) * te;
    }
  }
  // chemical, obstacle, dissipation, penalty: dW/d eta_i per phase
  T geta[NPH];
#pragma unroll
  for (int i = 0; i < NPH; ++i) {
    T d = eta[i] - etan[i];
    T neg = eta[i] < T(0) ? eta[i] : T(0);
    Wloc += eta[i] * T(P.F0[i]) + T(0.5) * T(P.inv_mtau[i]) * d * d + T(0.5) * T(P.eps_eta) * neg * neg;
    T go = 0;
#pragma unroll
    for (int j = 0; j < NPH; ++j) {
      if (j > i) Wloc += T(P.cobst[i][j]) * eta[i] * eta[j];
      go += T(P.cobst[i][j]) * eta[j];
    }
    geta[i] = T(P.F0[i]) + go + T(P.inv_mtau[i]) * d + T(P.eps_eta) * neg;
  }
  *W = Wloc;

  // gradient: P_el = 2 M S A, then eta_hat_k = eta_k - eta_0 (Sec. 3.1)
  {
    T MS[3][3], Pm[3][3];
    mm3(M, S, MS);
    mm3(MS, A, Pm);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) g[3 * i + j] = T(2) * Pm[i][j];
#pragma unroll
    for (int k = 0; k < NV; ++k) g[9 + k] = gel[k] + (geta[k + 1] - geta[0]);
  }
  if (!WANT_HESS) return;
  // the direction eta_hat_k carries dU_k = U_k - U_0; A dU_k enters below
  T dU[NV][3][3], AdU[NV][3][3];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) dU[k][i][j] = T(P.U[k + 1][i][j]) - T(P.U[0][i][j]);
    mm3(A, dU[k], AdU[k]);
  }

  // ---------------------------------------------------------------------
  // Hessian in the 9 + N unknowns z = (F_pQ: 0..8, eta_hat_1..N: 9..8+N), packed
  // into Hp[hidx(r, c)], r <= c. With eta_0 = 1 - sum eta_hat (Sec. 3.1) every
  // eta-dependence enters through U(eta) = sum eta_i U_i and L(eta) =
  // sum eta_i L_i, so the direction eta_hat_k carries dU_k = U_k - U_0 and
  // dL_k = L_k - L_0 (dU_k, A dU_k and tr(A dU_k) from above) and the
  // elimination of eta_0 holds term by term.
  constexpr int ND = NZ;
  // Rotated directions X~_k = Q^T dE_k Q, symmetric, stored as 6 values
  // (00, 11, 22, 12, 02, 01).
  T Xs[ND][6];
  {
    T Aq[3][3], Mq[3][3];  // Aq[c] = Q^T (column c of A), Mq[p] = Q^T (row p of M)
    for (int c = 0; c < 3; ++c)
      for (int a = 0; a < 3; ++a) {
        Aq[c][a] = Q[0][a] * A[0][c] + Q[1][a] * A[1][c] + Q[2][a] * A[2][c];
        Mq[c][a] = Q[0][a] * M[c][0] + Q[1][a] * M[c][1] + Q[2][a] * M[c][2];
      }
    for (int p = 0; p < 3; ++p)
      for (int c = 0; c < 3; ++c) {
        T* X = Xs[3 * p + c];
        for (int v = 0; v < 6; ++v) {
          const int a = sym_i(v), b = sym_j(v);
          X[v] = Aq[c][a] * Mq[p][b] + Mq[p][a] * Aq[c][b];
        }
      }
  }
  for (int k = 0; k < NV; ++k) {
    T B[3][3];
    rot_in(Q, AdU[k], B);  // B = Q^T A dU_k Q ; dE~ = -(B Lambda + Lambda B^T)
    for (int v = 0; v < 6; ++v) {
      const int a = sym_i(v), b = sym_j(v);
      Xs[9 + k][v] = -(B[a][b] * lam[b] + lam[a] * B[b][a]);
    }
  }
  // d~_k = Dh~[X~_k] = 1/2 f1 o X~_k as Voigt strain vectors (engineering
  // shear): d~_k[v] = c[v] X~_k[v]
  T cv[6];
  for (int v = 0; v < 6; ++v) cv[v] = T(0.5) * f1[sym_i(v)][sym_j(v)] * (v < 3 ? T(1) : T(2));
  // L~ = Nv^T L(eta) Nv with v(Q d~ Q^T) = Nv v(d~)
  T Lt[6][6];
  if (P.cubic) {
    // cubic stiffness: the isotropic part lambda I x I + 2 mu I_sym is the
    // same in every basis, and the cubic part delta sum_n e_n^4 turns into
    // delta sum_n w_n w_n^T with w_n[A] = r_a r_b for the slot A = (a, b) and
    // r = row n of Q (e_n in the eigenbasis); all scaled by sum eta
    const T lam_c = T(P.cub_lambda) * esum, mu_c = T(P.cub_mu) * esum, del_c = T(P.cub_delta) * esum;
    T w[3][6];
#pragma unroll
    for (int n = 0; n < 3; ++n)
#pragma unroll
      for (int A_ = 0; A_ < 6; ++A_) w[n][A_] = Q[n][sym_i(A_)] * Q[n][sym_j(A_)];
#pragma unroll
    for (int A_ = 0; A_ < 6; ++A_)
#pragma unroll
      for (int B = A_; B < 6; ++B) {
        T v = del_c * (w[0][A_] * w[0][B] + w[1][A_] * w[1][B] + w[2][A_] * w[2][B]);
        if (A_ < 3 && B < 3) v += lam_c;
        if (A_ == B) v += A_ < 3 ? T(2) * mu_c : mu_c;
        Lt[A_][B] = Lt[B][A_] = v;
      }
  } else {
    T Nv[6][6];
    for (int I = 0; I < 6; ++I) {
      const int i = sym_i(I), j = sym_j(I);
      const T cI = (I < 3) ? T(1) : T(2);
      for (int B = 0; B < 6; ++B) {
        const int a = sym_i(B), b = sym_j(B);
        Nv[I][B] = (B < 3) ? cI * Q[i][a] * Q[j][a] : cI * T(0.5) * (Q[i][a] * Q[j][b] + Q[i][b] * Q[j][a]);
      }
    }
    T Le[6][6];  // L(eta) = sum_p eta_p L_p
    for (int I = 0; I < 6; ++I)
      for (int J = 0; J < 6; ++J) {
        T lij = 0;
        if (P.same_L) {
          lij = T(P.Lv[0][I][J]) * esum;
        } else {
          for (int p = 0; p < NPH; ++p) lij += eta[p] * T(P.Lv[p][I][J]);
        }
        Le[I][J] = lij;
      }
    T LN[6][6];
    for (int I = 0; I < 6; ++I)
      for (int B = 0; B < 6; ++B) {
        T s = 0;
        for (int J = 0; J < 6; ++J) s += Le[I][J] * Nv[J][B];
        LN[I][B] = s;
      }
    for (int A_ = 0; A_ < 6; ++A_)
      for (int B = 0; B < 6; ++B) {
        T s = 0;
        for (int I = 0; I < 6; ++I) s += Nv[I][A_] * LN[I][B];
        Lt[A_][B] = s;
      }
  }
  // The second-order part of the elastic energy along directions k, l,
  // J_t (d~_k . L~ d~_l + K(k,l)) with K(k,l) = sum_abc f2_abc T~_ab X~_k[a][c]
  // X~_l[b][c] (f2: second divided differences, symmetric), is one symmetric
  // bilinear form in the 6 stored entries of X~: X~_k^T Mb X~_l with
  // Mb[v][w] = J_t (c[v] L~[v][w] c[w] + sum of f2_abc T~_ab over the (a, b, c)
  // whose pairs (a, c) and (b, c) have the Voigt slots v and w).
  T f2[3][3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b)
      for (int c = b; c < 3; ++c) {
        T v;
        if (npade == 0) {
          // one eigenvalue: f'' / 2 = -1 / (2 lam^2)
          v = (a == c) ? T(-0.5) * f1[a][a] * f1[a][a]
                       : dd2_log_f1(lam[a], lam[b], lam[c], f1[a][b], f1[b][c], f1[a][c]);
        } else {
          v = T(0);
          for (int k = 0; k < 3; ++k)
            if (k < npade) v -= T(P.pade_w[k]) * T(P.pade_s[k]) * rp[k][a] * rp[k][b] * rp[k][c];
        }
        f2[a][b][c] = f2[a][c][b] = f2[b][a][c] = f2[b][c][a] = f2[c][a][b] = f2[c][b][a] = v;
      }
  T Mb[6][6];
  for (int I = 0; I < 6; ++I)
    for (int J = 0; J < 6; ++J) Mb[I][J] = cv[I] * Lt[I][J] * cv[J];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) Mb[voigt_slot(a, c)][voigt_slot(b, c)] += f2[a][b][c] * Tt[a][b];
  for (int I = 0; I < 6; ++I)
    for (int J = 0; J < 6; ++J) Mb[I][J] *= Jt;
  // (dL_k h) rotated and scaled by c, so that (dL_k h)~ : d~_l = LhT[k] . X~_l;
  // zero when every phase has the same stiffness
  T LhT[NV][6];
  if (!P.same_L) {
    for (int k = 0; k < NV; ++k) {
      T lv[6], lm[3][3], lr[3][3];
      for (int I = 0; I < 6; ++I) {
        T s = 0;
        for (int J = 0; J < 6; ++J) s += (T(P.Lv[k + 1][I][J]) - T(P.Lv[0][I][J])) * hv[J];
        lv[I] = s;
      }
      from_voigt_stress(lv, lm);
      rot_in(Q, lm, lr);
      for (int v = 0; v < 6; ++v) LhT[k][v] = cv[v] * lr[sym_i(v)][sym_j(v)];
    }
  }
  // second-order part X~_k^T Mb X~_l, and the first-order terms
  // g_{E eta_p}[X_k] = tr(A dU_p) S~:X~_k + J_t (dL_p h)~ : d~_k, added to the
  // F-eta and eta-eta entries (the latter for both index orders).
  for (int k = 0; k < ND; ++k) {
    T Y[6];
    for (int I = 0; I < 6; ++I) {
      T s = 0;
      for (int J = 0; J < 6; ++J) s += Mb[I][J] * Xs[k][J];
      Y[I] = s;
    }
    for (int l = k; l < ND; ++l) {
      T acc = 0;
      for (int I = 0; I < 6; ++I) acc += Xs[l][I] * Y[I];
      Hp[hidx(k, l)] = acc;
    }
    // S~ : X~_k (tensor double contraction of symmetric matrices)
    T SX = 0;
    for (int v = 0; v < 6; ++v) SX += (v < 3 ? T(1) : T(2)) * St[sym_i(v)][sym_j(v)] * Xs[k][v];
    for (int p = 0; p < NV; ++p) {
      T ge = trAdU[p] * SX;
      if (!P.same_L) {
        T d = 0;
        for (int v = 0; v < 6; ++v) d += LhT[p][v] * Xs[k][v];
        ge += Jt * d;
      }
      if (k < 9) {
        Hp[hidx(k, 9 + p)] += ge;
      } else {
        const int q = k - 9;
        const int lo = p < q ? p : q, hi = p < q ? q : p;
        Hp[hidx(9 + lo, 9 + hi)] += (p == q) ? T(2) * ge : ge;
      }
    }
  }
  // S : d^2E, F-F block: delta_pr 2 (A S A)_QS
  T ASA[3][3];
  {
    T t[3][3];
    mm3(S, A, t);
    mm3(A, t, ASA);
  }
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q)
      for (int s2 = q; s2 < 3; ++s2) Hp[hidx(3 * p + q, 3 * p + s2)] += T(2) * ASA[q][s2];
  // per direction: Y_k = A dU_k A, S Y_k, C Y_k, S E dU_k
  T C[3][3], SE[3][3];
  mtm3(F, F, C);
  mm3(S, E, SE);
  T Yk[NV][3][3], SY[NV][3][3], CY[NV][3][3], SEU[NV][3][3];
  for (int k = 0; k < NV; ++k) {
    mm3(AdU[k], A, Yk[k]);
    mm3(S, Yk[k], SY[k]);
    mm3(C, Yk[k], CY[k]);
    mm3(SE, dU[k], SEU[k]);
  }
  // F-eta block: -2 (F N_k)_rQ with N_k = ASA dU_k A + A dU_k ASA, where
  // F ASA dU_k A = M (S Y_k) and F A dU_k ASA = (M dU_k) ASA
  for (int k = 0; k < NV; ++k) {
    T MdU[3][3], t1[3][3], t2[3][3];
    mm3(M, SY[k], t1);
    mm3(M, dU[k], MdU);
    mm3(MdU, ASA, t2);
    for (int r = 0; r < 9; ++r) Hp[hidx(r, 9 + k)] += T(-2) * (t1[r / 3][r % 3] + t2[r / 3][r % 3]);
  }
  // eta-eta block: S:d2E + explicit eta derivatives of g + local terms
  // (obstacle, dissipation, penalty), the last written in eta_hat:
  // c_kl - c_k0 - c_0l + c_00 + d_0 + delta_kl d_k, d_i = 1/(m_i tau) + eps [eta_i < 0]
  const T d0 = T(P.inv_mtau[0]) + (eta[0] < T(0) ? T(P.eps_eta) : T(0));
  for (int p = 0; p < NV; ++p) {
    const T hLp = hLh[p + 1] - hLh[0];
    for (int q = p; q < NV; ++q) {
      const T hLq = hLh[q + 1] - hLh[0];
      T sd2E = T(2) * (tr_ab(SEU[p], Yk[q]) + tr_ab(SEU[q], Yk[p]) + tr_ab(SY[p], CY[q]));
      T Jpq = Jt * (trAdU[p] * trAdU[q] - tr_ab(AdU[p], AdU[q]));
      T gee = T(0.5) * Jpq * hT + T(0.5) * Jt * trAdU[p] * hLq + T(0.5) * Jt * trAdU[q] * hLp;
      T loc = T(P.cobst[p + 1][q + 1]) - T(P.cobst[p + 1][0]) - T(P.cobst[0][q + 1]) + T(P.cobst[0][0]) + d0;
      if (p == q) loc += T(P.inv_mtau[p + 1]) + (eta[p + 1] < T(0) ? T(P.eps_eta) : T(0));
      Hp[hidx(9 + p, 9 + q)] += sd2E + gee + loc;
    }
  }
}

}  // namespace pfm
