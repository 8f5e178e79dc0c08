// Internal declarations shared by the CUDA translation units of libpfm.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <limits>

#include "qp_physics.cuh"

namespace pfm {

constexpr int NF = 3 + NV;          // unknowns per node: u (3) + eta_hat (N): 9 for N = 6
constexpr int NBD = NF * (NF + 1) / 2;  // packed upper triangle of a nodal NF x NF block (45)
constexpr int NF2 = NF * NF;            // entries of a nodal block (81)
constexpr int NED = 8 * NF;             // unknowns of one element (72)

// Gauss points of the 2-point rule mapped to [0,1]: (1 -+ 1/sqrt(3)) / 2.
constexpr double GA = 0.21132486540518711775;
constexpr double GB = 0.78867513459481288225;

// Structured grid of one multigrid level.
struct Grid {
  int nx, ny, nz;
  double hx, hy, hz;
  __host__ __device__ int64_t nn() const { return int64_t(nx + 1) * (ny + 1) * (nz + 1); }
  __host__ __device__ int64_t ne() const { return int64_t(nx) * ny * nz; }
  // element blocks of 4 elements (one warp: 4 elements x 8 Gauss points)
  __host__ __device__ int64_t nblk() const { return (ne() + 3) / 4; }
  __host__ __device__ double w() const { return hx * hy * hz / 8.0; }
};

// Gauss-point Hessian store: element blocks of 4, lane = 8*(e%4) + q, and per
// lane the NH packed entries (120 for N = 6), padded with zeros to NHP, in
// 16-byte vectors of V = 16/sizeof(S) entries:
// offset ((blk*(NHP/V) + entry/V)*32 + lane)*V + entry%V. One warp therefore
// reads 512 contiguous bytes per vector load.
template <typename S>
__host__ __device__ inline int64_t hstore_offset(int64_t blk, int entry, int lane) {
  constexpr int V = 16 / sizeof(S);
  return ((blk * (NHP / V) + entry / V) * 32 + lane) * V + entry % V;
}
constexpr int64_t HBLK = int64_t(NHP) * 32;  // entries per element block

// Unsigned 32-bit division by a divisor fixed at launch, as a multiply-high
// and a shift (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, the round-up variant): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (umulhi(n, m) + n) >> l for every
// n < 2^31 (the sum stays below 2^32).
struct FastDiv {
  uint32_t d = 1, m = 1, l = 0;
  static FastDiv make(uint32_t d) {
    FastDiv f;
    f.d = d;
    f.l = 0;
    while ((uint64_t(1) << f.l) < d) ++f.l;
    f.m = uint32_t(((uint64_t(1) << 32) * ((uint64_t(1) << f.l) - d)) / d + 1);
    return f;
  }
  __host__ __device__ uint32_t div(uint32_t n) const {
#ifdef __CUDA_ARCH__
    const uint32_t t = __umulhi(n, m);
#else
    const uint32_t t = uint32_t((uint64_t(n) * m) >> 32);
#endif
    return (t + n) >> l;
  }
};

// Largest eigenvalue of the symmetric tridiagonal matrix T of a Lanczos run
// (host code): diagonal alpha[0..m), squared off-diagonal beta2[0..m-1).
// The run is cut at the first alpha that is not finite, or the first beta2
// that is not positive and finite (an invariant subspace was reached; T is
// then exact). Bisection on the Sturm count of T - x I (the number of negative
// pivots of its LDL^T factorisation equals the number of eigenvalues below x;
// Wilkinson, The Algebraic Eigenvalue Problem, 1965, Ch. 5) inside the
// Gershgorin interval. Returns NaN if no step is usable.
inline double tridiag_max_eig(const double* alpha, const double* beta2, int m) {
  int k = 0;
  while (k < m && alpha[k] == alpha[k] && alpha[k] - alpha[k] == 0.0) {
    ++k;
    if (k < m && !(beta2[k - 1] > 0.0 && beta2[k - 1] - beta2[k - 1] == 0.0)) break;
  }
  m = k;
  if (m == 0) return std::numeric_limits<double>::quiet_NaN();
  auto offd = [&](int i) { return (i >= 0 && i < m - 1) ? std::sqrt(beta2[i]) : 0.0; };
  double lo = alpha[0], hi = alpha[0];
  for (int i = 0; i < m; ++i) {
    const double r = offd(i - 1) + offd(i);
    lo = alpha[i] - r < lo ? alpha[i] - r : lo;
    hi = alpha[i] + r > hi ? alpha[i] + r : hi;
  }
  auto below = [&](double x) {  // eigenvalues of T below x
    int c = 0;
    double d = 1.0;
    for (int i = 0; i < m; ++i) {
      d = alpha[i] - x - (i > 0 ? beta2[i - 1] / d : 0.0);
      if (d == 0.0) d = -1e-300;  // x at an eigenvalue of a leading block: count it below
      c += d < 0.0;
    }
    return c;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-15 * (hi > -lo ? hi : -lo); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (below(mid) == m) hi = mid;
    else lo = mid;
  }
  return hi;
}

// Per-node Dirichlet bit mask (bit f set = DOF f prescribed).
using dmask_t = uint16_t;
static_assert(NF <= 16, "one 16-bit Dirichlet mask per node");
constexpr dmask_t MASK_ALL = dmask_t((1u << NF) - 1u);  // every field
constexpr dmask_t MASK_ETA = dmask_t(MASK_ALL & ~7u);    // the order-parameter fields

}  // namespace pfm

// ---- launchers (host functions; every launch goes on the given stream) ----
namespace pfm {

// Kernel launches issued by the library (incremented by every launcher).
void count_launches(int n);

// element kernels (fe_kernels.cu)
// The element kernels below take an optional scratch W: null = element
// contributions added with atomics (rounding order varies between runs);
// non-null = the atomic-free two-pass form (per-(element, node) contributions
// in W, summed per node in a fixed order; bitwise reproducible). W holds
// 9 * 32 * nblk entries of the output type (+ nblk for the residual's energy).
// df: the point physics in double-float arithmetic (FP32 pipes) instead of FP64
void launch_residual(const Grid& g, const DevParams& P, const double* U, const double* Un,
                     const dmask_t* mask, double* R, double* energy, cudaStream_t s, double* W = nullptr,
                     bool df = false);
// arithmetic of the point physics in the linearisation
enum { LIN_F64 = 0, LIN_F32 = 1, LIN_DF = 2 };
// optional residual of the same state formed in the linearisation pass
// (arith == LIN_F64 only; ignored otherwise): R (zeroed by the caller unless W
// is set), energy (optional), W the atomic-free scratch as for launch_residual
struct LinResidual {
  const dmask_t* mask;
  double* R;
  double* energy;
  double* W;
};
void launch_linearize(const Grid& g, const DevParams& P, const double* U, const double* Un,
                      double* H64, float* H32, float* H32lo, int arith, cudaStream_t s,
                      const LinResidual* res = nullptr);
void launch_japply_df(const Grid& g, const DevParams& P, const float* Hhi, const float* Hlo, const dmask_t* mask,
                      const float* v, double* y, cudaStream_t s, double* W = nullptr);
template <typename T>
void launch_japply(const Grid& g, const DevParams& P, const T* H, const dmask_t* mask, const T* v,
                   T* y, cudaStream_t s, T* W = nullptr);
// y = J v from a binary16 copy of the FP32 store holding s H (FP32 arithmetic;
// inv_scale = 1/s), and the conversion that makes that copy: returns s, a
// power of two putting max |H| in [2^14, 2^15), or 0 on failure (scratch: one
// device word).
void launch_japply_h16(const Grid& g, const DevParams& P, const __half* H, float inv_scale, const dmask_t* mask,
                       const float* v, float* y, cudaStream_t s, float* W = nullptr);
float launch_store_to_half(const Grid& g, const float* H32, __half* H16, unsigned* scratch, cudaStream_t s);
// power-of-two scale s of the binary16 copy for a store whose largest entry
// has magnitude amax (finite)
float half_store_scale(float amax);
// Number of staged tangent applications whose bounded wait gave up since the
// last call (they write NaN into y[0]); resets the count.
int take_wait_timeouts();
// element blocks [b0, b1) only, on at most `blocks` CTAs (slab pipeline)
template <typename T>
void launch_japply_range(const Grid& g, const DevParams& P, const T* H, const dmask_t* mask, const T* v, T* y,
                         int64_t b0, int64_t b1, int blocks, cudaStream_t s);
template <typename T>
void launch_identity_rows(int64_t nn, const dmask_t* mask, const T* v, T* y, int64_t n0, int64_t n1, cudaStream_t s);
int japply_range_blocks();  // persistent grid of k_japply_range
template <typename T>
void launch_blockdiag(const Grid& g, const DevParams& P, const T* H, const dmask_t* mask, T* D, T* W,
                      cudaStream_t s);  // W: scratch of NBD * 32 * nblk entries
template <typename T>
void launch_block_invert(int64_t nn, const dmask_t* mask, T* D, int* singular, cudaStream_t s);
void launch_qp_eval(const DevParams& P, int64_t n, const double* F, const double* eta,
                    const double* eta_n, double* W, double* grad, double* hess, cudaStream_t s);

// multigrid kernels (mg_kernels.cu)
void launch_inject_state(const Grid& fine, const Grid& coarse, const double* Uf, double* Uc,
                         cudaStream_t s);
void launch_coarse_mask(const Grid& fine, const Grid& coarse, const dmask_t* mf, dmask_t* mc,
                        cudaStream_t s);
template <typename T>
void launch_prolong_add(const Grid& fine, const Grid& coarse, const T* xc, const dmask_t* mf, T* xf,
                        cudaStream_t s);
template <typename T>
void launch_restrict(const Grid& fine, const Grid& coarse, const T* rf, const dmask_t* mc, T* rc,
                     cudaStream_t s);
template <typename T>
void launch_smooth(int64_t nn, const T* D, const T* b, const T* y, T omega, T* x, cudaStream_t s);
template <typename T>
void launch_sub(int64_t n, const T* b, const T* y, T* r, cudaStream_t s);
// det: eight element colours one after another, no atomics (bitwise reproducible)
template <typename T>
void launch_coarse_assemble(const Grid& g, const DevParams& P, const T* H, const dmask_t* mask,
                            double* K, int ld, cudaStream_t s, bool det = false);
template <typename T>
void launch_cheb_first(int64_t nn, const T* D, const T* src, T c, bool copy_r, bool zero_x, T* r, T* d, T* x,
                       cudaStream_t s);
template <typename T>
void launch_cheb_step(int64_t nn, const T* D, const T* y, T a, T c, T* r, T* d, T* x, cudaStream_t s);
template <typename T>
void launch_power_init(int64_t nn, const dmask_t* mask, T* x, cudaStream_t s);
template <typename T>
void launch_scale_inv_sqrt(int64_t n, const T* y, const double* dot, T* x, cudaStream_t s);
// Lanczos step: u -= alpha q + sqrt(beta2prev) qp (alpha, beta2prev: device
// scalars; beta2prev null for the first step)
template <typename T>
void launch_lanczos_orth(int64_t n, T* u, const T* q, const T* qp, const double* alpha, const double* beta2prev,
                         cudaStream_t s);
int dense_gauss_jordan_inverse(double* Maug, int n, double* Ainv, unsigned long long* keys, int* used, int* piv,
                               int* singular, cudaStream_t s);
template <typename T>
void launch_coarse_solve(int n, const double* Ainv, const T* b, T* x, cudaStream_t s);

// penalty contact with a rigid sphere on the top face (contact_kernels.cu)
struct ContactParams {
  double center[3];
  double radius;
  double eps_N;
};
int64_t contact_points(const Grid& g);  // surface Gauss points of the top face
void launch_contact_residual(const Grid& g, const ContactParams& c, const double* U, const dmask_t* mask, double* R,
                             double* energy, double* load, cudaStream_t s);
void launch_contact_linearize(const Grid& g, const ContactParams& c, const double* U, double* K64, float* K32,
                              cudaStream_t s);
template <typename TK, typename TV, typename TY>
void launch_contact_apply(const Grid& g, const TK* K, const dmask_t* mask, const TV* v, TY* y, cudaStream_t s);
template <typename T>
void launch_contact_blockdiag(const Grid& g, const T* K, T* D, cudaStream_t s);
void launch_contact_coarse(const Grid& g, const double* K, const dmask_t* mask, double* M, int ld, cudaStream_t s);

// microstructure diagnostics (diag_kernels.cu); partial holds (nz+1)*DIAG_MAX_CHUNKS*4 doubles
constexpr int DIAG_MAX_CHUNKS = 8;
void launch_diagnostics(const Grid& g, const double* U, double* Iv, double* Id, double* es, double* partial,
                        double* stats, cudaStream_t s);

// vector kernels (krylov_kernels.cu)
template <typename T>
void launch_fill(int64_t n, T val, T* x, cudaStream_t s);
void launch_cast_d2f(int64_t n, const double* a, float* b, cudaStream_t s);
void launch_cast_f2d(int64_t n, const float* a, double* b, cudaStream_t s);
// x = hi + lo as two FP32 vectors; r = b - a - c
void launch_split_f64(int64_t n, const double* x, float* hi, float* lo, cudaStream_t s);
void launch_sub2(int64_t n, const double* b, const double* a, const float* c, double* r, cudaStream_t s);
void launch_mdot(int64_t n, int k, const double* V, int64_t ldv, const double* w, double* partial,
                 double* out, cudaStream_t s);
template <typename T>
void launch_dot(int64_t n, const T* a, const T* b, double* partial, double* out, cudaStream_t s);
void launch_maxpy(int64_t n, int k, const double* V, int64_t ldv, const double* h, double* w,
                  cudaStream_t s);
void launch_scale_copy(int64_t n, const double* a, const double* alpha_dev, double* b,
                       cudaStream_t s);
template <typename T>
void launch_gemv_add(int64_t n, int k, const T* Z, int64_t ldz, const double* y, double* x,
                     cudaStream_t s);
void launch_axpy(int64_t n, double a, const double* x, double* y, cudaStream_t s);
void launch_mask_values(int64_t nn, const dmask_t* mask, const double* val, double* U,
                        cudaStream_t s);
void launch_build_mask(int64_t nn, const uint8_t* m8, dmask_t* mask, int* bad, cudaStream_t s);
int reduction_blocks(int64_t n);

}  // namespace pfm
