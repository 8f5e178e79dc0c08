// C ABI of libpfm (include/pfm.h): problem handle, multigrid hierarchy and
// the solver drivers (V-cycle, FGMRES, Newton) that sequence the kernels of
// fe_kernels.cu, mg_kernels.cu and krylov_kernels.cu on one CUDA stream.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "handle.h"
#include "params.h"

using namespace pfm;

namespace {
std::atomic<int64_t> g_launches{0};

// Arithmetic peak probe: every thread runs 8 independent chains of fused
// multiply-adds (x = x * a + b) for `iters` steps and stores their sum, so
// the compiler keeps every operation.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, T a, T b, T* __restrict__ out) {
  T x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = T(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  out[int64_t(blockIdx.x) * blockDim.x + threadIdx.x] = s;
}
}  // namespace

void pfm::count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {
std::string g_create_error;

// Records a start event on construction and a stop event on destruction
// (both on the handle's stream) when profiling is enabled.
struct ProfScope {
  pfm_handle* h;
  int id;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(pfm_handle* h_, int id_, bool on = true) : h(h_), id(id_) {
    if (!h->prof || !on) { h = nullptr; return; }
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, h->stream);
  }
  ~ProfScope() {
    if (!h) return;
    cudaEventRecord(b, h->stream);
    h->prof_ev[id].emplace_back(a, b);
  }
};

void prof_collect(pfm_handle* h) {
  for (int id = 0; id < PFM_PROF_COUNT; ++id) {
    for (auto& e : h->prof_ev[id]) {
      float ms = 0.f;
      cudaEventSynchronize(e.second);
      cudaEventElapsedTime(&ms, e.first, e.second);
      h->prof_ms[id] += ms;
      h->prof_n[id] += 1;
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
    h->prof_ev[id].clear();
  }
}

pfm_status bd_scratch(pfm_handle* h, size_t bytes);

// Deterministic mode: make sure the scratch of the atomic-free element kernels
// exists (9 * 32 + 1 doubles per element block of the finest level, enough for
// every level and output type); contact terms are not covered.
pfm_status det_ready(pfm_handle* h) {
  if (!h->det) return PFM_OK;
  if (h->contact_on)
    return h->fail(PFM_ERR_INVALID_ARG, "deterministic mode does not cover penalty contact");
  return bd_scratch(h, size_t(NF * 32 + 1) * size_t(h->L[0].nblk) * sizeof(double));
}

// Scratch of the atomic-free element kernels (after det_ready), or null.
template <typename T>
T* det_W(pfm_handle* h) {
  return h->det ? static_cast<T*>(h->bd_scratch) : nullptr;
}

// Tangent application inside the preconditioner on level l: from the level's
// store, or from its binary16 copy when that is enabled and current (FP32);
// timed on the finest level unless `timed` is false.
template <typename T>
void precond_apply(pfm_handle* h, size_t l, const T* x, T* y, bool timed = true) {
  Level& lv = h->L[l];
  const bool on = timed && l == 0;
  if constexpr (sizeof(T) == 4) {
    if (lv.H16 && lv.h16_scale > 0.f) {
      ProfScope ps(h, PFM_PROF_JAPPLY_F16, on);
      launch_japply_h16(lv.g, h->dp, lv.H16, 1.f / lv.h16_scale, lv.mask, x, y, h->stream, det_W<float>(h));
      if (h->contact_on) launch_contact_apply<T, T, T>(lv.g, LvVec<T>::Kc(lv), lv.mask, x, y, h->stream);
      return;
    }
  }
  ProfScope ps(h, sizeof(T) == 4 ? PFM_PROF_JAPPLY_F32 : PFM_PROF_JAPPLY_F64, on);
  launch_japply<T>(lv.g, h->dp, LvVec<T>::H(lv), lv.mask, x, y, h->stream, det_W<T>(h));
  if (h->contact_on) launch_contact_apply<T, T, T>(lv.g, LvVec<T>::Kc(lv), lv.mask, x, y, h->stream);
}

// ---------------------------------------------------------------------------
// Level smoothing. Chebyshev (type 0): the Chebyshev iteration for D^-1 J on
// [lo, hi] = [cheb_lo, cheb_hi] * lambda_max(D^-1 J) (Saad, Iterative Methods
// for Sparse Linear Systems, Alg. 12.1), i.e. point-block Jacobi relaxation
// (Sec. 3.4) with Chebyshev step lengths. Damped Jacobi (type 1):
// x += omega D^-1 (b - J x). Both cost one tangent application per step.
struct SmoothCfg {
  int nu_pre = 4, nu_post = 4, type = 0;
  double omega = 0.7, lo = 0.05, hi = 1.1;
  int gamma = 1;
  double growth = 1.0;
};

SmoothCfg smooth_cfg(const pfm_solve_opts* o) {
  SmoothCfg c;
  if (o) {
    c.nu_pre = o->nu_pre;
    c.nu_post = o->nu_post;
    c.type = o->smoother;
    c.omega = o->omega;
    c.lo = o->cheb_lo;
    c.hi = o->cheb_hi;
    c.gamma = o->cycle_gamma > 0 ? o->cycle_gamma : 1;
    c.growth = o->nu_growth > 0 ? o->nu_growth : 1.0;
  }
  return c;
}

// nu steps on level l from x = 0 (zero_x) or from the current x; with
// want_res the final residual b - J x is left in the level's r vector.
template <typename T>
pfm_status smooth(pfm_handle* h, size_t l, bool zero_x, int nu, bool want_res, const SmoothCfg& c) {
  Level& lv = h->L[l];
  cudaStream_t s = h->stream;
  T* x = LvVec<T>::x(lv);
  T* b = LvVec<T>::b(lv);
  T* y = LvVec<T>::y(lv);
  T* r = LvVec<T>::r(lv);
  T* d = LvVec<T>::d(lv);
  const T* D = LvVec<T>::D(lv);
  const int64_t n = ndof(lv);
  if (c.type == 1) {
    if (zero_x) {
      CK(cudaMemsetAsync(x, 0, sizeof(T) * n, s));
      launch_smooth<T>(lv.nn, D, b, nullptr, T(c.omega), x, s);
    } else {
      precond_apply<T>(h, l, x, y);
      launch_smooth<T>(lv.nn, D, b, y, T(c.omega), x, s);
    }
    for (int k = 1; k < nu; ++k) {
      precond_apply<T>(h, l, x, y);
      launch_smooth<T>(lv.nn, D, b, y, T(c.omega), x, s);
    }
    if (want_res) {
      precond_apply<T>(h, l, x, y);
      launch_sub<T>(n, b, y, r, s);
    }
    CKL();
    return PFM_OK;
  }
  const double hi = c.hi * lv.lam, lo = c.lo * lv.lam;
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  double rho = 1.0 / sigma;
  if (zero_x) {
    launch_cheb_first<T>(lv.nn, D, b, T(1.0 / theta), true, true, r, d, x, s);
  } else {
    precond_apply<T>(h, l, x, y);
    launch_sub<T>(n, b, y, r, s);
    launch_cheb_first<T>(lv.nn, D, r, T(1.0 / theta), false, false, r, d, x, s);
  }
  for (int k = 1; k < nu; ++k) {
    precond_apply<T>(h, l, d, y);
    const double rho_n = 1.0 / (2.0 * sigma - rho);
    launch_cheb_step<T>(lv.nn, D, y, T(rho_n * rho), T(2.0 * rho_n / delta), r, d, x, s);
    rho = rho_n;
  }
  if (want_res) {
    precond_apply<T>(h, l, d, y);
    launch_sub<T>(n, r, y, r, s);
  }
  CKL();
  return PFM_OK;
}

// V-cycle (Sec. 3.4): pre-smooth, restrict the residual, recurse, coarse
// solve, prolong the correction, post-smooth.
template <typename T>
pfm_status vcycle_level(pfm_handle* h, size_t l, const SmoothCfg& c) {
  ProfScope ps(h, PFM_PROF_VCYCLE, l == 0);
  Level& lv = h->L[l];
  cudaStream_t s = h->stream;
  T* x = LvVec<T>::x(lv);
  T* b = LvVec<T>::b(lv);
  if (l + 1 == h->L.size()) {
    launch_coarse_solve<T>(h->nc_dofs, h->Kinv, b, x, s);
    CKL();
    return PFM_OK;
  }
  const double gl = std::pow(c.growth, double(l));
  const int nu_pre = std::max(1, int(std::lround(c.nu_pre * gl)));
  const int nu_post = c.nu_post > 0 ? std::max(1, int(std::lround(c.nu_post * gl))) : 0;
  TRY(smooth<T>(h, l, true, nu_pre, true, c));
  Level& cv = h->L[l + 1];
  for (int g = 0; g < c.gamma; ++g) {
    // coarse correction of the current residual r (recomputed after the first one)
    if (g > 0) {
      precond_apply<T>(h, l, x, LvVec<T>::y(lv));
      launch_sub<T>(ndof(lv), b, LvVec<T>::y(lv), LvVec<T>::r(lv), s);
    }
    launch_restrict<T>(lv.g, cv.g, LvVec<T>::r(lv), cv.mask, LvVec<T>::b(cv), s);
    CKL();
    TRY(vcycle_level<T>(h, l + 1, c));
    launch_prolong_add<T>(lv.g, cv.g, LvVec<T>::x(cv), lv.mask, x, s);
    CKL();
  }
  if (nu_post > 0) TRY(smooth<T>(h, l, false, nu_post, false, c));
  return PFM_OK;
}

template <typename T>
pfm_status ensure_level_vectors(pfm_handle* h) {
  for (auto& lv : h->L) {
    TRY(dalloc(h, &LvVec<T>::x(lv), ndof(lv)));
    TRY(dalloc(h, &LvVec<T>::b(lv), ndof(lv)));
    TRY(dalloc(h, &LvVec<T>::y(lv), ndof(lv)));
    TRY(dalloc(h, &LvVec<T>::r(lv), ndof(lv)));
    TRY(dalloc(h, &LvVec<T>::d(lv), ndof(lv)));
  }
  return PFM_OK;
}

// lambda_max(D^-1 J) on level l by power_its steps of the Lanczos process
// (Saad, Numerical Methods for Large Eigenvalue Problems, Alg. 6.5) for
// A = J D^-1, which is self-adjoint in the inner product <u, v> = u^T D^-1 v
// and has the eigenvalues of D^-1 J: from a fixed pseudo-random q_0 with
// z_0 = D^-1 q_0 (both scaled to <q_0, q_0> = 1), step j forms u = J z_j,
// alpha_j = z_j^T u, u -= alpha_j q_j + beta_{j-1} q_{j-1}, w = D^-1 u,
// beta_j^2 = u^T w, q_{j+1} = u / beta_j, z_{j+1} = w / beta_j; the scalars stay
// on the device (FP64 dots) and are read once at the end, and the largest
// eigenvalue of the tridiagonal (alpha, beta) is the estimate. Its Ritz
// value approaches lambda_max from below much faster than a power iteration
// (the spectrum of D^-1 J is dense near its top).
template <typename T>
pfm_status estimate_lambda(pfm_handle* h, size_t l) {
  Level& lv = h->L[l];
  cudaStream_t s = h->stream;
  const int64_t n = ndof(lv);
  const int K = h->power_its;
  if (h->lz_cap < 2 * K + 1) {
    dfree(h->lz);
    TRY(dalloc(h, &h->lz, size_t(2 * K + 1)));
    h->lz_cap = 2 * K + 1;
  }
  double* al = h->lz;
  double* be = h->lz + K;
  double* nrm = h->lz + 2 * K;
  T* q = LvVec<T>::x(lv);
  T* qp = LvVec<T>::b(lv);
  T* z = LvVec<T>::d(lv);
  T* u = LvVec<T>::y(lv);
  T* w = LvVec<T>::r(lv);
  const T* D = LvVec<T>::D(lv);
  auto dinv = [&](const T* src, T* dst) {  // dst = D^-1 src
    CK(cudaMemsetAsync(dst, 0, sizeof(T) * n, s));
    launch_smooth<T>(lv.nn, D, src, nullptr, T(1), dst, s);
    return PFM_OK;
  };
  launch_power_init<T>(lv.nn, lv.mask, q, s);
  TRY(dinv(q, z));
  launch_dot<T>(n, q, z, h->partial, nrm, s);
  launch_scale_inv_sqrt<T>(n, q, nrm, q, s);
  launch_scale_inv_sqrt<T>(n, z, nrm, z, s);
  CK(cudaMemsetAsync(qp, 0, sizeof(T) * n, s));
  CKL_AT("eigenvalue estimate start");
  for (int j = 0; j < K; ++j) {
    precond_apply<T>(h, l, z, u, false);
    CKL_AT("eigenvalue estimate: tangent application");
    launch_dot<T>(n, z, u, h->partial, al + j, s);
    launch_lanczos_orth<T>(n, u, q, qp, al + j, j > 0 ? be + j - 1 : nullptr, s);
    TRY(dinv(u, w));
    launch_dot<T>(n, u, w, h->partial, be + j, s);
    if (j + 1 < K) {
      std::swap(q, qp);
      launch_scale_inv_sqrt<T>(n, u, be + j, q, s);
      launch_scale_inv_sqrt<T>(n, w, be + j, z, s);
    }
    CKL_AT("eigenvalue estimate");
  }
  std::vector<double> hab(size_t(2 * K));
  CK(cudaMemcpyAsync(hab.data(), h->lz, sizeof(double) * 2 * K, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double lam = tridiag_max_eig(hab.data(), hab.data() + K, K);
  if (!(lam > 0.0) || !std::isfinite(lam)) return h->fail(PFM_ERR_BREAKDOWN, "smoother eigenvalue estimate failed");
  lv.lam = lam;
  return PFM_OK;
}

// z = M r with r, z in the preconditioner's precision (device arrays of the finest level).
template <typename T>
pfm_status apply_vcycle(pfm_handle* h, const T* r, T* z, const SmoothCfg& c) {
  TRY(det_ready(h));
  TRY(ensure_level_vectors<T>(h));
  Level& f = h->L[0];
  CK(cudaMemcpyAsync(LvVec<T>::b(f), r, sizeof(T) * ndof(f), cudaMemcpyDeviceToDevice, h->stream));
  TRY(vcycle_level<T>(h, 0, c));
  CK(cudaMemcpyAsync(z, LvVec<T>::x(f), sizeof(T) * ndof(f), cudaMemcpyDeviceToDevice, h->stream));
  return PFM_OK;
}

pfm_status check_ready(pfm_handle* h, bool need_lin) {
  if (!h) return PFM_ERR_INVALID_ARG;
  if (!h->have_state) return h->fail(PFM_ERR_STATE, "no state: call pfm_set_state first");
  if (need_lin && !h->linearized) return h->fail(PFM_ERR_STATE, "no tangent: call pfm_linearize first");
  return PFM_OK;
}

pfm_status residual_impl(pfm_handle* h, double* R, double* energy_host) {
  Level& f = h->L[0];
  cudaStream_t s = h->stream;
  TRY(det_ready(h));
  if (!h->det) CK(cudaMemsetAsync(R, 0, sizeof(double) * ndof(f), s));  // the atomic form adds into R
  CK(cudaMemsetAsync(h->energy_dev, 0, sizeof(double), s));
  {
    ProfScope ps(h, PFM_PROF_RESIDUAL);
    launch_residual(f.g, h->dp, f.U, f.Un, f.mask, R, h->energy_dev, s, det_W<double>(h), h->res_df);
    if (h->contact_on) launch_contact_residual(f.g, h->contact, f.U, f.mask, R, h->energy_dev, nullptr, s);
  }
  CKL();
  if (energy_host) {
    CK(cudaMemcpyAsync(energy_host, h->energy_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  return PFM_OK;
}

pfm_status norm2(pfm_handle* h, const double* x, int64_t n, double* out) {
  launch_mdot(n, 1, x, 0, x, h->partial, h->hdev, h->stream);
  CKL();
  double v = 0.0;
  CK(cudaMemcpyAsync(&v, h->hdev, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *out = std::sqrt(v);
  return PFM_OK;
}

// Scratch of at least `bytes` for the diagonal-block passes (kept on the handle).
pfm_status bd_scratch(pfm_handle* h, size_t bytes) {
  if (h->bd_bytes >= bytes) return PFM_OK;
  if (h->bd_scratch) CK(cudaStreamSynchronize(h->stream));
  if (h->bd_scratch) cudaFree(h->bd_scratch);
  h->bd_scratch = nullptr;
  h->bd_bytes = 0;
  char* p = nullptr;
  TRY(dalloc(h, &p, bytes));
  h->bd_scratch = p;
  h->bd_bytes = bytes;
  return PFM_OK;
}

// Residual of the finest level formed by its linearisation pass (both in FP64
// arithmetic): the two share the point physics of the state.
bool residual_fusable(const pfm_handle* h) { return !h->res_df && !h->lin_df; }

// R_fused: when set (residual_fusable), the finest level's linearisation also
// writes the residual of the state into R_fused (and the energy into
// energy_dev), as residual_impl would.
pfm_status linearize_impl(pfm_handle* h, pfm_precision prec, double* R_fused = nullptr) {
  cudaStream_t s = h->stream;
  if (h->vgraph) {  // smoother coefficients change with the eigenvalue estimates
    cudaGraphExecDestroy(h->vgraph);
    h->vgraph = nullptr;
  }
  TRY(det_ready(h));
  const size_t nl = h->L.size();
  for (size_t l = 1; l < nl; ++l) {
    launch_inject_state(h->L[l - 1].g, h->L[l].g, h->L[l - 1].U, h->L[l].U, s);
    launch_inject_state(h->L[l - 1].g, h->L[l].g, h->L[l - 1].Un, h->L[l].Un, s);
  }
  CKL_AT("state injection");
  CK(cudaMemsetAsync(h->flag_dev, 0, sizeof(int), s));
  for (size_t l = 0; l < nl; ++l) {
    Level& lv = h->L[l];
    const bool coarsest = (l + 1 == nl);
    const bool fine = (l == 0);
    const size_t hsz = size_t(lv.nblk) * HBLK;
    const bool need64 = fine || coarsest || prec == PFM_F64;
    // the finest level of a mixed solve always needs the FP32 pair (the
    // double-float outer operator reads it), also when it is the only level
    const bool need32 = prec == PFM_F32 && (fine || !coarsest);
    if (need64) TRY(dalloc(h, &lv.H64, hsz));
    if (need32) TRY(dalloc(h, &lv.H32, hsz));
    const bool needlo = fine && need32;
    if (needlo) TRY(dalloc(h, &lv.H32lo, hsz));
    {
      ProfScope ps(h, PFM_PROF_LINEARIZE, fine);
      // intermediate levels of an FP32 preconditioner need only FP32 Hessians;
      // the others FP64-class ones (FP64 or double-float arithmetic)
      const bool fp32_compute = !fine && !coarsest && prec == PFM_F32;
      const int arith = fp32_compute ? LIN_F32 : (h->lin_df ? LIN_DF : LIN_F64);
      if (fine && R_fused) {
        if (!h->det) CK(cudaMemsetAsync(R_fused, 0, sizeof(double) * ndof(lv), s));
        CK(cudaMemsetAsync(h->energy_dev, 0, sizeof(double), s));
        const LinResidual res{lv.mask, R_fused, h->energy_dev, det_W<double>(h)};
        launch_linearize(lv.g, h->dp, lv.U, lv.Un, need64 ? lv.H64 : nullptr, need32 ? lv.H32 : nullptr,
                         needlo ? lv.H32lo : nullptr, arith, s, &res);
        if (h->contact_on) launch_contact_residual(lv.g, h->contact, lv.U, lv.mask, R_fused, h->energy_dev, nullptr, s);
      } else {
        launch_linearize(lv.g, h->dp, lv.U, lv.Un, need64 ? lv.H64 : nullptr, need32 ? lv.H32 : nullptr,
                         needlo ? lv.H32lo : nullptr, arith, s);
      }
    }
    CKL_AT("Gauss-point Hessians");
    lv.h16_scale = 0.f;
    if (need32 && h->pre_h16) {
      TRY(dalloc(h, &lv.H16, hsz));
      if (!h->amax_dev) TRY(dalloc(h, &h->amax_dev, 1));
      lv.h16_scale = launch_store_to_half(lv.g, lv.H32, lv.H16, h->amax_dev, s);
      if (!(lv.h16_scale > 0.f)) return h->fail(PFM_ERR_NONFINITE, "binary16 store: non-finite Hessian entries");
    }
    if (h->contact_on) {
      TRY(dalloc(h, &lv.Kc64, size_t(6) * contact_points(lv.g)));
      TRY(dalloc(h, &lv.Kc32, size_t(6) * contact_points(lv.g)));
      launch_contact_linearize(lv.g, h->contact, lv.U, lv.Kc64, lv.Kc32, s);
    }
    CKL();
    if (coarsest) continue;
    if (prec == PFM_F32) {
      TRY(dalloc(h, &lv.D32, size_t(NF2) * lv.nn));
      TRY(bd_scratch(h, size_t(NBD) * 32 * lv.nblk * sizeof(float)));
      launch_blockdiag<float>(lv.g, h->dp, lv.H32, lv.mask, lv.D32, static_cast<float*>(h->bd_scratch), s);
      if (h->contact_on) launch_contact_blockdiag<float>(lv.g, lv.Kc32, lv.D32, s);
      CKL_AT("diagonal blocks");
      launch_block_invert<float>(lv.nn, lv.mask, lv.D32, h->flag_dev, s);
      CKL_AT("block inverses");
      TRY(ensure_level_vectors<float>(h));
      TRY(estimate_lambda<float>(h, l));
    } else {
      TRY(dalloc(h, &lv.D64, size_t(NF2) * lv.nn));
      TRY(bd_scratch(h, size_t(NBD) * 32 * lv.nblk * sizeof(double)));
      launch_blockdiag<double>(lv.g, h->dp, lv.H64, lv.mask, lv.D64, static_cast<double*>(h->bd_scratch), s);
      if (h->contact_on) launch_contact_blockdiag<double>(lv.g, lv.Kc64, lv.D64, s);
      CKL_AT("diagonal blocks");
      launch_block_invert<double>(lv.nn, lv.mask, lv.D64, h->flag_dev, s);
      CKL_AT("block inverses");
      TRY(ensure_level_vectors<double>(h));
      TRY(estimate_lambda<double>(h, l));
    }
  }
  Level& c = h->L[nl - 1];
  launch_coarse_assemble<double>(c.g, h->dp, c.H64, c.mask, h->Kaug, 2 * h->nc_dofs, s, h->det);
  if (h->contact_on) launch_contact_coarse(c.g, c.Kc64, c.mask, h->Kaug, 2 * h->nc_dofs, s);
  CKL_AT("coarse operator");
  dense_gauss_jordan_inverse(h->Kaug, h->nc_dofs, h->Kinv, h->gj_keys, h->gj_used, h->gj_piv, h->flag_dev, s);
  CKL_AT("coarse inverse");
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, h->flag_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (flag) return h->fail(PFM_ERR_BREAKDOWN, "singular nodal block or coarse operator");
  h->linearized = true;
  h->lin_prec = prec;
  return PFM_OK;
}

template <typename T>
pfm_status japply_impl(pfm_handle* h, const T* v, T* y) {
  Level& f = h->L[0];
  const T* H = LvVec<T>::H(f);
  if (!H || (sizeof(T) == 4 && h->lin_prec != PFM_F32))
    return h->fail(PFM_ERR_STATE, "no tangent in the requested precision (linearize with PFM_F32 for FP32)");
  TRY(det_ready(h));
  precond_apply<T>(h, 0, v, y);
  CKL();
  return PFM_OK;
}

// FGMRES(m), right preconditioned, x0 = 0 (Sec. 3.4 uses GMRES; the flexible
// variant allows a preconditioner that changes between iterations, here an
// FP32 V-cycle). Orthogonalisation: classical Gram-Schmidt applied twice.
// Written as a resumable state machine so that a batch of problems can be
// advanced in lockstep: enqueue one iteration on every problem's stream,
// synchronise once, then finish the iteration of each (Givens rotation,
// convergence test, next basis vector or update and restart).
struct Fgm {
  pfm_solve_opts o{};
  const double* b = nullptr;
  double* x = nullptr;
  int m = 0;
  bool mixed = false;
  SmoothCfg sc;
  double beta0 = 0.0, beta = 0.0, tol = 0.0, relres = 1.0;
  int total = 0, j = 0;
  bool done = false, converged = false;
  // inner solve of iterative refinement (krylov 2): FP32 operator, one cycle,
  // stop at max(switch_rtol ||b||, tol_floor)
  bool inner = false;
  double tol_floor = 0.0;
  // relaxed products (krylov 1): FP32 products once the residual estimate
  // resest is at most switch_abs; the true residual decides convergence
  bool relax = false;
  double switch_abs = 0.0, resest = 0.0;
  int cycles = 0;
  pfm_status status = PFM_OK;
  std::vector<double> Hh, cs, sn, g;
};

pfm_status fgm_alloc(pfm_handle* h, Fgm& F) {
  Level& f = h->L[0];
  const int64_t n = ndof(f);
  const int m = F.m;
  if (h->kry_m < m || h->kry_prec != F.o.precond) {
    dfree(h->V);
    if (h->Z) cudaFree(h->Z);
    h->Z = nullptr;
    TRY(dalloc(h, &h->V, size_t(m + 1) * n));
    if (F.mixed) {
      float* z = nullptr;
      TRY(dalloc(h, &z, size_t(m) * n));
      h->Z = z;
    } else {
      double* z = nullptr;
      TRY(dalloc(h, &z, size_t(m) * n));
      h->Z = z;
    }
    h->kry_m = m;
    h->kry_prec = F.o.precond;
  }
  if (!h->hpin) {
    CK(cudaMallocHost(reinterpret_cast<void**>(&h->hpin), sizeof(double) * (2 * (MAX_RESTART + 1) + 2)));
  }
  if (F.mixed) {
    TRY(ensure_level_vectors<float>(h));
  } else {
    TRY(ensure_level_vectors<double>(h));
  }
  return PFM_OK;
}

// Set up and enqueue ||b|| (read back into the pinned slot hpin[0]).
pfm_status fgm_begin_enqueue(pfm_handle* h, Fgm& F, const pfm_solve_opts& o, const double* b, double* x) {
  F = Fgm{};
  F.o = o;
  F.b = b;
  F.x = x;
  F.m = o.restart;
  F.mixed = (o.precond == PFM_F32);
  F.relax = F.mixed && o.krylov == 1;
  F.sc = smooth_cfg(&o);
  if (F.mixed && h->lin_prec != PFM_F32)
    return h->fail(PFM_ERR_STATE, "FP32 preconditioner requested but the tangent was built for FP64");
  if (F.mixed && h->outer_df && (!h->L[0].H32 || !h->L[0].H32lo))
    return h->fail(PFM_ERR_STATE, "the double-float outer operator has no FP32 Hessian pair");
  TRY(det_ready(h));
  TRY(fgm_alloc(h, F));
  F.Hh.assign(size_t(F.m + 1) * F.m, 0.0);
  F.cs.assign(F.m, 0.0);
  F.sn.assign(F.m, 0.0);
  F.g.assign(F.m + 1, 0.0);
  const int64_t n = ndof(h->L[0]);
  cudaStream_t s = h->stream;
  CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
  CK(cudaMemcpyAsync(h->rv, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  launch_mdot(n, 1, b, 0, b, h->partial, h->hdev, s);
  CKL();
  CK(cudaMemcpyAsync(h->hpin, h->hdev, sizeof(double), cudaMemcpyDeviceToHost, s));
  return PFM_OK;
}

pfm_status fgm_start_cycle(pfm_handle* h, Fgm& F) {
  const int64_t n = ndof(h->L[0]);
  cudaStream_t s = h->stream;
  h->hpin[2 * (MAX_RESTART + 1) + 1] = F.beta;
  CK(cudaMemcpyAsync(h->hdev, &h->hpin[2 * (MAX_RESTART + 1) + 1], sizeof(double), cudaMemcpyHostToDevice, s));
  launch_scale_copy(n, h->rv, h->hdev, h->V, s);
  CKL();
  std::fill(F.g.begin(), F.g.end(), 0.0);
  F.g[0] = F.beta;
  F.j = 0;
  F.resest = F.beta;
  ++F.cycles;
  return PFM_OK;
}

// After the ||b|| copy has landed.
pfm_status fgm_begin_finish(pfm_handle* h, Fgm& F) {
  F.beta0 = std::sqrt(h->hpin[0]);
  if (!std::isfinite(F.beta0)) {
    F.done = true;
    return F.status = h->fail(PFM_ERR_NONFINITE, "non-finite right-hand side");
  }
  if (F.beta0 == 0.0) {
    F.done = F.converged = true;
    F.relres = 0.0;
    return PFM_OK;
  }
  F.tol = F.inner ? std::max(F.o.switch_rtol * F.beta0, F.tol_floor) : F.o.lin_rtol * F.beta0;
  F.switch_abs = F.o.switch_rtol * F.beta0;
  F.beta = F.beta0;
  return fgm_start_cycle(h, F);
}

template <typename T>
pfm_status capture_vcycle(pfm_handle* h, const SmoothCfg& sc);
pfm_status true_residual(pfm_handle* h, const double* b, const double* x, double* r);

// z_j = M v_j, w = J z_j, two Gram-Schmidt passes and ||w||^2, with the
// Hessenberg column copied to the pinned host slots (no synchronisation).
pfm_status fgm_enqueue(pfm_handle* h, Fgm& F) {
  Level& fl = h->L[0];
  cudaStream_t s = h->stream;
  const int64_t n = ndof(fl);
  const int m = F.m, j = F.j;
  double* vj = h->V + size_t(j) * n;
  if (F.mixed) {
    float* zj = static_cast<float*>(h->Z) + size_t(j) * n;
    launch_cast_d2f(n, vj, fl.b32, s);
    if (h->use_graphs) {
      TRY(capture_vcycle<float>(h, F.sc));
      CK(cudaGraphLaunch(h->vgraph, s));
    } else {
      TRY(vcycle_level<float>(h, 0, F.sc));
    }
    CK(cudaMemcpyAsync(zj, fl.x32, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
    // w = J z_j with the FP64-accurate operator: either the FP64 kernel or,
    // since z_j is exactly FP32, the double-float kernel on the FP32 pipes;
    // inside iterative refinement, and for the relaxed products once the
    // residual estimate is small, the FP32 operator of the FP32 store
    if (F.inner || (F.relax && F.resest <= F.switch_abs)) {
      {
        ProfScope ps(h, PFM_PROF_JAPPLY_F32);
        launch_japply<float>(fl.g, h->dp, fl.H32, fl.mask, zj, fl.y32, s, det_W<float>(h));
        if (h->contact_on) launch_contact_apply<float, float, float>(fl.g, fl.Kc32, fl.mask, zj, fl.y32, s);
      }
      launch_cast_f2d(n, fl.y32, h->wv, s);
    } else if (h->outer_df) {
      ProfScope ps(h, PFM_PROF_JAPPLY_F64);
      launch_japply_df(fl.g, h->dp, fl.H32, fl.H32lo, fl.mask, zj, h->wv, s, det_W<double>(h));
      if (h->contact_on) launch_contact_apply<double, float, double>(fl.g, fl.Kc64, fl.mask, zj, h->wv, s);
    } else {
      launch_cast_f2d(n, zj, h->zd, s);
      TRY(japply_impl<double>(h, h->zd, h->wv));
    }
    CKL();
  } else {
    double* zj = static_cast<double*>(h->Z) + size_t(j) * n;
    CK(cudaMemcpyAsync(fl.b64, vj, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if (h->use_graphs) {
      TRY(capture_vcycle<double>(h, F.sc));
      CK(cudaGraphLaunch(h->vgraph, s));
    } else {
      TRY(vcycle_level<double>(h, 0, F.sc));
    }
    CK(cudaMemcpyAsync(zj, fl.x64, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(h->zd, zj, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  }
  if (!F.mixed) TRY(japply_impl<double>(h, h->zd, h->wv));
  double* h1 = h->hdev;
  double* h2 = h->hdev + (m + 1);
  double* hn = h->hdev + 2 * (m + 1);
  launch_mdot(n, j + 1, h->V, n, h->wv, h->partial, h1, s);
  launch_maxpy(n, j + 1, h->V, n, h1, h->wv, s);
  launch_mdot(n, j + 1, h->V, n, h->wv, h->partial, h2, s);
  launch_maxpy(n, j + 1, h->V, n, h2, h->wv, s);
  launch_mdot(n, 1, h->wv, 0, h->wv, h->partial, hn, s);
  CKL();
  CK(cudaMemcpyAsync(h->hpin, h->hdev, sizeof(double) * (2 * (m + 1) + 1), cudaMemcpyDeviceToHost, s));
  return PFM_OK;
}

// x += Z y with y = R^-1 g (back substitution on the host).
pfm_status fgm_update(pfm_handle* h, Fgm& F, int kdone) {
  if (kdone == 0) return PFM_OK;
  const int m = F.m;
  const int64_t n = ndof(h->L[0]);
  cudaStream_t s = h->stream;
  std::vector<double> y(kdone, 0.0);
  for (int i = kdone - 1; i >= 0; --i) {
    double acc = F.g[i];
    for (int k = i + 1; k < kdone; ++k) acc -= F.Hh[i * m + k] * y[k];
    y[i] = acc / F.Hh[i * m + i];
  }
  double* ypin = h->hpin + (m + 1);  // the h2 slots are free at this point
  for (int i = 0; i < kdone; ++i) ypin[i] = y[i];
  CK(cudaMemcpyAsync(h->hdev, ypin, sizeof(double) * kdone, cudaMemcpyHostToDevice, s));
  if (F.mixed)
    launch_gemv_add<float>(n, kdone, static_cast<float*>(h->Z), n, h->hdev, F.x, s);
  else
    launch_gemv_add<double>(n, kdone, static_cast<double*>(h->Z), n, h->hdev, F.x, s);
  CKL();
  return PFM_OK;
}

// After the column copy of fgm_enqueue has landed.
pfm_status fgm_finish(pfm_handle* h, Fgm& F) {
  const int m = F.m, j = F.j;
  const int64_t n = ndof(h->L[0]);
  cudaStream_t s = h->stream;
  const double* hcol = h->hpin;
  ++F.total;
  const double hnorm = std::sqrt(hcol[2 * (m + 1)]);
  if (!std::isfinite(hnorm)) {
    F.done = true;
    return F.status = h->fail(PFM_ERR_NONFINITE, "non-finite Krylov vector");
  }
  for (int i = 0; i <= j; ++i) F.Hh[i * m + j] = hcol[i] + hcol[(m + 1) + i];
  F.Hh[(j + 1) * m + j] = hnorm;
  for (int i = 0; i < j; ++i) {
    const double a = F.Hh[i * m + j], bb = F.Hh[(i + 1) * m + j];
    F.Hh[i * m + j] = F.cs[i] * a + F.sn[i] * bb;
    F.Hh[(i + 1) * m + j] = -F.sn[i] * a + F.cs[i] * bb;
  }
  const double a = F.Hh[j * m + j], bb = F.Hh[(j + 1) * m + j];
  const double rr = std::hypot(a, bb);
  if (rr == 0.0) {
    F.done = true;
    return F.status = h->fail(PFM_ERR_BREAKDOWN, "zero Hessenberg column");
  }
  F.cs[j] = a / rr;
  F.sn[j] = bb / rr;
  F.Hh[j * m + j] = rr;
  F.Hh[(j + 1) * m + j] = 0.0;
  F.g[j + 1] = -F.sn[j] * F.g[j];
  F.g[j] = F.cs[j] * F.g[j];
  F.relres = std::fabs(F.g[j + 1]) / F.beta0;
  F.resest = std::fabs(F.g[j + 1]);
  const bool conv = std::fabs(F.g[j + 1]) <= F.tol;
  const bool happy = hnorm <= 1e-300;
  if (!conv && !happy && j + 1 < m && F.total < F.o.max_lin_it) {
    // next basis vector v_{j+1} = w / h_{j+1,j}
    h->hpin[2 * (MAX_RESTART + 1) + 1] = hnorm;
    CK(cudaMemcpyAsync(h->hdev + 2 * (m + 1), &h->hpin[2 * (MAX_RESTART + 1) + 1], sizeof(double),
                       cudaMemcpyHostToDevice, s));
    launch_scale_copy(n, h->wv, h->hdev + 2 * (m + 1), h->V + size_t(j + 1) * n, s);
    CKL();
    F.j = j + 1;
    return PFM_OK;
  }
  TRY(fgm_update(h, F, j + 1));
  if (conv && !F.relax) {
    F.done = F.converged = true;
    return PFM_OK;
  }
  if (F.inner) {  // one cycle: the refinement step computes the true residual
    F.done = true;
    return PFM_OK;
  }
  // restart from the true residual r = b - J x; with relaxed products this
  // residual also decides convergence (the estimate followed inexact products)
  if (F.relax) {
    TRY(true_residual(h, F.b, F.x, h->rv));
  } else {
    TRY(japply_impl<double>(h, F.x, h->wv));
    launch_sub<double>(n, F.b, h->wv, h->rv, s);
  }
  TRY(norm2(h, h->rv, n, &F.beta));
  F.relres = F.beta / F.beta0;
  if (F.beta <= F.tol) {
    F.done = F.converged = true;
    return PFM_OK;
  }
  if (F.total >= F.o.max_lin_it) {
    F.done = true;
    return F.status = h->fail(PFM_ERR_NOT_CONVERGED,
                              "FGMRES reached max_lin_it at relative residual " + std::to_string(F.relres));
  }
  return fgm_start_cycle(h, F);
}

pfm_status fgmres_impl(pfm_handle* h, const pfm_solve_opts& o, const double* b, double* x, int* its_out,
                       double* relres_out, int* cycles_out = nullptr) {
  Fgm F;
  TRY(fgm_begin_enqueue(h, F, o, b, x));
  CK(cudaStreamSynchronize(h->stream));
  pfm_status st = fgm_begin_finish(h, F);
  while (st == PFM_OK && !F.done) {
    st = fgm_enqueue(h, F);
    if (st != PFM_OK) break;
    CK(cudaStreamSynchronize(h->stream));
    st = fgm_finish(h, F);
  }
  if (its_out) *its_out = F.total;
  if (relres_out) *relres_out = F.relres;
  if (cycles_out) *cycles_out = F.relax ? F.cycles : 0;
  return st;
}

// y = J x for an FP64 x with FP64-class accuracy: x = x_hi + x_lo (two FP32
// vectors), J x_hi by the double-float operator and J x_lo (2^-24 smaller) by
// the FP32 operator, r = b - J x_hi - J x_lo; or with the FP64 kernel when
// the outer operator is FP64.
pfm_status true_residual(pfm_handle* h, const double* b, const double* x, double* r) {
  Level& fl = h->L[0];
  cudaStream_t s = h->stream;
  const int64_t n = ndof(fl);
  if (!h->outer_df) {
    TRY(japply_impl<double>(h, x, h->wv));
    launch_sub<double>(n, b, h->wv, r, s);
    CKL();
    return PFM_OK;
  }
  float* xhi = fl.x32;
  float* xlo = fl.r32;
  launch_split_f64(n, x, xhi, xlo, s);
  {
    ProfScope ps(h, PFM_PROF_JAPPLY_F64);
    launch_japply_df(fl.g, h->dp, fl.H32, fl.H32lo, fl.mask, xhi, h->wv, s, det_W<double>(h));
    if (h->contact_on) launch_contact_apply<double, float, double>(fl.g, fl.Kc64, fl.mask, xhi, h->wv, s);
  }
  launch_japply<float>(fl.g, h->dp, fl.H32, fl.mask, xlo, fl.y32, s, det_W<float>(h));
  if (h->contact_on) launch_contact_apply<float, float, float>(fl.g, fl.Kc32, fl.mask, xlo, fl.y32, s);
  launch_sub2(n, b, h->wv, fl.y32, r, s);
  CKL();
  return PFM_OK;
}

// Mixed-precision iterative refinement (GMRES-IR of Carson and Higham, 2018)
// for J x = b, x0 = 0: each step solves J d = r approximately with one cycle
// of FGMRES(m) whose operator is the FP32 tangent (and whose preconditioner is
// the FP32 V-cycle), to max(switch_rtol ||r||, 0.3 lin_rtol ||b||), then
// x += d and r = b - J x with the FP64-class operator, until ||r|| <=
// lin_rtol ||b|| (the true residual, Sec. 3.4) or max_lin_it inner iterations.
pfm_status refine_impl(pfm_handle* h, const pfm_solve_opts& o, const double* b, double* x, int* its_out,
                       double* relres_out, int* outer_out) {
  Level& fl = h->L[0];
  cudaStream_t s = h->stream;
  const int64_t n = ndof(fl);
  if (h->lin_prec != PFM_F32 || !fl.H32 || (h->outer_df && !fl.H32lo))
    return h->fail(PFM_ERR_STATE, "iterative refinement needs a tangent built with pfm_linearize(PFM_F32)");
  TRY(det_ready(h));
  TRY(ensure_level_vectors<float>(h));
  TRY(dalloc(h, &h->ir_r, n));
  TRY(dalloc(h, &h->ir_d, n));
  CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
  double beta0 = 0.0;
  TRY(norm2(h, b, n, &beta0));
  int total = 0, outer = 0;
  double rel = 1.0;
  pfm_status st = PFM_OK;
  if (!std::isfinite(beta0)) {
    st = h->fail(PFM_ERR_NONFINITE, "non-finite right-hand side");
  } else if (beta0 == 0.0) {
    rel = 0.0;
  } else {
    const double tol = o.lin_rtol * beta0;
    const double* r = b;  // r_0 = b - J 0
    for (;;) {
      Fgm F;
      pfm_solve_opts oi = o;
      oi.max_lin_it = o.max_lin_it - total;
      TRY(fgm_begin_enqueue(h, F, oi, r, h->ir_d));
      F.inner = true;
      F.tol_floor = 0.3 * tol;
      CK(cudaStreamSynchronize(s));
      st = fgm_begin_finish(h, F);
      while (st == PFM_OK && !F.done) {
        st = fgm_enqueue(h, F);
        if (st != PFM_OK) break;
        CK(cudaStreamSynchronize(s));
        st = fgm_finish(h, F);
      }
      total += F.total;
      ++outer;
      if (st != PFM_OK) break;
      launch_axpy(n, 1.0, h->ir_d, x, s);
      CKL();
      TRY(true_residual(h, b, x, h->ir_r));
      r = h->ir_r;
      double rn = 0.0;
      TRY(norm2(h, r, n, &rn));
      rel = rn / beta0;
      if (!std::isfinite(rn)) {
        st = h->fail(PFM_ERR_NONFINITE, "non-finite residual in iterative refinement");
        break;
      }
      if (rn <= tol) break;
      if (total >= o.max_lin_it) {
        st = h->fail(PFM_ERR_NOT_CONVERGED,
                     "iterative refinement reached max_lin_it at relative residual " + std::to_string(rel));
        break;
      }
    }
  }
  if (its_out) *its_out = total;
  if (relres_out) *relres_out = rel;
  if (outer_out) *outer_out = outer;
  return st;
}

// Linear solve of the Newton step with the options' method.
pfm_status linear_solve(pfm_handle* h, const pfm_solve_opts& o, const double* b, double* x, int* its_out,
                        double* relres_out, int* outer_out) {
  if (o.krylov == 2 && o.precond == PFM_F32) return refine_impl(h, o, b, x, its_out, relres_out, outer_out);
  return fgmres_impl(h, o, b, x, its_out, relres_out, outer_out);
}

// Capture the V-cycle on the handle's stream into a CUDA graph (once per
// linearisation and smoother configuration) so that a batch replays it with
// one launch per problem and iteration.
template <typename T>
pfm_status capture_vcycle(pfm_handle* h, const SmoothCfg& sc) {
  const int key_prec = sizeof(T) == 4 ? 0 : 1;
  if (h->vgraph && h->vgraph_prec == key_prec && h->vgraph_cfg.nu_pre == sc.nu_pre &&
      h->vgraph_cfg.nu_post == sc.nu_post && h->vgraph_cfg.type == sc.type && h->vgraph_cfg.omega == sc.omega &&
      h->vgraph_cfg.lo == sc.lo && h->vgraph_cfg.hi == sc.hi && h->vgraph_cfg.gamma == sc.gamma &&
      h->vgraph_cfg.growth == sc.growth && h->vgraph_cfg.det == h->det)
    return PFM_OK;
  if (h->vgraph) {
    cudaGraphExecDestroy(h->vgraph);
    h->vgraph = nullptr;
  }
  const bool prof = h->prof;
  h->prof = false;
  CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  pfm_status st = vcycle_level<T>(h, 0, sc);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
  h->prof = prof;
  if (st != PFM_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return h->fail(PFM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&h->vgraph, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    h->vgraph = nullptr;
    return h->fail(PFM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  h->vgraph_prec = key_prec;
  h->vgraph_cfg = {sc.nu_pre, sc.nu_post, sc.type, sc.omega, sc.lo, sc.hi, sc.gamma, sc.growth, h->det};
  return PFM_OK;
}

// opts.deterministic switches the handle's deterministic mode on for one solve
// (a Newton solve linearises inside it, so its coarse operator is assembled
// in the reproducible form too).
struct DetScope {
  pfm_handle* h;
  bool saved;
  DetScope(pfm_handle* h_, const pfm_solve_opts& o) : h(h_), saved(h_->det) {
    if (o.deterministic) h->det = true;
  }
  ~DetScope() {
    if (h) h->det = saved;
  }
  DetScope(const DetScope&) = delete;
  DetScope& operator=(const DetScope&) = delete;
  DetScope(DetScope&& o) noexcept : h(o.h), saved(o.saved) { o.h = nullptr; }
};

bool opts_valid(const pfm_solve_opts& o) {
  return o.restart >= 1 && o.restart <= MAX_RESTART && o.max_lin_it >= 1 && o.nu_pre >= 1 &&
         o.nu_post >= 0 && o.max_newton >= 1 && o.lin_rtol > 0 && o.omega > 0 &&
         (o.precond == PFM_F32 || o.precond == PFM_F64) && (o.smoother == 0 || o.smoother == 1) &&
         o.cheb_lo > 0 && o.cheb_hi > o.cheb_lo && (o.deterministic == 0 || o.deterministic == 1) &&
         (o.krylov == 0 || ((o.krylov == 1 || o.krylov == 2) && o.switch_rtol > 0 && o.switch_rtol < 1));
}

}  // namespace

// ============================================================================
namespace {

// Host-buffer tangent application as a pipeline over z-slabs of elements:
// slab s's input node planes travel host -> device on one copy stream while
// the slab before computes; once slabs <= s are done, the node planes below
// slab s+1 are complete and travel back on a second copy stream. Each copy is
// one transfer per field (field stride nn).
template <typename T>
pfm_status japply_host_pipelined(pfm_handle* h, const void* v_host, void* y_host) {
  Level& f = h->L[0];
  const Grid& g = f.g;
  const T* H = LvVec<T>::H(f);
  if (!H || (sizeof(T) == 4 && h->lin_prec != PFM_F32))
    return h->fail(PFM_ERR_STATE, "no tangent in the requested precision (linearize with PFM_F32 for FP32)");
  if (!h->pipe_in) {
    CK(cudaStreamCreateWithFlags(&h->pipe_in, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&h->pipe_out, cudaStreamNonBlocking));
    for (int k = 0; k < pfm_handle::PIPE_SLABS; ++k) {
      CK(cudaEventCreateWithFlags(&h->pipe_ev_in[k], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&h->pipe_ev_done[k], cudaEventDisableTiming));
    }
    CK(cudaEventCreateWithFlags(&h->pipe_ev_start, cudaEventDisableTiming));
  }
  T* vd = static_cast<T*>(h->stage_in);
  T* yd = static_cast<T*>(h->stage_out);
  const T* vh = static_cast<const T*>(v_host);
  T* yh = static_cast<T*>(y_host);
  const int64_t nn = f.nn, plane = int64_t(g.nx + 1) * (g.ny + 1);
  const int64_t eplane = int64_t(g.nx) * g.ny;  // elements per layer
  const int S = std::min(pfm_handle::PIPE_SLABS, g.nz);
  cudaStream_t sc = h->stream;
  const int blocks = japply_range_blocks();
  // the copy streams start after everything already queued on the compute stream
  CK(cudaEventRecord(h->pipe_ev_start, sc));
  CK(cudaStreamWaitEvent(h->pipe_in, h->pipe_ev_start, 0));
  CK(cudaStreamWaitEvent(h->pipe_out, h->pipe_ev_start, 0));
  CK(cudaMemsetAsync(yd, 0, sizeof(T) * NF * nn, sc));
  int64_t in_done = 0;   // node planes already on the device
  int64_t out_done = 0;  // node planes already returned
  for (int s = 0; s < S; ++s) {
    const int64_t k0 = int64_t(g.nz) * s / S, k1 = int64_t(g.nz) * (s + 1) / S;  // element layers [k0, k1)
    const int64_t need = k1 + 1;                                                   // node planes [0, k1]
    if (need > in_done) {  // node planes [in_done, need) of every field: one 2-D copy
      CK(cudaMemcpy2DAsync(vd + in_done * plane, sizeof(T) * nn, vh + in_done * plane, sizeof(T) * nn,
                           sizeof(T) * (need - in_done) * plane, NF, cudaMemcpyHostToDevice, h->pipe_in));
      in_done = need;
    }
    CK(cudaEventRecord(h->pipe_ev_in[s], h->pipe_in));
    CK(cudaStreamWaitEvent(sc, h->pipe_ev_in[s], 0));
    // element blocks (4 consecutive elements) that start in layers [k0, k1); a
    // block that reaches into layer k1 is left to the next slab, whose input
    // planes it needs
    const int64_t e0 = k0 * eplane, e1 = k1 * eplane;
    const int64_t b0 = e0 / 4, b1 = (s + 1 == S) ? f.nblk : e1 / 4;
    launch_japply_range<T>(g, h->dp, H, f.mask, vd, yd, b0, b1, blocks, sc);
    // node planes [out_done, ready) are final: plane k1 still gets the next
    // slab, and plane k1 - 1 too when a block straddles layers k1 - 1 and k1
    const int64_t ready = (s + 1 == S) ? int64_t(g.nz) + 1 : (eplane % 4 == 0 ? k1 : k1 - 1);
    launch_identity_rows<T>(nn, f.mask, vd, yd, out_done * plane, ready * plane, sc);
    CKL();
    CK(cudaEventRecord(h->pipe_ev_done[s], sc));
    CK(cudaStreamWaitEvent(h->pipe_out, h->pipe_ev_done[s], 0));
    if (ready > out_done) {
      CK(cudaMemcpy2DAsync(yh + out_done * plane, sizeof(T) * nn, yd + out_done * plane, sizeof(T) * nn,
                           sizeof(T) * (ready - out_done) * plane, NF, cudaMemcpyDeviceToHost, h->pipe_out));
      out_done = ready;
    }
  }
  CK(cudaStreamSynchronize(h->pipe_out));
  CK(cudaStreamSynchronize(sc));
  return PFM_OK;
}

}  // namespace

extern "C" {

const char* pfm_version(void) { return "pfm 0.2 (sm_103a)"; }

int pfm_variants(void) { return NV; }

pfm_status pfm_create(const pfm_mesh_desc* mesh, const pfm_params* params, pfm_handle** out) {
  if (!mesh || !params || !out) {
    g_create_error = "null argument";
    return PFM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1 || !(mesh->Lx > 0) || !(mesh->Ly > 0) || !(mesh->Lz > 0) ||
      mesh->n_levels < 0 || !(params->tau > 0) || params->hencky < 0 || params->hencky > 3) {
    g_create_error = "invalid mesh size, box length, level count, tau or Hencky mode";
    return PFM_ERR_INVALID_ARG;
  }
  pfm_handle* h = new pfm_handle();
  h->params = *params;
  make_dev_params(*params, h->dp);
  // level hierarchy: ceil-halving until max(n) <= 4 (or n_levels levels)
  int nx = mesh->nx, ny = mesh->ny, nz = mesh->nz;
  for (int l = 0;; ++l) {
    Level lv;
    lv.g = Grid{nx, ny, nz, mesh->Lx / nx, mesh->Ly / ny, mesh->Lz / nz};
    lv.nn = lv.g.nn();
    lv.ne = lv.g.ne();
    lv.nblk = lv.g.nblk();
    h->L.push_back(lv);
    const int mx = std::max(nx, std::max(ny, nz));
    if (mesh->n_levels > 0 && int(h->L.size()) == mesh->n_levels) break;
    if (mesh->n_levels == 0 && mx <= 4) break;
    if (mx <= 1) break;
    nx = (nx + 1) / 2;
    ny = (ny + 1) / 2;
    nz = (nz + 1) / 2;
  }
  h->nc_dofs = int(NF * h->L.back().nn);
  if (h->nc_dofs > MAX_COARSE_DOFS) {
    g_create_error = "coarsest level has " + std::to_string(h->nc_dofs) + " DOFs (max " +
                     std::to_string(MAX_COARSE_DOFS) + "): use more levels";
    delete h;
    return PFM_ERR_INVALID_ARG;
  }
  auto cleanup = [&](pfm_status st) {
    g_create_error = h->err;
    pfm_destroy(h);
    return st;
  };
  for (auto& lv : h->L) {
    pfm_status st;
    if ((st = dalloc(h, &lv.U, ndof(lv))) != PFM_OK) return cleanup(st);
    if ((st = dalloc(h, &lv.Un, ndof(lv))) != PFM_OK) return cleanup(st);
    if ((st = dalloc(h, &lv.mask, lv.nn)) != PFM_OK) return cleanup(st);
    cudaMemset(lv.mask, 0, sizeof(dmask_t) * lv.nn);
  }
  const int64_t n = ndof(h->L[0]);
  pfm_status st;
  if ((st = dalloc(h, &h->energy_dev, 1)) != PFM_OK) return cleanup(st);
  if ((st = dalloc(h, &h->flag_dev, 1)) != PFM_OK) return cleanup(st);
  if ((st = dalloc(h, &h->diag_part, size_t(h->L[0].g.nz + 1) * DIAG_MAX_CHUNKS * 4)) != PFM_OK) return cleanup(st);
  if ((st = dalloc(h, &h->R, n)) != PFM_OK) return cleanup(st);
  if ((st = dalloc(h, &h->dU, n)) != PFM_OK) return cleanup(st);
  if ((st = dalloc(h, &h->wv, n)) != PFM_OK) return cleanup(st);
  if ((st = dalloc(h, &h->rv, n)) != PFM_OK) return cleanup(st);
  if ((st = dalloc(h, &h->zd, n)) != PFM_OK) return cleanup(st);
  if ((st = dalloc(h, &h->partial, size_t(reduction_blocks(n)) * (MAX_RESTART + 1))) != PFM_OK) return cleanup(st);
  if ((st = dalloc(h, &h->hdev, size_t(3) * (MAX_RESTART + 2))) != PFM_OK) return cleanup(st);
  if ((st = dalloc(h, &h->Kaug, size_t(h->nc_dofs) * 2 * h->nc_dofs)) != PFM_OK) return cleanup(st);
  if ((st = dalloc(h, &h->Kinv, size_t(h->nc_dofs) * h->nc_dofs)) != PFM_OK) return cleanup(st);
  if ((st = dalloc(h, &h->gj_keys, size_t(h->nc_dofs) + 1)) != PFM_OK) return cleanup(st);
  if ((st = dalloc(h, &h->gj_used, h->nc_dofs)) != PFM_OK) return cleanup(st);
  if ((st = dalloc(h, &h->gj_piv, h->nc_dofs)) != PFM_OK) return cleanup(st);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    h->err = cudaGetErrorString(e);
    return cleanup(PFM_ERR_CUDA);
  }
  *out = h;
  return PFM_OK;
}

void pfm_destroy(pfm_handle* h) {
  if (!h) return;
  for (int id = 0; id < PFM_PROF_COUNT; ++id)
    for (auto& e : h->prof_ev[id]) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
  for (auto& lv : h->L) {
    dfree(lv.U); dfree(lv.Un); dfree(lv.mask); dfree(lv.H64); dfree(lv.H32); dfree(lv.H32lo); dfree(lv.H16); dfree(lv.D64);
    dfree(lv.D32);
    dfree(lv.x32); dfree(lv.b32); dfree(lv.y32); dfree(lv.x64); dfree(lv.b64); dfree(lv.y64);
    dfree(lv.r32); dfree(lv.d32); dfree(lv.r64); dfree(lv.d64); dfree(lv.Kc64); dfree(lv.Kc32);
  }
  dfree(h->lz);
  dfree(h->dirval); dfree(h->energy_dev); dfree(h->flag_dev); dfree(h->diag_part); dfree(h->load_dev); dfree(h->R); dfree(h->dU); dfree(h->wv);
  dfree(h->rv); dfree(h->zd); dfree(h->ir_r); dfree(h->ir_d); dfree(h->partial); dfree(h->hdev); dfree(h->V); dfree(h->Kaug); dfree(h->Kinv);
  dfree(h->gj_keys); dfree(h->gj_used); dfree(h->gj_piv); dfree(h->amax_dev);
  if (h->Z) cudaFree(h->Z);
  if (h->vgraph) cudaGraphExecDestroy(h->vgraph);
  if (h->hpin) cudaFreeHost(h->hpin);
  if (h->pipe_in) {
    cudaStreamDestroy(h->pipe_in);
    cudaStreamDestroy(h->pipe_out);
    for (int k = 0; k < pfm_handle::PIPE_SLABS; ++k) {
      cudaEventDestroy(h->pipe_ev_in[k]);
      cudaEventDestroy(h->pipe_ev_done[k]);
    }
    cudaEventDestroy(h->pipe_ev_start);
  }
  if (h->bd_scratch) cudaFree(h->bd_scratch);
  if (h->stage_in) cudaFree(h->stage_in);
  if (h->stage_out) cudaFree(h->stage_out);
  delete h;
}

const char* pfm_last_error(const pfm_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

pfm_status pfm_get_sizes(const pfm_handle* h, int64_t* n_nodes, int64_t* n_elems, int* n_levels) {
  if (!h) return PFM_ERR_INVALID_ARG;
  if (n_nodes) *n_nodes = h->L[0].nn;
  if (n_elems) *n_elems = h->L[0].ne;
  if (n_levels) *n_levels = int(h->L.size());
  return PFM_OK;
}

pfm_status pfm_get_level(const pfm_handle* h, int level, int* nx, int* ny, int* nz, double* lambda_max) {
  if (!h || level < 0 || level >= int(h->L.size())) return PFM_ERR_INVALID_ARG;
  const Level& l = h->L[level];
  if (nx) *nx = l.g.nx;
  if (ny) *ny = l.g.ny;
  if (nz) *nz = l.g.nz;
  if (lambda_max) *lambda_max = l.lam;
  return PFM_OK;
}

pfm_status pfm_set_outer_operator(pfm_handle* h, int double_float) {
  if (!h) return PFM_ERR_INVALID_ARG;
  h->outer_df = double_float != 0;
  return PFM_OK;
}

pfm_status pfm_set_deterministic(pfm_handle* h, int deterministic) {
  if (!h) return PFM_ERR_INVALID_ARG;
  if (deterministic != 0 && deterministic != 1) return h->fail(PFM_ERR_INVALID_ARG, "expected 0 or 1");
  h->det = deterministic != 0;
  return PFM_OK;
}

pfm_status pfm_set_power_iterations(pfm_handle* h, int iterations) {
  if (!h) return PFM_ERR_INVALID_ARG;
  if (iterations < 1 || iterations > 1000) return h->fail(PFM_ERR_INVALID_ARG, "Lanczos steps must be in 1..1000");
  h->power_its = iterations;
  h->linearized = false;
  return PFM_OK;
}

pfm_status pfm_set_stream(pfm_handle* h, void* stream) {
  if (!h) return PFM_ERR_INVALID_ARG;
  h->stream = static_cast<cudaStream_t>(stream);
  return PFM_OK;
}

pfm_status pfm_set_params(pfm_handle* h, const pfm_params* params) {
  if (!h || !params) return PFM_ERR_INVALID_ARG;
  if (!(params->tau > 0)) return h->fail(PFM_ERR_INVALID_ARG, "tau must be positive");
  if (params->hencky < 0 || params->hencky > 3) return h->fail(PFM_ERR_INVALID_ARG, "Hencky mode must be 0..3");
  h->params = *params;
  make_dev_params(*params, h->dp);
  h->linearized = false;
  return PFM_OK;
}

pfm_status pfm_set_dirichlet(pfm_handle* h, const uint8_t* mask_dev, const double* val_dev) {
  if (!h || !mask_dev) return PFM_ERR_INVALID_ARG;
  cudaStream_t s = h->stream;
  Level& f = h->L[0];
  CK(cudaMemsetAsync(h->flag_dev, 0, sizeof(int), s));
  launch_build_mask(f.nn, mask_dev, f.mask, h->flag_dev, s);
  CKL();
  for (size_t l = 1; l < h->L.size(); ++l) launch_coarse_mask(h->L[l - 1].g, h->L[l].g, h->L[l - 1].mask, h->L[l].mask, s);
  CKL();
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, h->flag_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (bad) return h->fail(PFM_ERR_INVALID_ARG, "only displacement DOFs (fields 0..2) may be prescribed");
  if (val_dev) {
    TRY(dalloc(h, &h->dirval, ndof(f)));
    CK(cudaMemcpyAsync(h->dirval, val_dev, sizeof(double) * ndof(f), cudaMemcpyDeviceToDevice, s));
    h->have_dirval = true;
    if (h->have_state) launch_mask_values(f.nn, f.mask, h->dirval, f.U, s);
  }
  h->linearized = false;
  return PFM_OK;
}

pfm_status pfm_set_state(pfm_handle* h, const double* U_dev, const double* Un_dev) {
  if (!h || !U_dev || !Un_dev) return PFM_ERR_INVALID_ARG;
  Level& f = h->L[0];
  cudaStream_t s = h->stream;
  CK(cudaMemcpyAsync(f.U, U_dev, sizeof(double) * ndof(f), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(f.Un, Un_dev, sizeof(double) * ndof(f), cudaMemcpyDeviceToDevice, s));
  if (h->have_dirval) launch_mask_values(f.nn, f.mask, h->dirval, f.U, s);
  CKL();
  h->have_state = true;
  h->linearized = false;
  return PFM_OK;
}

pfm_status pfm_get_state(pfm_handle* h, double* U_dev) {
  TRY(check_ready(h, false));
  if (!U_dev) return h->fail(PFM_ERR_INVALID_ARG, "null output");
  CK(cudaMemcpyAsync(U_dev, h->L[0].U, sizeof(double) * ndof(h->L[0]), cudaMemcpyDeviceToDevice, h->stream));
  return PFM_OK;
}

pfm_status pfm_diagnostics(pfm_handle* h, const double* U_dev, double* Iv_dev, double* Id_dev,
                           double* eta_star_dev, double* plane_stats_dev) {
  if (!h) return PFM_ERR_INVALID_ARG;
  if (!U_dev) {
    TRY(check_ready(h, false));
    U_dev = h->L[0].U;
  }
  const Grid& g = h->L[0].g;
  if (g.nz + 1 > 65535) return h->fail(PFM_ERR_INVALID_ARG, "more than 65535 node planes");
  launch_diagnostics(g, U_dev, Iv_dev, Id_dev, eta_star_dev, h->diag_part, plane_stats_dev, h->stream);
  CKL();
  return PFM_OK;
}

pfm_status pfm_set_linearize_arithmetic(pfm_handle* h, int double_float) {
  if (!h) return PFM_ERR_INVALID_ARG;
  if (double_float != 0 && double_float != 1) return h->fail(PFM_ERR_INVALID_ARG, "expected 0 or 1");
  h->lin_df = double_float != 0;
  h->linearized = false;
  return PFM_OK;
}

pfm_status pfm_set_residual_arithmetic(pfm_handle* h, int double_float) {
  if (!h) return PFM_ERR_INVALID_ARG;
  if (double_float != 0 && double_float != 1) return h->fail(PFM_ERR_INVALID_ARG, "expected 0 or 1");
  h->res_df = double_float != 0;
  return PFM_OK;
}

pfm_status pfm_set_preconditioner_store(pfm_handle* h, int half) {
  if (!h) return PFM_ERR_INVALID_ARG;
  if (half != 0 && half != 1) return h->fail(PFM_ERR_INVALID_ARG, "expected 0 or 1");
  h->pre_h16 = half != 0;
  h->linearized = false;
  if (h->vgraph) {  // may hold launches that read the copies
    cudaGraphExecDestroy(h->vgraph);
    h->vgraph = nullptr;
  }
  for (auto& lv : h->L) {
    lv.h16_scale = 0.f;
    if (!h->pre_h16) dfree(lv.H16);  // cudaFree waits for work still reading it
  }
  return PFM_OK;
}

pfm_status pfm_set_contact(pfm_handle* h, const double* center, double radius, double eps_N) {
  if (!h) return PFM_ERR_INVALID_ARG;
  if (radius <= 0.0) {
    h->contact_on = false;
    h->linearized = false;
    return PFM_OK;
  }
  if (!center || !(eps_N > 0.0) || !std::isfinite(radius) || !std::isfinite(center[0]) ||
      !std::isfinite(center[1]) || !std::isfinite(center[2]))
    return h->fail(PFM_ERR_INVALID_ARG, "contact needs a centre, a positive radius and a positive penalty");
  TRY(dalloc(h, &h->load_dev, 1));
  h->contact = ContactParams{{center[0], center[1], center[2]}, radius, eps_N};
  h->contact_on = true;
  h->linearized = false;
  return PFM_OK;
}

pfm_status pfm_contact_load(pfm_handle* h, double* load_host, double* energy_host) {
  TRY(check_ready(h, false));
  if (!load_host) return h->fail(PFM_ERR_INVALID_ARG, "null output");
  Level& f = h->L[0];
  cudaStream_t s = h->stream;
  double out[2] = {0.0, 0.0};
  if (h->contact_on) {
    CK(cudaMemsetAsync(h->load_dev, 0, sizeof(double), s));
    CK(cudaMemsetAsync(h->energy_dev, 0, sizeof(double), s));
    launch_contact_residual(f.g, h->contact, f.U, f.mask, nullptr, h->energy_dev, h->load_dev, s);
    CKL();
    CK(cudaMemcpyAsync(&out[0], h->load_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&out[1], h->energy_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  *load_host = out[0];
  if (energy_host) *energy_host = out[1];
  return PFM_OK;
}

pfm_status pfm_residual(pfm_handle* h, double* R_dev, double* energy_host) {
  TRY(check_ready(h, false));
  if (!R_dev) return h->fail(PFM_ERR_INVALID_ARG, "null output");
  return residual_impl(h, R_dev, energy_host);
}

pfm_status pfm_linearize(pfm_handle* h, pfm_precision precond) {
  TRY(check_ready(h, false));
  if (precond != PFM_F32 && precond != PFM_F64) return h->fail(PFM_ERR_INVALID_ARG, "bad precision");
  return linearize_impl(h, precond);
}

pfm_status pfm_linearize_residual(pfm_handle* h, pfm_precision precond, double* R_dev, double* energy_host) {
  TRY(check_ready(h, false));
  if (precond != PFM_F32 && precond != PFM_F64) return h->fail(PFM_ERR_INVALID_ARG, "bad precision");
  if (!R_dev) return h->fail(PFM_ERR_INVALID_ARG, "null output");
  if (!residual_fusable(h)) {
    TRY(residual_impl(h, R_dev, energy_host));
    return linearize_impl(h, precond);
  }
  TRY(linearize_impl(h, precond, R_dev));
  if (energy_host) {
    CK(cudaMemcpyAsync(energy_host, h->energy_dev, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  return PFM_OK;
}

pfm_status pfm_jacobian_apply(pfm_handle* h, const void* v_dev, void* y_dev, pfm_precision prec) {
  TRY(check_ready(h, true));
  if (!v_dev || !y_dev || v_dev == y_dev) return h->fail(PFM_ERR_INVALID_ARG, "null or aliased vectors");
  if (prec == PFM_F32) return japply_impl<float>(h, static_cast<const float*>(v_dev), static_cast<float*>(y_dev));
  if (prec == PFM_F64) return japply_impl<double>(h, static_cast<const double*>(v_dev), static_cast<double*>(y_dev));
  return h->fail(PFM_ERR_INVALID_ARG, "bad precision");
}

// The tangent is the Hessian of one scalar potential (Sec. 3.4), so every
// stored 15x15 point block is symmetric and packed once; J^T v reads the
// same packed blocks with the roles of rows and columns exchanged, which is
// the same product. Dirichlet rows and columns are identity in both.
pfm_status pfm_jacobian_transpose_apply(pfm_handle* h, const void* v_dev, void* y_dev, pfm_precision prec) {
  return pfm_jacobian_apply(h, v_dev, y_dev, prec);
}

pfm_status pfm_jacobian_apply_mixed(pfm_handle* h, const float* v_dev, double* y_dev) {
  TRY(check_ready(h, true));
  if (!v_dev || !y_dev) return h->fail(PFM_ERR_INVALID_ARG, "null vectors");
  Level& f = h->L[0];
  if (h->lin_prec != PFM_F32 || !f.H32 || !f.H32lo)
    return h->fail(PFM_ERR_STATE, "the mixed product needs a tangent built with pfm_linearize(PFM_F32)");
  TRY(det_ready(h));
  {
    ProfScope ps(h, PFM_PROF_JAPPLY_F64);
    launch_japply_df(f.g, h->dp, f.H32, f.H32lo, f.mask, v_dev, y_dev, h->stream, det_W<double>(h));
    if (h->contact_on)
      launch_contact_apply<double, float, double>(f.g, f.Kc64, f.mask, static_cast<const float*>(v_dev),
                                                  static_cast<double*>(y_dev), h->stream);
  }
  CKL();
  return PFM_OK;
}

pfm_status pfm_jacobian_apply_host(pfm_handle* h, const void* v_host, void* y_host, pfm_precision prec) {
  TRY(check_ready(h, true));
  if (!v_host || !y_host) return h->fail(PFM_ERR_INVALID_ARG, "null vectors");
  const size_t bytes = ndof(h->L[0]) * (prec == PFM_F32 ? sizeof(float) : sizeof(double));
  if (!h->stage_in) {
    char* a = nullptr;
    char* b = nullptr;
    TRY(dalloc(h, &a, ndof(h->L[0]) * sizeof(double)));
    TRY(dalloc(h, &b, ndof(h->L[0]) * sizeof(double)));
    h->stage_in = a;
    h->stage_out = b;
  }
  if (!h->contact_on && !h->det && (prec == PFM_F32 || prec == PFM_F64)) {
    if (prec == PFM_F32) return japply_host_pipelined<float>(h, v_host, y_host);
    return japply_host_pipelined<double>(h, v_host, y_host);
  }
  CK(cudaMemcpyAsync(h->stage_in, v_host, bytes, cudaMemcpyHostToDevice, h->stream));
  TRY(pfm_jacobian_apply(h, h->stage_in, h->stage_out, prec));
  CK(cudaMemcpyAsync(y_host, h->stage_out, bytes, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return PFM_OK;
}

pfm_status pfm_vcycle(pfm_handle* h, const void* r_dev, void* z_dev, pfm_precision prec, const pfm_solve_opts* opts) {
  TRY(check_ready(h, true));
  if (!r_dev || !z_dev) return h->fail(PFM_ERR_INVALID_ARG, "null vectors");
  const SmoothCfg c = smooth_cfg(opts);
  if (c.nu_pre < 1 || c.nu_post < 0 || (c.type != 0 && c.type != 1) || !(c.hi > c.lo) || !(c.lo > 0))
    return h->fail(PFM_ERR_INVALID_ARG, "bad smoother options");
  if (prec != h->lin_prec) return h->fail(PFM_ERR_STATE, "V-cycle precision differs from the linearisation");
  if (prec == PFM_F32) return apply_vcycle<float>(h, static_cast<const float*>(r_dev), static_cast<float*>(z_dev), c);
  return apply_vcycle<double>(h, static_cast<const double*>(r_dev), static_cast<double*>(z_dev), c);
}

pfm_status pfm_fgmres_solve(pfm_handle* h, const pfm_solve_opts* opts, const double* b_dev, double* x_dev,
                            pfm_solve_report* report) {
  TRY(check_ready(h, true));
  if (!opts || !b_dev || !x_dev || !opts_valid(*opts)) return h->fail(PFM_ERR_INVALID_ARG, "bad options or vectors");
  int its = 0;
  double rel = 0.0;
  double t0 = now_ms();
  DetScope ds(h, *opts);
  int outer = 0;
  pfm_status st = linear_solve(h, *opts, b_dev, x_dev, &its, &rel, &outer);
  if (report) {
    report->lin_outer_last = outer;
    report->lin_its_last = its;
    report->lin_its_total = its;
    report->lin_res_final = rel;
    report->ms_solve = now_ms() - t0;
    report->status = st;
  }
  return st;
}

pfm_status pfm_newton_solve(pfm_handle* h, const pfm_solve_opts* opts, double* U_inout_dev, pfm_solve_report* report) {
  if (!h) return PFM_ERR_INVALID_ARG;
  if (!opts || !U_inout_dev || !opts_valid(*opts)) return h->fail(PFM_ERR_INVALID_ARG, "bad options or state");
  if (!h->have_state) return h->fail(PFM_ERR_STATE, "no U_n: call pfm_set_state first");
  Level& f = h->L[0];
  cudaStream_t s = h->stream;
  const int64_t n = ndof(f);
  pfm_solve_report rep{};
  const double t_start = now_ms();
  DetScope ds(h, *opts);
  CK(cudaMemcpyAsync(f.U, U_inout_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  if (h->have_dirval) launch_mask_values(f.nn, f.mask, h->dirval, f.U, s);
  h->linearized = false;
  double t0 = now_ms();
  // The first iteration linearises at the starting state whatever its
  // residual (only a zero residual ends the solve before it), so that
  // residual comes out of the linearisation pass (Sec. 3.4: both evaluate the
  // point physics of the same state).
  const bool fused = opts->max_newton > 0 && residual_fusable(h);
  double res = 0.0;
  pfm_status st = PFM_OK;
  if (fused) {
    st = linearize_impl(h, opts->precond, h->R);
    rep.ms_linearize += now_ms() - t0;
    TRY(norm2(h, h->R, n, &res));
    if (st != PFM_OK && (res == 0.0 || !std::isfinite(res))) {
      // a failed linearisation of a state with a zero or non-finite residual
      // reports what the residual says
      h->linearized = false;
      st = PFM_OK;
    }
  } else {
    TRY(residual_impl(h, h->R, nullptr));
    TRY(norm2(h, h->R, n, &res));
    rep.ms_residual += now_ms() - t0;
  }
  rep.res0 = res;
  if (st == PFM_OK && !std::isfinite(res)) st = h->fail(PFM_ERR_NONFINITE, "non-finite residual");
  for (int it = 0; st == PFM_OK && it < opts->max_newton; ++it) {
    if (res == 0.0 || (it > 0 && res <= opts->newton_rtol * rep.res0)) break;
    if (!(fused && it == 0)) {
      t0 = now_ms();
      st = linearize_impl(h, opts->precond);
      rep.ms_linearize += now_ms() - t0;
    }
    if (st != PFM_OK) break;
    // J dU = b with b = -R (R negated in place; the solver uses wv/rv/zd as work)
    t0 = now_ms();
    int its = 0;
    double rel = 0.0;
    launch_axpy(n, -2.0, h->R, h->R, s);
    int outer = 0;
    st = linear_solve(h, *opts, h->R, h->dU, &its, &rel, &outer);
    rep.lin_outer_last = outer;
    rep.ms_solve += now_ms() - t0;
    rep.lin_its_total += its;
    rep.lin_its_last = its;
    rep.lin_res_final = rel;
    if (st != PFM_OK) break;
    launch_axpy(n, 1.0, h->dU, f.U, s);
    CKL();
    h->linearized = false;
    ++rep.newton_its;
    t0 = now_ms();
    TRY(residual_impl(h, h->R, nullptr));
    TRY(norm2(h, h->R, n, &res));
    rep.ms_residual += now_ms() - t0;
    if (!std::isfinite(res)) st = h->fail(PFM_ERR_NONFINITE, "non-finite residual");
  }
  rep.res_final = res;
  if (st == PFM_OK && opts->max_newton > 1 && !(res <= opts->newton_rtol * rep.res0) && res != 0.0)
    st = h->fail(PFM_ERR_NOT_CONVERGED, "Newton reached max_newton");
  CK(cudaMemcpyAsync(U_inout_dev, f.U, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  rep.ms_total = now_ms() - t_start;
  rep.status = st;
  if (report) *report = rep;
  return st;
}

pfm_status pfm_param_grad(pfm_handle* h, const double* w_dev, double* dPi, double* wdR, double* dR_dev) {
  TRY(check_ready(h, false));
  const pfm_params& p = h->params;
  // the stiffness must be one cubic matrix shared by every phase
  const double* L0 = p.Lvoigt[0];
  auto at = [&](const double* L, int i, int j) { return L[6 * i + j]; };
  for (int ph = 0; ph < NPH; ++ph)
    for (int k = 0; k < 36; ++k)
      if (p.Lvoigt[ph][k] != L0[k]) return h->fail(PFM_ERR_INVALID_ARG, "stiffness differs between phases");
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double expect;
      if (i < 3 && j < 3) expect = (i == j) ? at(L0, 0, 0) : at(L0, 0, 1);
      else expect = (i == j) ? at(L0, 3, 3) : 0.0;
      if (at(L0, i, j) != expect) return h->fail(PFM_ERR_INVALID_ARG, "stiffness is not cubic");
    }
  Level& f = h->L[0];
  cudaStream_t s = h->stream;
  const int64_t n = ndof(f);
  double* Rk = h->wv;  // work vector
  for (int k = 0; k < 4; ++k) {
    // the theta_k-part of the potential: unit C11 / C12 / C44 stiffness with
    // every other term off, or the interface terms alone at s_gamma = 1
    pfm_params q = p;
    for (int ph = 0; ph < NPH; ++ph) {
      for (int m = 0; m < 36; ++m) q.Lvoigt[ph][m] = 0.0;
      q.F0[ph] = 0.0;
    }
    q.eps_eta = 0.0;
    DevParams dq;
    if (k < 3) {
      for (int ph = 0; ph < NPH; ++ph)
        for (int i = 0; i < 6; ++i)
          for (int j = 0; j < 6; ++j) {
            double v = 0.0;
            if (k == 0 && i < 3 && i == j) v = 1.0;
            if (k == 1 && i < 3 && j < 3 && i != j) v = 1.0;
            if (k == 2 && i >= 3 && i == j) v = 1.0;
            q.Lvoigt[ph][6 * i + j] = v;
          }
      q.gamma_scale = 0.0;
    } else {
      q.gamma_scale = 1.0;
    }
    make_dev_params(q, dq);
    for (int ph = 0; ph < NPH; ++ph) dq.inv_mtau[ph] = 0.0;  // no dissipation
    if (dR_dev) Rk = dR_dev + int64_t(k) * n;
    CK(cudaMemsetAsync(Rk, 0, sizeof(double) * n, s));
    CK(cudaMemsetAsync(h->energy_dev, 0, sizeof(double), s));
    TRY(det_ready(h));
    launch_residual(f.g, dq, f.U, f.Un, f.mask, Rk, h->energy_dev, s, det_W<double>(h));
    CKL();
    double e = 0.0;
    CK(cudaMemcpyAsync(&e, h->energy_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (w_dev) {
      launch_dot<double>(n, w_dev, Rk, h->partial, h->hdev, s);
      double d = 0.0;
      CK(cudaMemcpyAsync(&d, h->hdev, sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (wdR) wdR[k] = d;
    }
    CK(cudaStreamSynchronize(s));
    // the gamma part scales with s_gamma: derivative = (interface energy at s=1)
    if (dPi) dPi[k] = e;
  }
  return PFM_OK;
}

pfm_status pfm_qp_eval(pfm_handle* h, int64_t n, const double* F_dev, const double* eta_dev, const double* eta_n_dev,
                       double* W_dev, double* grad_dev, double* hess_dev) {
  if (!h) return PFM_ERR_INVALID_ARG;
  if (n < 0 || !F_dev || !eta_dev || !eta_n_dev) return h->fail(PFM_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return PFM_OK;
  launch_qp_eval(h->dp, n, F_dev, eta_dev, eta_n_dev, W_dev, grad_dev, hess_dev, h->stream);
  CKL();
  CK(cudaStreamSynchronize(h->stream));
  return PFM_OK;
}

pfm_status pfm_get_hessians(pfm_handle* h, int64_t e0, int64_t count, double* hess_host) {
  TRY(check_ready(h, true));
  Level& f = h->L[0];
  if (e0 < 0 || count < 0 || e0 + count > f.ne || (!hess_host && count > 0))
    return h->fail(PFM_ERR_INVALID_ARG, "element range out of bounds");
  if (count == 0) return PFM_OK;
  const int64_t b0 = e0 / 4, b1 = (e0 + count - 1) / 4;
  std::vector<double> buf(size_t(b1 - b0 + 1) * HBLK);
  CK(cudaMemcpyAsync(buf.data(), f.H64 + b0 * HBLK, sizeof(double) * buf.size(), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int64_t e = e0; e < e0 + count; ++e)
    for (int q = 0; q < 8; ++q) {
      const int lane = int(e & 3) * 8 + q;
      for (int j = 0; j < NH; ++j)
        hess_host[((e - e0) * 8 + q) * NH + j] = buf[hstore_offset<double>(e / 4 - b0, j, lane)];
    }
  return PFM_OK;
}

pfm_status pfm_get_block_inverses(pfm_handle* h, int level, int64_t n0, int64_t count, double* inv_host) {
  TRY(check_ready(h, true));
  if (level < 0 || level + 1 >= int(h->L.size()))
    return h->fail(PFM_ERR_INVALID_ARG, "level out of range (the coarsest level has no block inverses)");
  Level& lv = h->L[level];
  if (n0 < 0 || count < 0 || n0 + count > lv.nn || (!inv_host && count > 0))
    return h->fail(PFM_ERR_INVALID_ARG, "node range out of bounds");
  if (count == 0) return PFM_OK;
  const bool f32 = h->lin_prec == PFM_F32;
  if ((f32 && !lv.D32) || (!f32 && !lv.D64)) return h->fail(PFM_ERR_STATE, "no block inverses on this level");
  std::vector<double> buf(size_t(NF2) * count);
  std::vector<float> b32(f32 ? size_t(count) : 0);
  for (int e = 0; e < NF2; ++e) {
    if (f32) {
      CK(cudaMemcpyAsync(b32.data(), lv.D32 + int64_t(e) * lv.nn + n0, sizeof(float) * count,
                         cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      for (int64_t i = 0; i < count; ++i) buf[size_t(e) * count + i] = b32[i];
    } else {
      CK(cudaMemcpyAsync(buf.data() + size_t(e) * count, lv.D64 + int64_t(e) * lv.nn + n0, sizeof(double) * count,
                         cudaMemcpyDeviceToHost, h->stream));
    }
  }
  CK(cudaStreamSynchronize(h->stream));
  for (int64_t i = 0; i < count; ++i)
    for (int e = 0; e < NF2; ++e) inv_host[i * NF2 + e] = buf[size_t(e) * count + i];
  return PFM_OK;
}

pfm_status pfm_profile_enable(pfm_handle* h, int enable) {
  if (!h) return PFM_ERR_INVALID_ARG;
  prof_collect(h);
  for (int id = 0; id < PFM_PROF_COUNT; ++id) { h->prof_n[id] = 0; h->prof_ms[id] = 0.0; }
  h->prof = enable != 0;
  return PFM_OK;
}

pfm_status pfm_profile_get(pfm_handle* h, int id, int64_t* launches, double* total_ms) {
  if (!h || id < 0 || id >= PFM_PROF_COUNT) return PFM_ERR_INVALID_ARG;
  prof_collect(h);
  if (launches) *launches = h->prof_n[id];
  if (total_ms) *total_ms = h->prof_ms[id];
  return PFM_OK;
}

int64_t pfm_launch_count(void) { return g_launches.load(); }

pfm_status pfm_arith_peak(int precision, double* tflops) {
  if (!tflops || (precision != PFM_F32 && precision != PFM_F64)) return PFM_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PFM_ERR_CUDA;
  const int blocks = sms * 8, threads = 256;
  const int iters = precision == PFM_F32 ? 1 << 16 : 1 << 11;
  const size_t bytes = size_t(blocks) * threads * 8;
  void* out = nullptr;
  if (cudaMalloc(&out, bytes) != cudaSuccess) return PFM_ERR_OOM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {  // the first run is a warm-up
    cudaEventRecord(e0);
    if (precision == PFM_F32)
      k_fma_peak<float><<<blocks, threads>>>(iters, 0.999f, 1e-3f, static_cast<float*>(out));
    else
      k_fma_peak<double><<<blocks, threads>>>(iters, 0.999, 1e-3, static_cast<double*>(out));
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  pfm::count_launches(4);
  const cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return PFM_ERR_CUDA;
  *tflops = 2.0 * 8.0 * double(iters) * double(blocks) * threads / (double(best) * 1e-3) / 1e12;
  return PFM_OK;
}

}  // extern "C"

// ============================================================================
// Batch of independent problems (uneven sizes), advanced in lockstep.


namespace {
std::string g_batch_create_error;

// Enqueue the residual of every listed problem and ||R||^2 into its pinned
// slot hpin[0]; synchronise all their streams once; return the norms.
pfm_status batch_residual_norms(pfm_batch* b, const std::vector<int>& ids, std::vector<double>& res) {
  for (int p : ids) {
    pfm_handle* h = b->hs[p];
    TRY(residual_impl(h, h->R, nullptr));
    const int64_t n = ndof(h->L[0]);
    launch_mdot(n, 1, h->R, 0, h->R, h->partial, h->hdev, h->stream);
    CKL();
    if (!h->hpin) CK(cudaMallocHost(reinterpret_cast<void**>(&h->hpin), sizeof(double) * (2 * (MAX_RESTART + 1) + 2)));
    CK(cudaMemcpyAsync(h->hpin, h->hdev, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  }
  for (int p : ids) {
    pfm_handle* h = b->hs[p];
    CK(cudaStreamSynchronize(h->stream));
    res[p] = std::sqrt(h->hpin[0]);
  }
  return PFM_OK;
}
}  // namespace

extern "C" {

pfm_status pfm_batch_create(pfm_handle* const* handles, int count, pfm_batch** out) {
  if (!handles || count < 1 || !out) {
    g_batch_create_error = "null handles or non-positive count";
    return PFM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  pfm_batch* b = new pfm_batch();
  for (int p = 0; p < count; ++p) {
    if (!handles[p]) {
      g_batch_create_error = "null handle in the batch";
      delete b;
      return PFM_ERR_INVALID_ARG;
    }
    b->hs.push_back(handles[p]);
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      g_batch_create_error = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
      for (auto x : b->streams) cudaStreamDestroy(x);
      delete b;
      return PFM_ERR_CUDA;
    }
    b->streams.push_back(st);
  }
  *out = b;
  return PFM_OK;
}

void pfm_batch_destroy(pfm_batch* b) {
  if (!b) return;
  if (b->engine) {
    cudaDeviceSynchronize();
    batch_engine_free(b->engine);
  }
  for (auto x : b->streams) cudaStreamDestroy(x);
  delete b;
}

const char* pfm_batch_last_error(const pfm_batch* b) { return b ? b->err.c_str() : g_batch_create_error.c_str(); }

pfm_status pfm_batch_set_mode(pfm_batch* b, int mode) {
  if (!b) return PFM_ERR_INVALID_ARG;
  if (mode != 0 && mode != 1) return b->fail(PFM_ERR_INVALID_ARG, "batch mode must be 0 or 1");
  b->mode = mode;
  return PFM_OK;
}

pfm_status pfm_batch_newton_solve(pfm_batch* b, const pfm_solve_opts* opts, double* const* U_inout,
                                  pfm_solve_report* reports) {
  if (!b) return PFM_ERR_INVALID_ARG;
  if (!opts || !U_inout || !opts_valid(*opts)) return b->fail(PFM_ERR_INVALID_ARG, "bad options or state arrays");
  if (opts->krylov == 2) return b->fail(PFM_ERR_INVALID_ARG, "batches run krylov modes 0 and 1");
  const int N = int(b->hs.size());
  for (int p = 0; p < N; ++p) {
    if (!b->hs[p]->have_state) return b->fail(PFM_ERR_STATE, "problem " + std::to_string(p) + " has no U_n");
    if (!U_inout[p]) return b->fail(PFM_ERR_INVALID_ARG, "null state of problem " + std::to_string(p));
  }
  if (b->mode == 0 && batch_engine_supports(*opts, b)) return batch_engine_newton(b, *opts, U_inout, reports);
  std::vector<cudaStream_t> saved(N);
  std::vector<DetScope> dets;
  dets.reserve(N);
  for (int p = 0; p < N; ++p) {
    pfm_handle* h = b->hs[p];
    if (!h->have_state) return b->fail(PFM_ERR_STATE, "problem " + std::to_string(p) + " has no U_n");
    if (!U_inout[p]) return b->fail(PFM_ERR_INVALID_ARG, "null state of problem " + std::to_string(p));
    saved[p] = h->stream;
    h->stream = b->streams[p];
    h->use_graphs = true;
    dets.emplace_back(h, *opts);
  }
  std::vector<pfm_solve_report> rep(N);
  std::vector<double> res(N, 0.0);
  std::vector<int> all(N);
  pfm_status st = PFM_OK;
  const double t_start = now_ms();
  auto restore = [&]() {
    for (int p = 0; p < N; ++p) {
      pfm_handle* h = b->hs[p];
      cudaStreamSynchronize(h->stream);
      h->use_graphs = false;
      h->stream = saved[p];
    }
  };
  for (int p = 0; p < N; ++p) {
    all[p] = p;
    pfm_handle* h = b->hs[p];
    Level& f = h->L[0];
    if (cudaMemcpyAsync(f.U, U_inout[p], sizeof(double) * ndof(f), cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess) {
      restore();
      return b->fail(PFM_ERR_CUDA, "state copy failed");
    }
    if (h->have_dirval) launch_mask_values(f.nn, f.mask, h->dirval, f.U, h->stream);
    h->linearized = false;
  }
  double t0 = now_ms();
  st = batch_residual_norms(b, all, res);
  for (int p = 0; p < N; ++p) {
    rep[p].res0 = res[p];
    rep[p].ms_residual += now_ms() - t0;
  }
  for (int it = 0; st == PFM_OK && it < opts->max_newton; ++it) {
    std::vector<int> act;
    for (int p = 0; p < N; ++p) {
      if (!std::isfinite(res[p])) {
        rep[p].status = PFM_ERR_NONFINITE;
        continue;
      }
      if (res[p] == 0.0 || (it > 0 && res[p] <= opts->newton_rtol * rep[p].res0)) continue;
      act.push_back(p);
    }
    if (act.empty()) break;
    t0 = now_ms();
    for (int p : act) {
      st = linearize_impl(b->hs[p], opts->precond);
      if (st != PFM_OK) {
        b->err = "problem " + std::to_string(p) + ": " + b->hs[p]->err;
        break;
      }
    }
    const double ms_lin = now_ms() - t0;
    if (st != PFM_OK) break;
    t0 = now_ms();
    // lockstep FGMRES over the active problems (b = -R kept in R)
    std::vector<Fgm> F(N);
    for (int p : act) {
      pfm_handle* h = b->hs[p];
      launch_axpy(ndof(h->L[0]), -2.0, h->R, h->R, h->stream);
      st = fgm_begin_enqueue(h, F[p], *opts, h->R, h->dU);
      if (st != PFM_OK) break;
    }
    if (st != PFM_OK) break;
    std::vector<int> live;
    for (int p : act) {
      pfm_handle* h = b->hs[p];
      cudaStreamSynchronize(h->stream);
      st = fgm_begin_finish(h, F[p]);
      if (st != PFM_OK) break;
      if (!F[p].done) live.push_back(p);
    }
    while (st == PFM_OK && !live.empty()) {
      for (int p : live)
        if ((st = fgm_enqueue(b->hs[p], F[p])) != PFM_OK) break;
      if (st != PFM_OK) break;
      for (int p : live) cudaStreamSynchronize(b->hs[p]->stream);
      std::vector<int> next;
      for (int p : live) {
        pfm_status fs = fgm_finish(b->hs[p], F[p]);
        if (fs != PFM_OK && fs != PFM_ERR_NOT_CONVERGED) {
          st = fs;
          b->err = "problem " + std::to_string(p) + ": " + b->hs[p]->err;
          break;
        }
        if (!F[p].done) next.push_back(p);
      }
      live.swap(next);
    }
    const double ms_solve = now_ms() - t0;
    if (st != PFM_OK) break;
    for (int p : act) {
      pfm_handle* h = b->hs[p];
      rep[p].ms_linearize += ms_lin;
      rep[p].ms_solve += ms_solve;
      rep[p].lin_its_total += F[p].total;
      rep[p].lin_its_last = F[p].total;
      rep[p].lin_res_final = F[p].relres;
      if (!F[p].converged) rep[p].status = PFM_ERR_NOT_CONVERGED;
      launch_axpy(ndof(h->L[0]), 1.0, h->dU, h->L[0].U, h->stream);
      h->linearized = false;
      ++rep[p].newton_its;
    }
    t0 = now_ms();
    st = batch_residual_norms(b, act, res);
    for (int p : act) rep[p].ms_residual += now_ms() - t0;
  }
  for (int p = 0; p < N; ++p) {
    pfm_handle* h = b->hs[p];
    cudaMemcpyAsync(U_inout[p], h->L[0].U, sizeof(double) * ndof(h->L[0]), cudaMemcpyDeviceToDevice, h->stream);
    rep[p].res_final = res[p];
    if (rep[p].status == PFM_OK && opts->max_newton > 1 && !(res[p] <= opts->newton_rtol * rep[p].res0) && res[p] != 0.0)
      rep[p].status = PFM_ERR_NOT_CONVERGED;
  }
  restore();
  const double total = now_ms() - t_start;
  for (int p = 0; p < N; ++p) {
    rep[p].ms_total = total;
    if (st != PFM_OK && rep[p].status == PFM_OK) rep[p].status = st;
    if (reports) reports[p] = rep[p];
  }
  if (st != PFM_OK) return st;
  for (int p = 0; p < N; ++p)
    if (rep[p].status != PFM_OK) {
      b->err = "problem " + std::to_string(p) + " did not converge";
      return rep[p].status;
    }
  return PFM_OK;
}

}  // extern "C"
