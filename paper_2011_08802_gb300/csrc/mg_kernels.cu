// Geometric-multigrid kernels (Sec. 3.4): state injection to coarse levels
// for re-discretisation, trilinear prolongation P and restriction R = P^T
// between nested or non-nested structured grids on the same box, the damped
// point-block Jacobi update, and the dense coarse-level operator with its
// inverse by Gauss-Jordan elimination with partial pivoting.
//
// Grid transfer in 1-D: fine node i sits at coarse coordinate i*nc/nf; with
// i*nc = I0*nf + rem, its interpolation weights are (1 - rem/nf) on coarse
// node I0 and rem/nf on I0+1. All index arithmetic is integer, so P and
// R = P^T use identical weights on nested (nf = 2 nc) and non-nested grids.
#include "common.cuh"
#include "mg_device.cuh"

namespace pfm {
namespace {

inline unsigned grid_for(int64_t threads, int block) {
  int64_t b = (threads + block - 1) / block;
  return unsigned(b > 0 ? b : 1);
}

// Coarse state = fine Q1 field evaluated at coarse node positions.
__global__ void k_inject_state(Grid f, Grid c, const double* __restrict__ Uf, double* __restrict__ Uc) {
  const int64_t nnc = c.nn();
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < nnc;
       idx += int64_t(gridDim.x) * blockDim.x)
    inject_node(f, c, Uf, Uc, idx);
}

// Coarse Dirichlet bits = bits of the nearest fine node.
__global__ void k_coarse_mask(Grid f, Grid c, const dmask_t* __restrict__ mf, dmask_t* __restrict__ mc) {
  const int64_t nnc = c.nn();
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < nnc;
       idx += int64_t(gridDim.x) * blockDim.x) {
    int I = int(idx % (c.nx + 1));
    int J = int((idx / (c.nx + 1)) % (c.ny + 1));
    int K = int(idx / (int64_t(c.nx + 1) * (c.ny + 1)));
    auto nearest = [](int Ic, int nc, int nf) { return int((2LL * Ic * nf + nc) / (2LL * nc)); };
    int i = nearest(I, c.nx, f.nx), j = nearest(J, c.ny, f.ny), k = nearest(K, c.nz, f.nz);
    mc[idx] = mf[i + int64_t(f.nx + 1) * (j + int64_t(f.ny + 1) * k)];
  }
}

// xf += P xc at free fine DOFs.
template <typename T>
__global__ void k_prolong_add(Grid f, Grid c, const T* __restrict__ xc, const dmask_t* __restrict__ mf,
                              T* __restrict__ xf) {
  const int64_t nnf = f.nn();
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < nnf;
       idx += int64_t(gridDim.x) * blockDim.x)
    prolong_node<T>(f, c, xc, mf, xf, idx);
}

// Nested grids: one thread per fine node (i over x-blocks and threads, j and
// k over the grid's y and z dimensions, so no index division).
template <typename T>
__global__ void __launch_bounds__(128) k_prolong_add_nested(Grid f, Grid c, const T* __restrict__ xc,
                                                            const dmask_t* __restrict__ mf, T* __restrict__ xf) {
  const int i = int(blockIdx.x * blockDim.x + threadIdx.x);
  if (i > f.nx) return;
  prolong_node_nested<T>(f, c, xc, mf, xf, i, int(blockIdx.y), int(blockIdx.z));
}

// Nested grids: one thread per coarse node.
template <typename T>
__global__ void __launch_bounds__(128) k_restrict_nested(Grid f, Grid c, const T* __restrict__ rf,
                                                         const dmask_t* __restrict__ mc, T* __restrict__ rc) {
  const int I = int(blockIdx.x * blockDim.x + threadIdx.x);
  if (I > c.nx) return;
  restrict_node_nested<T>(f, c, rf, mc, rc, I, int(blockIdx.y), int(blockIdx.z));
}

// rc = P^T rf, zero at coarse Dirichlet DOFs.
template <typename T>
__global__ void k_restrict(Grid f, Grid c, const T* __restrict__ rf, const dmask_t* __restrict__ mc,
                           T* __restrict__ rc) {
  const int64_t nnc = c.nn();
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < nnc;
       idx += int64_t(gridDim.x) * blockDim.x)
    restrict_node<T>(f, c, rf, mc, rc, idx);
}

// x += omega D^-1 (b - y) per node (y == nullptr: y = 0).
template <typename T>
__global__ void k_smooth(int64_t nn, const T* __restrict__ D, const T* __restrict__ b,
                         const T* __restrict__ y, T omega, T* __restrict__ x) {
  for (int64_t node = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; node < nn;
       node += int64_t(gridDim.x) * blockDim.x) {
    T r[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) r[f] = b[f * nn + node] - (y ? y[f * nn + node] : T(0));
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      T s = T(0);
#pragma unroll
      for (int c = 0; c < NF; ++c) s += D[(f * NF + c) * nn + node] * r[c];
      x[f * nn + node] += omega * s;
    }
  }
}

template <typename T>
__global__ void k_sub(int64_t n, const T* __restrict__ b, const T* __restrict__ y, T* __restrict__ r) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    r[i] = b[i] - y[i];
}

// Dense coarse operator K (row-major, leading dimension ld) from the stored
// point Hessians: thread (element, local row l = f*8 + a) adds row l of the
// element matrix sum_q w (Bz^T H_q Bz + Bg^T G Bg). color < 0: every element,
// added with atomics; color = 0..7: only the elements with
// (ei & 1) + 2 (ej & 1) + 4 (ek & 1) == color, which share no node, added
// without atomics (eight launches in colour order give a fixed summation order).
template <typename T>
__global__ void k_coarse_assemble(Grid g, DevParams P, const T* __restrict__ H, double* __restrict__ K,
                                  int ld, int color) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t e = tid / NED;
  if (e >= g.ne()) return;
  if (color >= 0) {
    const int64_t ei = e % g.nx, ej = (e / g.nx) % g.ny, ek = e / (int64_t(g.nx) * g.ny);
    if (int((ei & 1) + 2 * (ej & 1) + 4 * (ek & 1)) != color) return;
  }
  const int l = int(tid % NED);
  const int fl = l / 8, al = l % 8;
  const int64_t nn = g.nn();
  const double ih[3] = {1.0 / g.hx, 1.0 / g.hy, 1.0 / g.hz};
  const double w = g.w();
  auto node_of = [&](int a) {
    int64_t ei = e % g.nx, r = e / g.nx, ej = r % g.ny, ek = r / g.ny;
    return (ei + (a & 1)) + int64_t(g.nx + 1) * ((ej + ((a >> 1) & 1)) + int64_t(g.ny + 1) * (ek + (a >> 2)));
  };
  auto shape = [&](int a, int q, double& N, double dN[3]) {
    double phi[3], dphi[3];
    for (int d = 0; d < 3; ++d) {
      const int ad = (a >> d) & 1, qd = (q >> d) & 1;
      phi[d] = (ad == qd) ? GB : GA;
      dphi[d] = (ad ? 1.0 : -1.0) * ih[d];
    }
    N = phi[0] * phi[1] * phi[2];
    dN[0] = dphi[0] * phi[1] * phi[2];
    dN[1] = phi[0] * dphi[1] * phi[2];
    dN[2] = phi[0] * phi[1] * dphi[2];
  };
  const int64_t row = fl * nn + node_of(al);
  const int64_t blk = e >> 2;
  const int lane0 = int(e & 3) * 8;
  for (int m = 0; m < NED; ++m) {
    const int fm = m / 8, am = m % 8;
    double s = 0.0;
    for (int q = 0; q < 8; ++q) {
      double Nl, dNl[3], Nm, dNm[3];
      shape(al, q, Nl, dNl);
      shape(am, q, Nm, dNm);
      // z-rows touched by DOF (f, a): u_i -> 3i+J (dN_J); eta_k -> 9+k (N)
      int rl[3], rm[3];
      double cl[3], cm[3];
      int nl, nm;
      if (fl < 3) { nl = 3; for (int J = 0; J < 3; ++J) { rl[J] = 3 * fl + J; cl[J] = dNl[J]; } }
      else { nl = 1; rl[0] = 9 + fl - 3; cl[0] = Nl; }
      if (fm < 3) { nm = 3; for (int J = 0; J < 3; ++J) { rm[J] = 3 * fm + J; cm[J] = dNm[J]; } }
      else { nm = 1; rm[0] = 9 + fm - 3; cm[0] = Nm; }
      for (int x = 0; x < nl; ++x)
        for (int y = 0; y < nm; ++y) {
          const int r = rl[x] < rm[y] ? rl[x] : rm[y];
          const int cc = rl[x] < rm[y] ? rm[y] : rl[x];
          s += cl[x] * cm[y] * double(H[hstore_offset<T>(blk, hidx(r, cc), lane0 + q)]);
        }
      if (fl >= 3 && fm >= 3)
        s += (dNl[0] * dNm[0] + dNl[1] * dNm[1] + dNl[2] * dNm[2]) * P.G[fl - 3][fm - 3];
    }
    const int64_t col = fm * nn + node_of(am);
    if (color >= 0)
      K[row * ld + col] += w * s;
    else
      atomicAdd(&K[row * ld + col], w * s);
  }
}

// Dirichlet rows/columns -> identity, and the identity block of the augmented matrix.
__global__ void k_coarse_bc(int n, int64_t nn, const dmask_t* __restrict__ mask, double* __restrict__ K,
                            int ld) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (tid >= int64_t(n) * n) return;
  const int r = int(tid / n), c = int(tid % n);
  const bool dr = (mask[r % nn] >> (r / nn)) & 1;
  const bool dc = (mask[c % nn] >> (c / nn)) & 1;
  if (dr || dc) K[int64_t(r) * ld + c] = (r == c) ? 1.0 : 0.0;
  K[int64_t(r) * ld + n + c] = (r == c) ? 1.0 : 0.0;
}

__global__ void k_gj_first_key(const double* __restrict__ M, int n, int ld, unsigned long long* keys) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    atomicMax(&keys[0], pivot_key(M[int64_t(i) * ld], i));
}

// One block per row i; threads stride over the columns.
__global__ void __launch_bounds__(256) k_gj_step(double* __restrict__ M, int n, int ld, int k,
                                                 unsigned long long* __restrict__ keys, int* __restrict__ used,
                                                 int* __restrict__ piv, int* singular) {
  gj_step_row(M, n, ld, k, keys, used, piv, singular, int(blockIdx.x), blockIdx.x == 0);
}

// Ainv[k][c] = M[piv[k]][n + c] / M[piv[k]][k]
__global__ void k_gj_extract(const double* __restrict__ M, int n, int ld, const int* __restrict__ piv,
                             double* __restrict__ Ainv) {
  const int k = blockIdx.x;
  if (k >= n) return;
  const int p = piv[k];
  const double inv = 1.0 / M[int64_t(p) * ld + k];
  for (int c = threadIdx.x; c < n; c += blockDim.x) Ainv[int64_t(k) * n + c] = M[int64_t(p) * ld + n + c] * inv;
}

// x = Ainv b (Ainv dense n x n, row-major).
template <typename T>
__global__ void k_coarse_solve(int n, const double* __restrict__ Ainv, const T* __restrict__ b,
                               T* __restrict__ x) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double* row = Ainv + int64_t(warp) * n;
  double s = 0.0;
  for (int c = lane; c < n; c += 32) s += row[c] * double(b[c]);
  for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
  if (lane == 0) x[warp] = T(s);
}

// Chebyshev-accelerated point-block Jacobi (Saad, Iterative Methods, Alg. 12.1
// applied to D^-1 J): first step d = c D^-1 r0 with r0 = src (also stored in r
// when copy_r), x = d (zero_x) or x += d.
template <typename T>
__global__ void k_cheb_first(int64_t nn, const T* __restrict__ D, const T* src, T c, bool copy_r,
                             bool zero_x, T* r, T* __restrict__ d, T* __restrict__ x) {
  for (int64_t node = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; node < nn;
       node += int64_t(gridDim.x) * blockDim.x)
    cheb_first_node<T>(nn, D, src, c, copy_r, zero_x, r, d, x, node);
}

// r -= y; d = a d + c D^-1 r; x += d.
template <typename T>
__global__ void k_cheb_step(int64_t nn, const T* __restrict__ D, const T* __restrict__ y, T a, T c,
                            T* __restrict__ r, T* __restrict__ d, T* __restrict__ x) {
  for (int64_t node = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; node < nn;
       node += int64_t(gridDim.x) * blockDim.x)
    cheb_step_node<T>(nn, D, y, a, c, r, d, x, node);
}

// Deterministic start vector of the power iteration (power_init_value).
template <typename T>
__global__ void k_power_init(int64_t nn, const dmask_t* __restrict__ mask, T* __restrict__ x) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < NF * nn; i += int64_t(gridDim.x) * blockDim.x)
    x[i] = T(power_init_value(i, nn, mask));
}

// x = y / sqrt(*dot)
template <typename T>
__global__ void k_scale_inv_sqrt(int64_t n, const T* __restrict__ y, const double* __restrict__ dot, T* __restrict__ x) {
  __shared__ T s;  // one FP64 square root and division per block, not per thread
  if (threadIdx.x == 0) s = T(1.0 / sqrt(*dot));
  __syncthreads();
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i] = y[i] * s;
}

// u -= alpha q + sqrt(beta2prev) qp (one Lanczos three-term step)
template <typename T>
__global__ void k_lanczos_orth(int64_t n, T* __restrict__ u, const T* __restrict__ q, const T* __restrict__ qp,
                               const double* __restrict__ alpha, const double* __restrict__ beta2prev) {
  const T a = T(*alpha);
  const T b = beta2prev ? T(sqrt(*beta2prev)) : T(0);
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    u[i] -= a * q[i] + (beta2prev ? b * qp[i] : T(0));
}

}  // namespace

template <typename T>
void launch_lanczos_orth(int64_t n, T* u, const T* q, const T* qp, const double* alpha, const double* beta2prev,
                         cudaStream_t s) {
  k_lanczos_orth<T><<<grid_for(n, 256), 256, 0, s>>>(n, u, q, qp, alpha, beta2prev);
  count_launches(1);
}

template <typename T>
void launch_cheb_first(int64_t nn, const T* D, const T* src, T c, bool copy_r, bool zero_x, T* r, T* d, T* x,
                       cudaStream_t s) {
  k_cheb_first<T><<<grid_for(nn, 256), 256, 0, s>>>(nn, D, src, c, copy_r, zero_x, r, d, x);
  count_launches(1);
}

template <typename T>
void launch_cheb_step(int64_t nn, const T* D, const T* y, T a, T c, T* r, T* d, T* x, cudaStream_t s) {
  k_cheb_step<T><<<grid_for(nn, 256), 256, 0, s>>>(nn, D, y, a, c, r, d, x);
  count_launches(1);
}

template <typename T>
void launch_power_init(int64_t nn, const dmask_t* mask, T* x, cudaStream_t s) {
  k_power_init<T><<<grid_for(NF * nn, 256), 256, 0, s>>>(nn, mask, x);
  count_launches(1);
}

template <typename T>
void launch_scale_inv_sqrt(int64_t n, const T* y, const double* dot, T* x, cudaStream_t s) {
  k_scale_inv_sqrt<T><<<grid_for(n, 256), 256, 0, s>>>(n, y, dot, x);
  count_launches(1);
}

void launch_inject_state(const Grid& fine, const Grid& coarse, const double* Uf, double* Uc,
                         cudaStream_t s) {
  k_inject_state<<<grid_for(coarse.nn(), 128), 128, 0, s>>>(fine, coarse, Uf, Uc);
  count_launches(1);
}

void launch_coarse_mask(const Grid& fine, const Grid& coarse, const dmask_t* mf, dmask_t* mc,
                        cudaStream_t s) {
  k_coarse_mask<<<grid_for(coarse.nn(), 128), 128, 0, s>>>(fine, coarse, mf, mc);
  count_launches(1);
}

// y and z node counts within the grid-dimension limit of a 3-D launch
inline bool grid3_ok(const Grid& g) { return g.ny + 1 <= 65535 && g.nz + 1 <= 65535; }

template <typename T>
void launch_prolong_add(const Grid& fine, const Grid& coarse, const T* xc, const dmask_t* mf, T* xf,
                        cudaStream_t s) {
  if (nested(fine, coarse) && grid3_ok(fine)) {
    const dim3 grid(unsigned((fine.nx + 1 + 127) / 128), unsigned(fine.ny + 1), unsigned(fine.nz + 1));
    k_prolong_add_nested<T><<<grid, 128, 0, s>>>(fine, coarse, xc, mf, xf);
  } else {
    k_prolong_add<T><<<grid_for(fine.nn(), 256), 256, 0, s>>>(fine, coarse, xc, mf, xf);
  }
  count_launches(1);
}

template <typename T>
void launch_restrict(const Grid& fine, const Grid& coarse, const T* rf, const dmask_t* mc, T* rc,
                     cudaStream_t s) {
  if (nested(fine, coarse) && grid3_ok(coarse)) {
    const dim3 grid(unsigned((coarse.nx + 1 + 127) / 128), unsigned(coarse.ny + 1), unsigned(coarse.nz + 1));
    k_restrict_nested<T><<<grid, 128, 0, s>>>(fine, coarse, rf, mc, rc);
  } else {
    k_restrict<T><<<grid_for(coarse.nn(), 128), 128, 0, s>>>(fine, coarse, rf, mc, rc);
  }
  count_launches(1);
}

template <typename T>
void launch_smooth(int64_t nn, const T* D, const T* b, const T* y, T omega, T* x, cudaStream_t s) {
  k_smooth<T><<<grid_for(nn, 256), 256, 0, s>>>(nn, D, b, y, omega, x);
  count_launches(1);
}

template <typename T>
void launch_sub(int64_t n, const T* b, const T* y, T* r, cudaStream_t s) {
  k_sub<T><<<grid_for(n, 256), 256, 0, s>>>(n, b, y, r);
  count_launches(1);
}

template <typename T>
void launch_coarse_assemble(const Grid& g, const DevParams& P, const T* H, const dmask_t* mask,
                            double* K, int ld, cudaStream_t s, bool det) {
  const int n = int(NF * g.nn());
  cudaMemsetAsync(K, 0, sizeof(double) * size_t(n) * ld, s);
  for (int c = det ? 0 : -1; c < (det ? 8 : 0); ++c) {
    k_coarse_assemble<T><<<grid_for(g.ne() * NED, 128), 128, 0, s>>>(g, P, H, K, ld, c);
    count_launches(1);
  }
  k_coarse_bc<<<grid_for(int64_t(n) * n, 256), 256, 0, s>>>(n, g.nn(), mask, K, ld);
  count_launches(1);
}

// Invert the dense coarse operator from the augmented [K | I] (n x 2n,
// ld = 2n; overwritten) into Ainv (n x n). work: (n+1) keys, n used flags and
// n pivot rows. Returns the number of kernel launches.
int dense_gauss_jordan_inverse(double* Maug, int n, double* Ainv, unsigned long long* keys, int* used, int* piv,
                               int* singular, cudaStream_t s) {
  const int ld = 2 * n;
  cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * (n + 1), s);
  cudaMemsetAsync(used, 0, sizeof(int) * n, s);
  k_gj_first_key<<<grid_for(n, 256), 256, 0, s>>>(Maug, n, ld, keys);
  count_launches(1);
  for (int k = 0; k < n; ++k) {
    k_gj_step<<<n, 256, 0, s>>>(Maug, n, ld, k, keys, used, piv, singular);
    count_launches(1);
  }
  k_gj_extract<<<n, 256, 0, s>>>(Maug, n, ld, piv, Ainv);
  count_launches(1);
  return n + 2;
}

template <typename T>
void launch_coarse_solve(int n, const double* Ainv, const T* b, T* x, cudaStream_t s) {
  k_coarse_solve<T><<<grid_for(int64_t(n) * 32, 256), 256, 0, s>>>(n, Ainv, b, x);
  count_launches(1);
}

#define PFM_INST(T)                                                                              \
  template void launch_prolong_add<T>(const Grid&, const Grid&, const T*, const dmask_t*, T*,     \
                                      cudaStream_t);                                            \
  template void launch_restrict<T>(const Grid&, const Grid&, const T*, const dmask_t*, T*,        \
                                   cudaStream_t);                                               \
  template void launch_smooth<T>(int64_t, const T*, const T*, const T*, T, T*, cudaStream_t);     \
  template void launch_sub<T>(int64_t, const T*, const T*, T*, cudaStream_t);                     \
  template void launch_coarse_assemble<T>(const Grid&, const DevParams&, const T*, const dmask_t*, \
                                          double*, int, cudaStream_t, bool);                    \
  template void launch_coarse_solve<T>(int, const double*, const T*, T*, cudaStream_t);         \
  template void launch_cheb_first<T>(int64_t, const T*, const T*, T, bool, bool, T*, T*, T*,       \
                                     cudaStream_t);                                             \
  template void launch_cheb_step<T>(int64_t, const T*, const T*, T, T, T*, T*, T*, cudaStream_t); \
  template void launch_power_init<T>(int64_t, const dmask_t*, T*, cudaStream_t);                  \
  template void launch_scale_inv_sqrt<T>(int64_t, const T*, const double*, T*, cudaStream_t);     \
  template void launch_lanczos_orth<T>(int64_t, T*, const T*, const T*, const double*, const double*, \
                                       cudaStream_t);
PFM_INST(float)
PFM_INST(double)
#undef PFM_INST

}  // namespace pfm
