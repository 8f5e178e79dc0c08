// Vector kernels of the Krylov solver (FGMRES with classical Gram-Schmidt
// applied twice, Sec. 3.4 uses GMRES): block-partial multi-dot products
// reduced deterministically in a second pass, multi-axpy, casts between FP64
// and FP32 and Dirichlet bookkeeping.
#include "common.cuh"

namespace pfm {
namespace {

constexpr int RED_THREADS = 256;
constexpr int RED_MAX_BLOCKS = 1024;
constexpr int MDOT_CHUNK = 8;

inline unsigned grid_for(int64_t threads, int block) {
  int64_t b = (threads + block - 1) / block;
  if (b < 1) b = 1;
  if (b > 65535 * 4) b = 65535 * 4;
  return unsigned(b);
}

template <typename T>
__global__ void k_fill(int64_t n, T val, T* __restrict__ x) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i] = val;
}

__global__ void k_cast_d2f(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    b[i] = float(a[i]);
}

__global__ void k_cast_f2d(int64_t n, const float* __restrict__ a, double* __restrict__ b) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    b[i] = double(a[i]);
}

// x = hi + lo with hi = x rounded to FP32 and lo = the remainder rounded to
// FP32 (x - hi is exact in FP64; |x - hi - lo| <= 2^-48 |x| roughly).
__global__ void k_split_f64(int64_t n, const double* __restrict__ x, float* __restrict__ hi, float* __restrict__ lo) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double v = x[i];
    const float h = float(v);
    hi[i] = h;
    lo[i] = float(v - double(h));
  }
}

// r = b - a - c (FP64 b, a; FP32 c).
__global__ void k_sub2(int64_t n, const double* __restrict__ b, const double* __restrict__ a,
                       const float* __restrict__ c, double* __restrict__ r) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    r[i] = (b[i] - a[i]) - double(c[i]);
}

// partial[blk*kstride + j0 + j] = sum over this block's slice of V_j . w,
// j = 0..cnt-1 (cnt <= MDOT_CHUNK).
__global__ void __launch_bounds__(RED_THREADS) k_mdot_partial(int64_t n, int j0, int cnt,
                                                               const double* __restrict__ V, int64_t ldv,
                                                               const double* __restrict__ w,
                                                               double* __restrict__ partial, int kstride) {
  double acc[MDOT_CHUNK];
#pragma unroll
  for (int j = 0; j < MDOT_CHUNK; ++j) acc[j] = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double wi = w[i];
#pragma unroll
    for (int j = 0; j < MDOT_CHUNK; ++j)
      if (j < cnt) acc[j] += V[int64_t(j0 + j) * ldv + i] * wi;
  }
  __shared__ double red[RED_THREADS / 32][MDOT_CHUNK];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < MDOT_CHUNK; ++j) {
    double v = acc[j];
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    if (lane == 0) red[wid][j] = v;
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double s = 0.0;
    for (int q = 0; q < RED_THREADS / 32; ++q) s += red[q][threadIdx.x];
    partial[int64_t(blockIdx.x) * kstride + j0 + threadIdx.x] = s;
  }
}

// out[j] = sum_b partial[b*kstride + j], one block per j, fixed order.
__global__ void k_mdot_final(int nblocks, int k, const double* __restrict__ partial, int kstride,
                             double* __restrict__ out) {
  const int j = blockIdx.x;
  if (j >= k) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[int64_t(b) * kstride + j];
  __shared__ double red[RED_THREADS];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int m = blockDim.x / 2; m > 0; m >>= 1) {
    if (threadIdx.x < m) red[threadIdx.x] += red[threadIdx.x + m];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = red[0];
}

// partial[blk] = sum over this block's slice of a . b (accumulated in FP64)
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_dot_partial(int64_t n, const T* __restrict__ a,
                                                              const T* __restrict__ b,
                                                              double* __restrict__ partial) {
  double acc = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    acc += double(a[i]) * double(b[i]);
  __shared__ double red[RED_THREADS / 32];
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < RED_THREADS / 32; ++q) s += red[q];
    partial[blockIdx.x] = s;
  }
}

__global__ void k_maxpy(int64_t n, int k, const double* __restrict__ V, int64_t ldv,
                        const double* __restrict__ h, double* __restrict__ w) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    double s = w[i];
    for (int j = 0; j < k; ++j) s -= h[j] * V[int64_t(j) * ldv + i];
    w[i] = s;
  }
}

__global__ void k_scale_copy(int64_t n, const double* __restrict__ a, const double* __restrict__ alpha,
                             double* __restrict__ b) {
  const double inv = 1.0 / *alpha;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    b[i] = a[i] * inv;
}

template <typename T>
__global__ void k_gemv_add(int64_t n, int k, const T* __restrict__ Z, int64_t ldz, const double* __restrict__ y,
                           double* __restrict__ x) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    double s = x[i];
    for (int j = 0; j < k; ++j) s += y[j] * double(Z[int64_t(j) * ldz + i]);
    x[i] = s;
  }
}

__global__ void k_axpy(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] += a * x[i];
}

__global__ void k_mask_values(int64_t nn, const dmask_t* __restrict__ mask, const double* __restrict__ val,
                              double* __restrict__ U) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < NF * nn; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t node = i % nn;
    const int f = int(i / nn);
    if ((mask[node] >> f) & 1) U[i] = val[i];
  }
}

__global__ void k_build_mask(int64_t nn, const uint8_t* __restrict__ m8, dmask_t* __restrict__ mask, int* bad) {
  for (int64_t node = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; node < nn;
       node += int64_t(gridDim.x) * blockDim.x) {
    dmask_t m = 0;
    for (int f = 0; f < NF; ++f)
      if (m8[f * nn + node]) m |= dmask_t(1u << f);
    if (m & MASK_ETA) atomicExch(bad, 1);  // order parameters cannot be prescribed
    mask[node] = m;
  }
}

}  // namespace

int reduction_blocks(int64_t n) {
  int64_t b = (n + RED_THREADS * 8 - 1) / (RED_THREADS * 8);
  if (b < 1) b = 1;
  if (b > RED_MAX_BLOCKS) b = RED_MAX_BLOCKS;
  return int(b);
}

template <typename T>
void launch_fill(int64_t n, T val, T* x, cudaStream_t s) {
  k_fill<T><<<grid_for(n, 256), 256, 0, s>>>(n, val, x);
  count_launches(1);
}
void launch_cast_d2f(int64_t n, const double* a, float* b, cudaStream_t s) {
  k_cast_d2f<<<grid_for(n, 256), 256, 0, s>>>(n, a, b);
  count_launches(1);
}
void launch_split_f64(int64_t n, const double* x, float* hi, float* lo, cudaStream_t s) {
  k_split_f64<<<grid_for(n, 256), 256, 0, s>>>(n, x, hi, lo);
  count_launches(1);
}

void launch_sub2(int64_t n, const double* b, const double* a, const float* c, double* r, cudaStream_t s) {
  k_sub2<<<grid_for(n, 256), 256, 0, s>>>(n, b, a, c, r);
  count_launches(1);
}

void launch_cast_f2d(int64_t n, const float* a, double* b, cudaStream_t s) {
  k_cast_f2d<<<grid_for(n, 256), 256, 0, s>>>(n, a, b);
  count_launches(1);
}

// out[0..k) = V_j . w (V_j at V + j*ldv). partial: >= reduction_blocks(n)*k doubles.
void launch_mdot(int64_t n, int k, const double* V, int64_t ldv, const double* w, double* partial,
                 double* out, cudaStream_t s) {
  const int nb = reduction_blocks(n);
  for (int j0 = 0; j0 < k; j0 += MDOT_CHUNK) {
    const int cnt = (k - j0) < MDOT_CHUNK ? (k - j0) : MDOT_CHUNK;
    k_mdot_partial<<<nb, RED_THREADS, 0, s>>>(n, j0, cnt, V, ldv, w, partial, k);
    count_launches(1);
  }
  k_mdot_final<<<k, RED_THREADS, 0, s>>>(nb, k, partial, k, out);
  count_launches(1);
}

template <typename T>
void launch_dot(int64_t n, const T* a, const T* b, double* partial, double* out, cudaStream_t s) {
  const int nb = reduction_blocks(n);
  k_dot_partial<T><<<nb, RED_THREADS, 0, s>>>(n, a, b, partial);
  count_launches(1);
  k_mdot_final<<<1, RED_THREADS, 0, s>>>(nb, 1, partial, 1, out);
  count_launches(1);
}
template void launch_dot<float>(int64_t, const float*, const float*, double*, double*, cudaStream_t);
template void launch_dot<double>(int64_t, const double*, const double*, double*, double*, cudaStream_t);

void launch_maxpy(int64_t n, int k, const double* V, int64_t ldv, const double* h, double* w,
                  cudaStream_t s) {
  k_maxpy<<<grid_for(n, 256), 256, 0, s>>>(n, k, V, ldv, h, w);
  count_launches(1);
}

void launch_scale_copy(int64_t n, const double* a, const double* alpha_dev, double* b, cudaStream_t s) {
  k_scale_copy<<<grid_for(n, 256), 256, 0, s>>>(n, a, alpha_dev, b);
  count_launches(1);
}

template <typename T>
void launch_gemv_add(int64_t n, int k, const T* Z, int64_t ldz, const double* y, double* x, cudaStream_t s) {
  k_gemv_add<T><<<grid_for(n, 256), 256, 0, s>>>(n, k, Z, ldz, y, x);
  count_launches(1);
}

void launch_axpy(int64_t n, double a, const double* x, double* y, cudaStream_t s) {
  k_axpy<<<grid_for(n, 256), 256, 0, s>>>(n, a, x, y);
  count_launches(1);
}

void launch_mask_values(int64_t nn, const dmask_t* mask, const double* val, double* U, cudaStream_t s) {
  k_mask_values<<<grid_for(NF * nn, 256), 256, 0, s>>>(nn, mask, val, U);
  count_launches(1);
}

void launch_build_mask(int64_t nn, const uint8_t* m8, dmask_t* mask, int* bad, cudaStream_t s) {
  k_build_mask<<<grid_for(nn, 256), 256, 0, s>>>(nn, m8, mask, bad);
  count_launches(1);
}

template void launch_fill<float>(int64_t, float, float*, cudaStream_t);
template void launch_fill<double>(int64_t, double, double*, cudaStream_t);
template void launch_gemv_add<float>(int64_t, int, const float*, int64_t, const double*, double*, cudaStream_t);
template void launch_gemv_add<double>(int64_t, int, const double*, int64_t, const double*, double*, cudaStream_t);

}  // namespace pfm
