// Frictionless penalty contact with a rigid sphere on the top face z = Lz
// (Sec. 2.5, Eq. Ngap, Eq. PenPot): at a surface Gauss point X the current
// position is x = X + u(X) (bilinear face interpolation of the four face
// nodes' displacements), the normal gap to a sphere of centre c and radius R
// is g = |x - c| - R (closest-point projection: xbar = c + R n, n = (x-c)/|x-c|),
// and the potential gains w * 1/2 eps_N <g>_-^2 with w the reference area
// weight of the 2x2 Gauss rule on the face quad. With r = |x - c|:
//   d/dx   = eps_N <g>_- n,
//   d2/dx2 = eps_N [g < 0] (n n^T + (g / r)(I - n n^T)).
// One thread per surface Gauss point (4 per face quad); nodal results are
// scattered with atomics. The work is two-dimensional and negligible next to
// the volume kernels.
#include "common.cuh"

namespace pfm {
namespace {

inline unsigned grid_for_c(int64_t threads, int block) {
  int64_t b = (threads + block - 1) / block;
  return unsigned(b > 0 ? b : 1);
}

struct SurfPoint {
  int64_t node[4];
  double N[4];
  double X[3];
};

// Gauss point q (0..3) of top-face quad (i, j): nodes, shape values, reference position.
__device__ __forceinline__ SurfPoint surf_point(const Grid& g, int64_t tid) {
  SurfPoint s;
  const int q = int(tid & 3);
  const int64_t quad = tid >> 2;
  const int i = int(quad % g.nx), j = int(quad / g.nx);
  const double gs = (q & 1) ? GB : GA, gt = (q & 2) ? GB : GA;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    s.node[a] = (i + (a & 1)) + int64_t(g.nx + 1) * ((j + (a >> 1)) + int64_t(g.ny + 1) * g.nz);
    s.N[a] = ((a & 1) ? gs : 1.0 - gs) * ((a & 2) ? gt : 1.0 - gt);
  }
  s.X[0] = (i + gs) * g.hx;
  s.X[1] = (j + gt) * g.hy;
  s.X[2] = g.nz * g.hz;
  return s;
}

__device__ __forceinline__ double surf_w(const Grid& g) { return 0.25 * g.hx * g.hy; }

__global__ void k_contact_residual(Grid g, ContactParams c, const double* __restrict__ U,
                                   const dmask_t* __restrict__ mask, double* __restrict__ R, double* energy,
                                   double* load) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (tid >= int64_t(g.nx) * g.ny * 4) return;
  const SurfPoint s = surf_point(g, tid);
  const int64_t nn = g.nn();
  double d[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double u = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a) u += s.N[a] * U[k * nn + s.node[a]];
    d[k] = s.X[k] + u - c.center[k];
  }
  const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  const double gap = r - c.radius;
  if (!(gap < 0.0)) return;
  const double w = surf_w(g);
  const double f = c.eps_N * gap / r;  // eps <g>_- n = f d
  if (R) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const dmask_t dm = mask[s.node[a]];
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (!((dm >> k) & 1)) atomicAdd(&R[k * nn + s.node[a]], w * s.N[a] * f * d[k]);
    }
  }
  if (energy) atomicAdd(energy, w * 0.5 * c.eps_N * gap * gap);
  if (load) atomicAdd(load, w * c.eps_N * gap * d[2] / r);
}

// Surface Hessian at every surface Gauss point, symmetric 3x3 stored as
// (xx, yy, zz, yz, xz, xy), in FP64 and/or FP32.
__global__ void k_contact_linearize(Grid g, ContactParams c, const double* __restrict__ U, double* __restrict__ K64,
                                    float* __restrict__ K32) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (tid >= int64_t(g.nx) * g.ny * 4) return;
  const SurfPoint s = surf_point(g, tid);
  const int64_t nn = g.nn();
  double d[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double u = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a) u += s.N[a] * U[k * nn + s.node[a]];
    d[k] = s.X[k] + u - c.center[k];
  }
  const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  const double gap = r - c.radius;
  double K[6] = {0, 0, 0, 0, 0, 0};
  if (gap < 0.0) {
    const double n[3] = {d[0] / r, d[1] / r, d[2] / r};
    const double t = gap / r;
    const int ii[6] = {0, 1, 2, 1, 0, 0}, jj[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
    for (int v = 0; v < 6; ++v) {
      const double nn_ = n[ii[v]] * n[jj[v]];
      K[v] = c.eps_N * (nn_ + t * ((ii[v] == jj[v] ? 1.0 : 0.0) - nn_));
    }
  }
#pragma unroll
  for (int v = 0; v < 6; ++v) {
    if (K64) K64[tid * 6 + v] = K[v];
    if (K32) K32[tid * 6 + v] = float(K[v]);
  }
}

template <typename T>
__device__ __forceinline__ void sym_mul(const T* K, const T x[3], T y[3]) {
  y[0] = K[0] * x[0] + K[5] * x[1] + K[4] * x[2];
  y[1] = K[5] * x[0] + K[1] * x[1] + K[3] * x[2];
  y[2] = K[4] * x[0] + K[3] * x[1] + K[2] * x[2];
}

// y += Jc v (Dirichlet DOFs read as 0 and left untouched). TV: input type,
// TY: output and arithmetic type.
template <typename TK, typename TV, typename TY>
__global__ void k_contact_apply(Grid g, const TK* __restrict__ K, const dmask_t* __restrict__ mask,
                                const TV* __restrict__ v, TY* __restrict__ y) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (tid >= int64_t(g.nx) * g.ny * 4) return;
  const SurfPoint s = surf_point(g, tid);
  const int64_t nn = g.nn();
  TY Kq[6];
  bool any = false;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    Kq[k] = TY(K[tid * 6 + k]);
    any |= Kq[k] != TY(0);
  }
  if (!any) return;
  dmask_t dm[4];
  TY du[3] = {TY(0), TY(0), TY(0)};
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    dm[a] = mask[s.node[a]];
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (!((dm[a] >> k) & 1)) du[k] += TY(s.N[a]) * TY(v[k * nn + s.node[a]]);
  }
  TY f[3];
  sym_mul(Kq, du, f);
  const TY w = TY(surf_w(g));
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (!((dm[a] >> k) & 1)) atomicAdd(&y[k * nn + s.node[a]], w * TY(s.N[a]) * f[k]);
}

// Nodal diagonal blocks: D_a(u, u) += w N_a^2 K (before the block inversion).
template <typename T>
__global__ void k_contact_blockdiag(Grid g, const T* __restrict__ K, T* __restrict__ D) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (tid >= int64_t(g.nx) * g.ny * 4) return;
  const SurfPoint s = surf_point(g, tid);
  const int64_t nn = g.nn();
  const T* Kq = K + tid * 6;
  const int sv[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};
  const double w = surf_w(g);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        const T val = Kq[sv[r][cc]];
        if (val != T(0)) atomicAdd(&D[(r * NF + cc) * nn + s.node[a]], T(w * s.N[a] * s.N[a]) * val);
      }
}

// Dense coarse operator: K[(k, a), (l, b)] += w N_a N_b K_kl at free DOFs.
__global__ void k_contact_coarse(Grid g, const double* __restrict__ K, const dmask_t* __restrict__ mask,
                                 double* __restrict__ M, int ld) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (tid >= int64_t(g.nx) * g.ny * 4) return;
  const SurfPoint s = surf_point(g, tid);
  const int64_t nn = g.nn();
  const double* Kq = K + tid * 6;
  const int sv[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};
  const double w = surf_w(g);
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
          if (((mask[s.node[a]] >> k) & 1) || ((mask[s.node[b]] >> l) & 1)) continue;
          const double val = Kq[sv[k][l]];
          if (val != 0.0) atomicAdd(&M[(k * nn + s.node[a]) * ld + l * nn + s.node[b]], w * s.N[a] * s.N[b] * val);
        }
}

}  // namespace

int64_t contact_points(const Grid& g) { return int64_t(g.nx) * g.ny * 4; }

void launch_contact_residual(const Grid& g, const ContactParams& c, const double* U, const dmask_t* mask, double* R,
                             double* energy, double* load, cudaStream_t s) {
  k_contact_residual<<<grid_for_c(contact_points(g), 128), 128, 0, s>>>(g, c, U, mask, R, energy, load);
  count_launches(1);
}

void launch_contact_linearize(const Grid& g, const ContactParams& c, const double* U, double* K64, float* K32,
                              cudaStream_t s) {
  k_contact_linearize<<<grid_for_c(contact_points(g), 128), 128, 0, s>>>(g, c, U, K64, K32);
  count_launches(1);
}

template <typename TK, typename TV, typename TY>
void launch_contact_apply(const Grid& g, const TK* K, const dmask_t* mask, const TV* v, TY* y, cudaStream_t s) {
  k_contact_apply<TK, TV, TY><<<grid_for_c(contact_points(g), 128), 128, 0, s>>>(g, K, mask, v, y);
  count_launches(1);
}

template <typename T>
void launch_contact_blockdiag(const Grid& g, const T* K, T* D, cudaStream_t s) {
  k_contact_blockdiag<T><<<grid_for_c(contact_points(g), 128), 128, 0, s>>>(g, K, D);
  count_launches(1);
}

void launch_contact_coarse(const Grid& g, const double* K, const dmask_t* mask, double* M, int ld, cudaStream_t s) {
  k_contact_coarse<<<grid_for_c(contact_points(g), 128), 128, 0, s>>>(g, K, mask, M, ld);
  count_launches(1);
}

template void launch_contact_apply<float, float, float>(const Grid&, const float*, const dmask_t*, const float*,
                                                        float*, cudaStream_t);
template void launch_contact_apply<double, double, double>(const Grid&, const double*, const dmask_t*,
                                                           const double*, double*, cudaStream_t);
template void launch_contact_apply<double, float, double>(const Grid&, const double*, const dmask_t*, const float*,
                                                          double*, cudaStream_t);
template void launch_contact_blockdiag<float>(const Grid&, const float*, float*, cudaStream_t);
template void launch_contact_blockdiag<double>(const Grid&, const double*, double*, cudaStream_t);

}  // namespace pfm
