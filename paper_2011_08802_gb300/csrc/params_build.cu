// Host construction of parameter blocks (pfm_params_from_cubic,
// pfm_params_orthorhombic_stiffness, pfm_params_rotate): the model data of
// Sec. 5.1 and the anisotropic constants of Table 1 written into a pfm_params
// without any CUDA call, so that a C caller does not have to rebuild the
// variant stretches, Voigt stiffnesses and Bond-matrix rotations itself.
#include <cmath>
#include <cstring>

#include "../../include/pfm.h"
#include "qp_physics.cuh"

namespace {

constexpr int NPH_ = PFM_NV + 1;

// Voigt order of the strain vector: (11, 22, 33, 23, 13, 12)
constexpr int VI[6] = {0, 1, 2, 1, 0, 0};
constexpr int VJ[6] = {0, 1, 2, 2, 2, 1};

// Bond matrix M of an orthogonal a (x' = a x) for stiffnesses acting on
// engineering shear strains: L' = M L M^T, M[I][J] = a_ik a_jk (J a normal
// slot (k, k)), a_ik a_jl + a_il a_jk (J a shear slot (k, l)).
void bond(const double a[3][3], double M[6][6]) {
  for (int I = 0; I < 6; ++I)
    for (int J = 0; J < 6; ++J) {
      const int i = VI[I], j = VJ[I], k = VI[J], l = VJ[J];
      M[I][J] = J < 3 ? a[i][k] * a[j][k] : a[i][k] * a[j][l] + a[i][l] * a[j][k];
    }
}

void congruence6(const double M[6][6], double L[6][6]) {  // L <- M L M^T
  double T[6][6], R[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double s = 0.0;
      for (int k = 0; k < 6; ++k) s += L[i][k] * M[j][k];
      T[i][j] = s;
    }
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double s = 0.0;
      for (int k = 0; k < 6; ++k) s += M[i][k] * T[k][j];
      R[i][j] = s;
    }
  std::memcpy(L, R, sizeof(R));
}

void cubic_voigt(double c11, double c12, double c44, double L[6][6]) {
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) L[i][j] = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) L[i][j] = i == j ? c11 : c12;
  L[3][3] = L[4][4] = L[5][5] = c44;
}

}  // namespace

extern "C" {

pfm_status pfm_params_from_cubic(const pfm_cubic_material* m, double tau, int hencky, pfm_params* out) {
  if (!m || !out || hencky < 0 || hencky > 3 || PFM_NV != 6) return PFM_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  const double p = 0.5 * (m->stretch_alpha + m->stretch_gamma), q = 0.5 * (m->stretch_alpha - m->stretch_gamma);
  const double b = m->stretch_beta;
  double U[NPH_][3][3] = {};
  U[0][0][0] = U[0][1][1] = U[0][2][2] = 1.0;
  for (int t = 0; t < 2; ++t) {
    const double sq = t == 0 ? q : -q;
    double* A = &U[1 + t][0][0];  // shear in the (1,3) plane, beta on axis 2
    const double a1[9] = {p, 0, sq, 0, b, 0, sq, 0, p};
    double* B = &U[3 + t][0][0];  // shear in the (1,2) plane, beta on axis 3
    const double b1[9] = {p, sq, 0, sq, p, 0, 0, 0, b};
    double* C = &U[5 + t][0][0];  // beta on axis 1, shear in the (2,3) plane
    const double c1[9] = {b, 0, 0, 0, p, sq, 0, sq, p};
    for (int k = 0; k < 9; ++k) {
      A[k] = a1[k];
      B[k] = b1[k];
      C[k] = c1[k];
    }
  }
  double L[6][6];
  cubic_voigt(m->C11, m->C12, m->C44, L);
  for (int i = 0; i < NPH_; ++i) {
    std::memcpy(out->Ut[i], &U[i][0][0], sizeof(double) * 9);
    std::memcpy(out->Lvoigt[i], &L[0][0], sizeof(double) * 36);
    out->F0[i] = i == 0 ? m->F0_austenite : m->F0_martensite;
    out->mobility[i] = m->mobility;
    for (int j = 0; j < NPH_; ++j) {
      out->gamma[i][j] = i == j ? 0.0 : ((i == 0 || j == 0) ? m->gamma_am : m->gamma_mm);
      out->ell[i][j] = m->ell;
    }
  }
  out->eps_eta = m->eps_eta;
  out->tau = tau;
  out->gamma_scale = 1.0;
  out->hencky = hencky;
  return PFM_OK;
}

pfm_status pfm_params_orthorhombic_stiffness(pfm_params* p, const double cubic[3], const double ortho[9],
                                             const double axis_stretch[3]) {
  if (!p || !cubic || !ortho || !axis_stretch) return PFM_ERR_INVALID_ARG;
  // orthorhombic matrix in its own axes: (c11, c22, c33, c44, c55, c66, c12, c13, c23)
  double Lo[6][6] = {};
  Lo[0][0] = ortho[0];
  Lo[1][1] = ortho[1];
  Lo[2][2] = ortho[2];
  Lo[3][3] = ortho[3];
  Lo[4][4] = ortho[4];
  Lo[5][5] = ortho[5];
  Lo[0][1] = Lo[1][0] = ortho[6];
  Lo[0][2] = Lo[2][0] = ortho[7];
  Lo[1][2] = Lo[2][1] = ortho[8];
  double Lc[6][6];
  cubic_voigt(cubic[0], cubic[1], cubic[2], Lc);
  double out[NPH_][6][6];
  std::memcpy(out[0], Lc, sizeof(Lc));
  for (int i = 1; i < NPH_; ++i) {
    double a[3][3], lam[3], Q[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) a[r][c] = p->Ut[i][3 * r + c];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < r; ++c)
        if (std::fabs(a[r][c] - a[c][r]) > 1e-12 * (std::fabs(a[r][c]) + 1.0)) return PFM_ERR_INVALID_ARG;
    pfm::jacobi_eig3<double>(a, lam, Q);
    if (!(lam[0] > 0.0 && lam[1] > 0.0 && lam[2] > 0.0)) return PFM_ERR_INVALID_ARG;
    // variant axis k: the eigenvector whose eigenvalue is closest to axis_stretch[k]
    double axes[3][3];
    for (int k = 0; k < 3; ++k) {
      int best = 0;
      for (int e = 1; e < 3; ++e)
        if (std::fabs(lam[e] - axis_stretch[k]) < std::fabs(lam[best] - axis_stretch[k])) best = e;
      for (int r = 0; r < 3; ++r) axes[r][k] = Q[r][best];
    }
    double M[6][6];
    bond(axes, M);
    std::memcpy(out[i], Lo, sizeof(Lo));
    congruence6(M, out[i]);
  }
  for (int i = 0; i < NPH_; ++i) std::memcpy(p->Lvoigt[i], &out[i][0][0], sizeof(double) * 36);
  return PFM_OK;
}

pfm_status pfm_params_rotate(pfm_params* p, const double R[9]) {
  if (!p || !R) return PFM_ERR_INVALID_ARG;
  double a[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) a[r][c] = R[3 * r + c];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      const double d = a[r][0] * a[c][0] + a[r][1] * a[c][1] + a[r][2] * a[c][2];
      if (std::fabs(d - (r == c ? 1.0 : 0.0)) > 1e-12) return PFM_ERR_INVALID_ARG;
    }
  double M[6][6];
  bond(a, M);
  for (int i = 0; i < NPH_; ++i) {
    double U[3][3], T[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) U[r][c] = p->Ut[i][3 * r + c];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) T[r][c] = U[r][0] * a[c][0] + U[r][1] * a[c][1] + U[r][2] * a[c][2];  // U R^T
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        p->Ut[i][3 * r + c] = a[r][0] * T[0][c] + a[r][1] * T[1][c] + a[r][2] * T[2][c];  // R U R^T
    double L[6][6];
    std::memcpy(L, p->Lvoigt[i], sizeof(L));
    congruence6(M, L);
    std::memcpy(p->Lvoigt[i], L, sizeof(L));
  }
  return PFM_OK;
}

}  // extern "C"
