// Conversion of the public parameter block into the kernels' parameter block.
#pragma once

#include <cmath>

#include "../../include/pfm.h"
#include "qp_physics.cuh"

namespace pfm {

// Derived coefficients (Sec. 2.2-2.3, Eq. IntEnergy, Eq. PenPot):
//   inv_mtau_i = 1/(m_i tau)                       (dissipation Hessian)
//   cobst_ij   = 4 s gamma_ij / (pi ell_ij)         (local obstacle term)
//   a_ij       = cobst_ij ell_ij^2                  (gradient term)
// The gradient energy -sum_{i<j} a_ij grad eta_i . grad eta_j, written in the
// condensed unknowns (grad eta_0 = -sum grad eta_k), is 1/2 sum_d
// (d_d eta_hat)^T G (d_d eta_hat) with G = T^T Ahat T, Ahat_ij = -a_ij (i != j),
// Ahat_ii = 0, and T the 7x6 map eta = e_0 + T eta_hat.
inline void make_dev_params(const pfm_params& in, DevParams& out) {
  const double pi = 3.14159265358979323846;
  for (int p = 0; p < NPH; ++p) {
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) out.U[p][i][j] = in.Ut[p][3 * i + j];
    for (int I = 0; I < 6; ++I)
      for (int J = 0; J < 6; ++J) out.Lv[p][I][J] = in.Lvoigt[p][6 * I + J];
    out.F0[p] = in.F0[p];
    out.inv_mtau[p] = 1.0 / (in.mobility[p] * in.tau);
  }
  double Ahat[NPH][NPH];
  for (int i = 0; i < NPH; ++i)
    for (int j = 0; j < NPH; ++j) {
      if (i == j) {
        out.cobst[i][j] = 0.0;
        Ahat[i][j] = 0.0;
      } else {
        double c = 4.0 * in.gamma_scale * in.gamma[i][j] / (pi * in.ell[i][j]);
        out.cobst[i][j] = c;
        Ahat[i][j] = -c * in.ell[i][j] * in.ell[i][j];
      }
    }
  for (int k = 0; k < NV; ++k)
    for (int l = 0; l < NV; ++l)
      out.G[k][l] = Ahat[k + 1][l + 1] - Ahat[0][l + 1] - Ahat[k + 1][0] + Ahat[0][0];
  out.eps_eta = in.eps_eta;
  // Hencky mode: m-point Gauss-Legendre nodes s_k and weights w_k on [0, 1]
  out.hencky = in.hencky;
  for (int k = 0; k < 3; ++k) out.pade_s[k] = out.pade_w[k] = 0.0;
  if (in.hencky == 1) {
    out.pade_s[0] = 0.5;
    out.pade_w[0] = 1.0;
  } else if (in.hencky == 2) {
    const double d = std::sqrt(3.0) / 6.0;
    out.pade_s[0] = 0.5 - d;
    out.pade_s[1] = 0.5 + d;
    out.pade_w[0] = out.pade_w[1] = 0.5;
  } else if (in.hencky == 3) {
    const double d = 0.5 * std::sqrt(0.6);
    out.pade_s[0] = 0.5 - d;
    out.pade_s[1] = 0.5;
    out.pade_s[2] = 0.5 + d;
    out.pade_w[0] = out.pade_w[2] = 5.0 / 18.0;
    out.pade_w[1] = 8.0 / 18.0;
  }
  out.same_L = 1;
  for (int p = 1; p < NPH; ++p)
    for (int k = 0; k < 36; ++k)
      if (in.Lvoigt[p][k] != in.Lvoigt[0][k]) out.same_L = 0;
  // one stiffness with cubic symmetry in the frame of the parameter block:
  // c11 on the normal diagonal, c12 off it, c44 on the shear diagonal, zero
  // elsewhere; then L = c12 I x I + c44 (2 I_sym) + (c11 - c12 - 2 c44) sum_n e_n^4
  const double* L0 = in.Lvoigt[0];
  const double c11 = L0[0], c12 = L0[1], c44 = L0[21];
  bool cubic = out.same_L == 1;
  for (int I = 0; I < 6 && cubic; ++I)
    for (int J = 0; J < 6; ++J) {
      const double want = (I < 3 && J < 3) ? (I == J ? c11 : c12) : (I == J ? c44 : 0.0);
      if (L0[6 * I + J] != want) cubic = false;
    }
  out.cubic = cubic ? 1 : 0;
  out.cub_lambda = c12;
  out.cub_mu = c44;
  out.cub_delta = c11 - c12 - 2.0 * c44;
}

}  // namespace pfm
