// Element-matrix form of the element RHS, for comparison with the direct,
// restructured form (the paper's Sec. V-A restructuring removed exactly this:
// its baseline built element matrices and multiplied them by the unknowns).
//
// With the nonlinear coefficients frozen at the current state — advection
// velocity a_g = u_h(xi_g), tau_g and mu_eff — every term of the weak form is
// linear in the element unknowns U = (u_b,j, p_b), so F_e = K_e U exactly:
//   K[(a,i),(b,i)] += -rho sum_g w N_a(g) (a_g.grad N_b)             convection
//                     - mu_eff V grad N_a . grad N_b                 viscous
//                     - rho^2 sum_g w tau_g (a_g.grad N_a)(a_g.grad N_b)   SUPG
//   K[(a,i),(b,p)] +=  w sum_g N_b(g) dN_a/dx_i                      pressure
//                     - rho sum_g w tau_g (a_g.grad N_a) dN_b/dx_i   SUPG
//   K[(a,p),(b,j)] += -w sum_g N_a(g) dN_b/dx_j                      continuity
//                     - rho sum_g w tau_g dN_a/dx_j (a_g.grad N_b)   PSPG
//   K[(a,p),(b,p)] += -sum_g w tau_g grad N_a . grad N_b             PSPG
// with w = V/4. The matrix is built in full, Gauss point by Gauss point, and
// then multiplied by U, as an element-matrix code does.
#pragma once

#include "element.cuh"

namespace nsrhs {

template <bool VREMAN>
__device__ __forceinline__ void element_rhs_by_matrix(const double c[3][3], double inv_det,
                                                      double rh, const double u[4][3],
                                                      const double p[4],
                                                      const ElemParams<double>& P,
                                                      double F[4][4]) {
  using M = MathOps<double>;
  // shape-function gradients
  double dN[4][3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    dN[1][j] = c[0][j] * inv_det;
    dN[2][j] = c[1][j] * inv_det;
    dN[3][j] = c[2][j] * inv_det;
    dN[0][j] = -(dN[1][j] + dN[2][j] + dN[3][j]);
  }
  const double det = M::rcp(inv_det);
  const double V = det * (1.0 / 6.0);
  const double w = 0.25 * V;
  // mu_eff (Vreman on the velocity gradient), as in the direct form
  double mu_eff = P.mu;
  if (VREMAN) {
    double G[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        G[i][j] = 0.0;
        for (int a = 0; a < 4; ++a) G[i][j] += u[a][i] * dN[a][j];
      }
    double A = 0.0, be[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        A += G[i][j] * G[i][j];
        be[i][j] = 0.0;
        for (int m = 0; m < 3; ++m) be[i][j] += G[i][m] * G[j][m];
      }
    const double B = be[0][0] * be[1][1] - be[0][1] * be[0][1] + be[0][0] * be[2][2] -
                     be[0][2] * be[0][2] + be[1][1] * be[2][2] - be[1][2] * be[1][2];
    if (A > 0.0 && B > 0.0) {
      const double h2 = M::rcp(rh * rh);
      mu_eff = P.mu + P.rho * P.c_vreman * h2 * M::sqrt_(B * M::rcp(A));
    }
  }
  const double k1 = P.c1 * mu_eff * rh * rh, k2 = P.c2 * P.rho * rh;
  double K[16][16];
  for (int r = 0; r < 16; ++r)
    for (int q = 0; q < 16; ++q) K[r][q] = 0.0;
  // viscous (constant gradients)
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      const double kv = -mu_eff * V * (dN[a][0] * dN[b][0] + dN[a][1] * dN[b][1] + dN[a][2] * dN[b][2]);
      for (int i = 0; i < 3; ++i) K[4 * a + i][4 * b + i] += kv;
    }
  for (int g = 0; g < 4; ++g) {
    double Ng[4];
    for (int a = 0; a < 4; ++a) Ng[a] = (a == g) ? kQA : kQB;
    double ag[3];
    for (int i = 0; i < 3; ++i) {
      ag[i] = 0.0;
      for (int a = 0; a < 4; ++a) ag[i] += Ng[a] * u[a][i];
    }
    const double tau = M::rcp(k1 + k2 * M::sqrt_(ag[0] * ag[0] + ag[1] * ag[1] + ag[2] * ag[2]));
    double adN[4];
    for (int a = 0; a < 4; ++a) adN[a] = ag[0] * dN[a][0] + ag[1] * dN[a][1] + ag[2] * dN[a][2];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        const double kuu = -P.rho * w * Ng[a] * adN[b] - P.rho * P.rho * w * tau * adN[a] * adN[b];
        for (int i = 0; i < 3; ++i) {
          K[4 * a + i][4 * b + i] += kuu;
          K[4 * a + i][4 * b + 3] += w * Ng[b] * dN[a][i] - P.rho * w * tau * adN[a] * dN[b][i];
          K[4 * a + 3][4 * b + i] += -w * Ng[a] * dN[b][i] - P.rho * w * tau * dN[a][i] * adN[b];
        }
        K[4 * a + 3][4 * b + 3] +=
            -w * tau * (dN[a][0] * dN[b][0] + dN[a][1] * dN[b][1] + dN[a][2] * dN[b][2]);
      }
  }
  double U[16];
  for (int b = 0; b < 4; ++b) {
    for (int j = 0; j < 3; ++j) U[4 * b + j] = u[b][j];
    U[4 * b + 3] = p[b];
  }
  for (int r = 0; r < 16; ++r) {
    double acc = 0.0;
    for (int q = 0; q < 16; ++q) acc += K[r][q] * U[q];
    F[r / 4][r % 4] = acc;
  }
}

}  // namespace nsrhs
