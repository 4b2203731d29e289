// CPU oracle for the element-by-element Navier-Stokes RHS assembly on linear
// tetrahedra. TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU
// baseline of the benchmark call it; the library never does.
//
// Plain, serial, double precision (and std::complex<double> for complex-step
// derivatives). Every volume integral is evaluated with the 4-point rule at
// the Gauss points exactly as written in the weak form below: no algebraic
// restructuring, no fusion, no reordering. It shares no code, header or
// constant with the CUDA path.
//
// What is computed (the paper names the method but prints no formulas; the
// readings below are this library's definition of it):
//  * the RHS of the explicit momentum step of an incompressible LES
//    (Sec. II), plus the continuity residual;
//  * linear tetrahedra, 4 nodes, 4 Gauss points, shape-function gradients
//    constant per element (Sec. V-B);
//  * constant density rho and viscosity mu (Sec. V-B);
//  * Vreman eddy viscosity, one value per element from the constant velocity
//    gradient (Sec. V-B);
//  * the element RHS computed directly, without an element matrix (Sec. V-A);
//  * SUPG/PSPG stabilisation with tau = 1/(c1 mu_eff/h^2 + c2 rho |u|/h) per
//    Gauss point, h = detJ^(1/3).
// Variants (off by default): the skew-symmetric Galerkin convection
//   -rho/2 int[ N_a (u.grad)u_i - (u.grad N_a) u_i ]
// whose convective RHS does no work on the discrete velocity (the
// "energy-preserving" property named in Sec. II), and one tau per element
// evaluated with the element-mean velocity.
// For test function N_a of element e (volume V, u_h, p_h linear):
//   F_a,i = int[ -rho N_a (u.grad)u_i - mu_eff grad N_a . grad u_i + p dN_a/dx_i
//                - tau rho (u . grad N_a) (rho (u.grad)u_i + dp/dx_i) ]
//   F_a,4 = int[ -N_a div u - tau grad N_a . (rho (u.grad)u + grad p) ]
// and RHS[conn[a][e]][:] += F_a over all elements.
//
// Parity note: the formulation itself cannot be pinned to the paper's own
// numbers (none are printed for the discretisation); the tests pin this code
// to closed forms, invariants and brute-force checks instead.

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

struct Params {  // mirrors the layout passed from Python (7 doubles)
  double rho, mu, c_vreman, c1, c2;
  double skew;     // 0: convective form, 1: skew-symmetric (energy-preserving) form
  double tau_elem; // 0: tau at each Gauss point, 1: one tau per element (mean velocity)
};

inline double re(double x) { return x; }
inline double re(const std::complex<double>& x) { return x.real(); }

// 4-point Gauss rule on the tetrahedron (degree 2): point g has barycentric
// coordinate A on node g and B on the other three nodes, weight V/4.
const double SQRT5 = std::sqrt(5.0);
const double QA = (5.0 + 3.0 * SQRT5) / 20.0;
const double QB = (5.0 - SQRT5) / 20.0;

// Term selection bits (all set = full RHS).
enum : unsigned {
  T_CONV = 1u,    // Galerkin convection
  T_VISC = 2u,    // viscous
  T_PRES = 4u,    // pressure
  T_SUPG = 8u,    // momentum stabilisation
  T_CONT = 16u,   // Galerkin continuity
  T_PSPG = 32u,   // continuity stabilisation
  T_ALL = 63u
};

// One element. X[a][d]: node coordinates; U[a][k]: (u, v, w, p) at node a.
// Writes F[a][k]. Returns false if detJ <= 0.
template <class T>
bool element_rhs(const double X[4][3], const T U[4][4], const Params& P, unsigned terms,
                 T F[4][4]) {
  // Geometry: J = [X1-X0 | X2-X0 | X3-X0] (columns are edges).
  double J[3][3];
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) J[i][k] = X[k + 1][i] - X[0][i];
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
               J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  if (!(det > 0.0)) return false;
  // Inverse by the adjugate: Jinv[r][c] = cofactor(c, r) / det.
  double Ji[3][3];
  Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  // Shape-function gradients (constant on the element): N_k = xi_k for k=1..3,
  // so grad N_k = row k of J^-1; N_0 = 1 - xi_1 - xi_2 - xi_3.
  double dN[4][3];
  for (int j = 0; j < 3; ++j) {
    dN[1][j] = Ji[0][j];
    dN[2][j] = Ji[1][j];
    dN[3][j] = Ji[2][j];
    dN[0][j] = -(Ji[0][j] + Ji[1][j] + Ji[2][j]);
  }
  const double V = det / 6.0;
  const double h = std::cbrt(det);

  // Element gradients: G[i][j] = d u_i / d x_j, grad p.
  T G[3][3], gp[3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      G[i][j] = 0.0;
      for (int a = 0; a < 4; ++a) G[i][j] += U[a][i] * dN[a][j];
    }
  for (int j = 0; j < 3; ++j) {
    gp[j] = 0.0;
    for (int a = 0; a < 4; ++a) gp[j] += U[a][3] * dN[a][j];
  }
  T divu = G[0][0] + G[1][1] + G[2][2];

  // Vreman eddy viscosity (one value per element): alpha_ij = du_j/dx_i,
  // beta_ij = h^2 sum_m alpha_mi alpha_mj,
  // B = b11 b22 - b12^2 + b11 b33 - b13^2 + b22 b33 - b23^2,
  // nu_t = c * sqrt(B / (alpha_ij alpha_ij)), zero when either factor is not > 0.
  T mu_eff = P.mu;
  if (P.c_vreman != 0.0) {
    T al[3][3], be[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) al[i][j] = G[j][i];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        be[i][j] = 0.0;
        for (int m = 0; m < 3; ++m) be[i][j] += h * h * al[m][i] * al[m][j];
      }
    T Bb = be[0][0] * be[1][1] - be[0][1] * be[0][1] + be[0][0] * be[2][2] -
           be[0][2] * be[0][2] + be[1][1] * be[2][2] - be[1][2] * be[1][2];
    T A = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) A += al[i][j] * al[i][j];
    if (re(A) > 0.0 && re(Bb) > 0.0) mu_eff = P.mu + P.rho * (P.c_vreman * std::sqrt(Bb / A));
  }

  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 4; ++k) F[a][k] = 0.0;

  // Per-element tau (variant): mean nodal velocity.
  T tau_e = 0.0;
  if (P.tau_elem != 0.0) {
    T ub[3];
    for (int i = 0; i < 3; ++i) ub[i] = 0.25 * (U[0][i] + U[1][i] + U[2][i] + U[3][i]);
    T un = std::sqrt(ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2]);
    tau_e = 1.0 / (P.c1 * mu_eff / (h * h) + P.c2 * P.rho * un / h);
  }

  // Gauss-point loop: every integrand evaluated at xi_g, weight V/4.
  for (int g = 0; g < 4; ++g) {
    double N[4];
    for (int a = 0; a < 4; ++a) N[a] = (a == g) ? QA : QB;
    T ug[3], pg = 0.0;
    for (int i = 0; i < 3; ++i) {
      ug[i] = 0.0;
      for (int a = 0; a < 4; ++a) ug[i] += N[a] * U[a][i];
    }
    for (int a = 0; a < 4; ++a) pg += N[a] * U[a][3];
    T cg[3];  // (u . grad) u
    for (int i = 0; i < 3; ++i) {
      cg[i] = 0.0;
      for (int j = 0; j < 3; ++j) cg[i] += ug[j] * G[i][j];
    }
    T unorm = std::sqrt(ug[0] * ug[0] + ug[1] * ug[1] + ug[2] * ug[2]);
    T tau = 1.0 / (P.c1 * mu_eff / (h * h) + P.c2 * P.rho * unorm / h);
    if (P.tau_elem != 0.0) tau = tau_e;
    T r[3];  // strong momentum residual (the viscous part vanishes for P1)
    for (int i = 0; i < 3; ++i) r[i] = P.rho * cg[i] + gp[i];
    const double w = V / 4.0;
    for (int a = 0; a < 4; ++a) {
      T ugradNa = ug[0] * dN[a][0] + ug[1] * dN[a][1] + ug[2] * dN[a][2];
      for (int i = 0; i < 3; ++i) {
        T f = 0.0;
        if (terms & T_CONV) {
          if (P.skew != 0.0)
            f += -0.5 * P.rho * (N[a] * cg[i] - ugradNa * ug[i]);
          else
            f += -P.rho * N[a] * cg[i];
        }
        if (terms & T_VISC) {
          T gg = 0.0;
          for (int j = 0; j < 3; ++j) gg += dN[a][j] * G[i][j];
          f += -mu_eff * gg;
        }
        if (terms & T_PRES) f += pg * dN[a][i];
        if (terms & T_SUPG) f += -tau * P.rho * ugradNa * r[i];
        F[a][i] += w * f;
      }
      T f4 = 0.0;
      if (terms & T_CONT) f4 += -N[a] * divu;
      if (terms & T_PSPG) f4 += -tau * (dN[a][0] * r[0] + dN[a][1] * r[1] + dN[a][2] * r[2]);
      F[a][3] += w * f4;
    }
  }
  return true;
}

template <class T>
void gather(int64_t N, int64_t E, const double* coords, const int32_t* conn, const T* up,
            int64_t e, double X[4][3], T U[4][4]) {
  for (int a = 0; a < 4; ++a) {
    int64_t v = conn[a * E + e];
    for (int d = 0; d < 3; ++d) X[a][d] = coords[d * N + v];
    for (int k = 0; k < 4; ++k) U[a][k] = up[k * N + v];
  }
}

bool valid_index(int64_t N, int64_t E, const int32_t* conn) {
  for (int64_t i = 0; i < 4 * E; ++i)
    if (conn[i] < 0 || conn[i] >= N) return false;
  return true;
}

}  // namespace

extern "C" {

// Status codes: 0 ok, 1 bad arguments, 2 bad mesh (index out of range or detJ <= 0).

// Single element: X [4][3], U [4][4] (u,v,w,p per node), F [4][4] out.
int or_element_f64(const double* X, const double* U, const double* params, unsigned terms,
                   double* F) {
  Params P;
  std::memcpy(&P, params, sizeof(P));
  double Xa[4][3], Ua[4][4], Fa[4][4];
  std::memcpy(Xa, X, sizeof(Xa));
  std::memcpy(Ua, U, sizeof(Ua));
  if (!element_rhs<double>(Xa, Ua, P, terms, Fa)) return 2;
  std::memcpy(F, Fa, sizeof(Fa));
  return 0;
}

// Complex version (U = Ure + i Uim) for complex-step derivatives.
int or_element_c128(const double* X, const double* Ure, const double* Uim, const double* params,
                    unsigned terms, double* Fre, double* Fim) {
  Params P;
  std::memcpy(&P, params, sizeof(P));
  double Xa[4][3];
  std::memcpy(Xa, X, sizeof(Xa));
  std::complex<double> Ua[4][4], Fa[4][4];
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 4; ++k) Ua[a][k] = {Ure[4 * a + k], Uim[4 * a + k]};
  if (!element_rhs(Xa, Ua, P, terms, Fa)) return 2;
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 4; ++k) {
      Fre[4 * a + k] = Fa[a][k].real();
      Fim[4 * a + k] = Fa[a][k].imag();
    }
  return 0;
}

// Global assembly over elements [e0, e1): rhs [4][N] is ZEROED then summed
// in element order, then local node order.
int or_assemble_f64(int64_t N, int64_t E, const double* coords, const int32_t* conn,
                    const double* up, const double* params, unsigned terms, int64_t e0,
                    int64_t e1, double* rhs) {
  if (N <= 0 || E < 0 || !coords || !conn || !up || !params || !rhs) return 1;
  if (e0 < 0 || e1 > E || e0 > e1) return 1;
  if (!valid_index(N, E, conn)) return 2;
  Params P;
  std::memcpy(&P, params, sizeof(P));
  std::memset(rhs, 0, sizeof(double) * 4 * N);
  for (int64_t e = e0; e < e1; ++e) {
    double X[4][3], U[4][4], F[4][4];
    gather(N, E, coords, conn, up, e, X, U);
    if (!element_rhs(X, U, P, terms, F)) return 2;
    for (int a = 0; a < 4; ++a) {
      int64_t v = conn[a * E + e];
      for (int k = 0; k < 4; ++k) rhs[k * N + v] += F[a][k];
    }
  }
  return 0;
}

// Complex global assembly (complex step on the nodal fields).
int or_assemble_c128(int64_t N, int64_t E, const double* coords, const int32_t* conn,
                     const double* up_re, const double* up_im, const double* params,
                     unsigned terms, double* rhs_re, double* rhs_im) {
  if (N <= 0 || E < 0 || !coords || !conn || !up_re || !up_im || !params || !rhs_re || !rhs_im)
    return 1;
  if (!valid_index(N, E, conn)) return 2;
  Params P;
  std::memcpy(&P, params, sizeof(P));
  std::vector<std::complex<double>> up(4 * N), rhs(4 * N, 0.0);
  for (int64_t i = 0; i < 4 * N; ++i) up[i] = {up_re[i], up_im[i]};
  for (int64_t e = 0; e < E; ++e) {
    double X[4][3];
    std::complex<double> U[4][4], F[4][4];
    gather(N, E, coords, conn, up.data(), e, X, U);
    if (!element_rhs(X, U, P, terms, F)) return 2;
    for (int a = 0; a < 4; ++a) {
      int64_t v = conn[a * E + e];
      for (int k = 0; k < 4; ++k) rhs[k * N + v] += F[a][k];
    }
  }
  for (int64_t i = 0; i < 4 * N; ++i) {
    rhs_re[i] = rhs[i].real();
    rhs_im[i] = rhs[i].imag();
  }
  return 0;
}

// Vector-Jacobian product grad = (dRHS/d up)^T w, [4][N] each (grad ZEROED).
// Per element, the 16x16 Jacobian dF_e/dU_e is taken column by column by the
// complex step (Squire & Trapp 1998): F(U + i s e_bk) has imaginary part
// s dF/dU_bk up to O(s^2) with no subtractive cancellation; s = 1e-30.
// Then grad[conn[b]][k] += sum_{a,i} w[conn[a]][i] dF_ai/dU_bk.
int or_vjp_f64(int64_t N, int64_t E, const double* coords, const int32_t* conn, const double* up,
               const double* w, const double* params, double* grad) {
  if (N <= 0 || E < 0 || !coords || !conn || !up || !w || !params || !grad) return 1;
  if (!valid_index(N, E, conn)) return 2;
  Params P;
  std::memcpy(&P, params, sizeof(P));
  const double s = 1e-30;
  std::memset(grad, 0, sizeof(double) * 4 * N);
  for (int64_t e = 0; e < E; ++e) {
    double X[4][3], U0[4][4];
    gather(N, E, coords, conn, up, e, X, U0);
    double W[4][4];
    for (int a = 0; a < 4; ++a) {
      int64_t v = conn[a * E + e];
      for (int k = 0; k < 4; ++k) W[a][k] = w[k * N + v];
    }
    for (int b = 0; b < 4; ++b)
      for (int k = 0; k < 4; ++k) {
        std::complex<double> U[4][4], F[4][4];
        for (int a = 0; a < 4; ++a)
          for (int q = 0; q < 4; ++q) U[a][q] = U0[a][q];
        U[b][k] += std::complex<double>(0.0, s);
        if (!element_rhs(X, U, P, T_ALL, F)) return 2;
        double acc = 0.0;
        for (int a = 0; a < 4; ++a)
          for (int i = 0; i < 4; ++i) acc += W[a][i] * (F[a][i].imag() / s);
        grad[k * N + conn[b * E + e]] += acc;
      }
  }
  return 0;
}

// detJ of every element (for mesh checks): det [E].
int or_detj(int64_t N, int64_t E, const double* coords, const int32_t* conn, double* det) {
  if (!valid_index(N, E, conn)) return 2;
  for (int64_t e = 0; e < E; ++e) {
    double X[4][3];
    for (int a = 0; a < 4; ++a)
      for (int d = 0; d < 3; ++d) X[a][d] = coords[d * N + conn[a * E + e]];
    double J[3][3];
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k) J[i][k] = X[k + 1][i] - X[0][i];
    det[e] = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
             J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
             J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  }
  return 0;
}

}  // extern "C"
