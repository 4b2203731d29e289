// Per-element arithmetic of the tetrahedral Navier-Stokes RHS (device code).
//
// The element RHS is the stabilised P1 weak form (Sec. II, V-A, V-B):
//   F_a,i = int[ -rho N_a (u.grad)u_i - mu_eff grad N_a.grad u_i + p dN_a/dx_i
//                - tau rho (u.grad N_a)(rho (u.grad)u_i + dp/dx_i) ]
//   F_a,4 = int[ -N_a div u - tau grad N_a.(rho (u.grad)u + grad p) ]
// with the 4-point rule (barycentric QA on node g, QB elsewhere, weight V/4),
// tau_g = 1/(c1 mu_eff/h^2 + c2 rho |u_g|/h), h = detJ^(1/3), and Vreman's
// eddy viscosity from the constant velocity gradient (Sec. V-B).
//
// This file evaluates that form RESTRUCTURED for short intermediate lifetimes
// (Sec. V-A) and specialised to linear tets (Sec. V-B); it is exactly the
// same function up to rounding. With the unscaled cofactor vectors
// c_k = e_{k+1} x e_{k+2} of the edge vectors e_k = X_k - X_0 (so that
// grad N_k = c_k / detJ, c_0 = -(c_1 + c_2 + c_3)):
//   Gh = sum_a u_a c_a^T   (= detJ grad u),   gph = sum_a p_a c_a (= detJ grad p)
//   Galerkin convection: sum_g N_a(xi_g) N_b(xi_g) = (1 + delta_ab)/5 turns the
//     Gauss sum into -(rho/120) Gh (S_u + u_a), S_u = sum_b u_b;
//   tau enters only through  stau = sum_g tau_g,  T = sum_g tau_g u_g,
//     Q = sum_g tau_g u_g u_g^T  (4 square roots and 4 reciprocals in total);
//   viscous + pressure + SUPG momentum = K c_a with
//     K = (p_bar/6) I - (1/(6 detJ)) [Gh (mu_eff I + rho^2/4 Q) + rho/4 gph T^T];
//   continuity = -(tr Gh)/24 - c_a . (rho Gh T + stau gph) / (24 detJ).
// The reverse (vector-Jacobian) sweep of exactly this sequence is
// element_vjp below; it recomputes the forward quantities instead of storing
// them.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fastmath.cuh"

namespace nsrhs {

// 4-point degree-2 Gauss rule on the tet: QA = (5 + 3 sqrt 5)/20, QB = (5 - sqrt 5)/20.
constexpr double kQA = 0.58541019662496845446;
constexpr double kQB = 0.13819660112501051518;

template <class R>
struct ElemParams {
  R rho, mu, c_vreman, c1, c2;
};

// Formulation flags (template parameter of the element routines).
constexpr int kVreman = 1;    // Vreman eddy viscosity on
constexpr int kSkew = 2;      // skew-symmetric (energy-preserving) Galerkin convection
constexpr int kTauElem = 4;   // one tau per element from the mean velocity

// a * b + c as one fused multiply-add (so that the FP64 instruction count is
// what the source says; the generic form serves the host flop census).
template <class R>
__device__ __forceinline__ R fmac(R a, R b, R c) {
  return a * b + c;
}
#if defined(__CUDA_ARCH__)
template <>
__device__ __forceinline__ double fmac<double>(double a, double b, double c) {
  return __fma_rn(a, b, c);
}
template <>
__device__ __forceinline__ float fmac<float>(float a, float b, float c) {
  return __fmaf_rn(a, b, c);
}
#endif

template <class R>
struct MathOps;

// Double precision: seed + one cubic correction (fastmath.cuh). Arguments
// are positive (reciprocals, cube roots) or non-negative (square roots).
template <>
struct MathOps<double> {
  static __device__ __forceinline__ double rcp(double x) { return rcp_pos(x); }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt_nonneg(x); }
  static __device__ __forceinline__ double rcbrt_(double x) { return rcbrt_pos(x); }
  static __device__ __forceinline__ double rsqrt_(double x) { return rsqrt_nonneg(x); }
};

// Single precision (the mixed form): the special-function unit's
// approximations (relative error about 2^-22 to 2^-23), far inside the mixed
// form's accuracy, one instruction each instead of a correctly rounded
// sequence. Arguments as for double.
template <>
struct MathOps<float> {
#if defined(__CUDA_ARCH__)
  static __device__ __forceinline__ float rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  }
  static __device__ __forceinline__ float sqrt_(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  }
  static __device__ __forceinline__ float rsqrt_(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return x > 0.0f ? y : 0.0f;
  }
#else
  static float rcp(float x) { return 1.0f / x; }
  static float sqrt_(float x) { return sqrtf(x); }
  static float rsqrt_(float x) { return x > 0.0f ? 1.0f / sqrtf(x) : 0.0f; }
#endif
  static __device__ __forceinline__ float rcbrt_(float x) { return rcbrtf(x); }
};

// Element geometry from the edge vectors e[k] = X_{k+1} - X_0: unscaled
// cofactor vectors c[k] (k = 0..2 for nodes 1..3), 1/detJ and
// 1/h = detJ^(-1/3); cofactors and determinant in GR, stored as R.
template <class R, class GR>
__device__ __forceinline__ void element_geometry_from_edges(const GR e[3][3], R c[3][3],
                                                            R& inv_det, R& rh,
                                                            double* det_out = nullptr) {
  GR cc[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const GR* a = e[(k + 1) % 3];
    const GR* b = e[(k + 2) % 3];
    cc[k][0] = a[1] * b[2] - a[2] * b[1];
    cc[k][1] = a[2] * b[0] - a[0] * b[2];
    cc[k][2] = a[0] * b[1] - a[1] * b[0];
  }
  GR det = e[0][0] * cc[0][0] + e[0][1] * cc[0][1] + e[0][2] * cc[0][2];
  if (det_out) *det_out = (double)det;
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int d = 0; d < 3; ++d) c[k][d] = (R)cc[k][d];
  inv_det = (R)MathOps<GR>::rcp(det);
  rh = (R)MathOps<GR>::rcbrt_(det);
}

// Element geometry from node coordinates X (edges formed in XT, then GR).
template <class R, class GR, class XT = double>
__device__ __forceinline__ void element_geometry(const XT X[4][3], R c[3][3], R& inv_det, R& rh,
                                                 double* det_out = nullptr) {
  GR e[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int d = 0; d < 3; ++d) e[k][d] = (GR)(X[k + 1][d] - X[0][d]);
  element_geometry_from_edges<R, GR>(e, c, inv_det, rh, det_out);
}

// The element's 16 outputs from its gradients and Gauss-point accumulators:
// K (viscous + pressure + SUPG momentum), Rs (continuity's PSPG part) and the
// Galerkin convection, as described at the top of this file. Qv and Pv are
// the symmetric 3x3 matrices Q = sum tau_g u_g u_g^T and P = sum u_g u_g^T
// as (00, 11, 22, 01, 02, 12); P is read only in the skew-symmetric form.
template <class R, int FLAGS>
__device__ __forceinline__ void element_outputs(const R c[3][3], R inv_det, const R u[4][3],
                                                const R G[3][3], const R gp[3], const R S[3],
                                                R psum, R trG, R mu_eff, R stau, const R T[3],
                                                const R Qv[6], const R Pv[6],
                                                const ElemParams<R>& P, R F[4][4]) {
  constexpr bool SKEW = (FLAGS & kSkew) != 0;
  const R Q00 = Qv[0], Q11 = Qv[1], Q22 = Qv[2], Q01 = Qv[3], Q02 = Qv[4], Q12 = Qv[5];
  const R P00 = Pv[0], P11 = Pv[1], P22 = Pv[2], P01 = Pv[3], P02 = Pv[4], P12 = Pv[5];
  // K = pbar/6 I - inv_det/6 [Gh (mu_eff I + rho^2/4 Q) + rho/4 gph T^T], with the
  // scalar factors folded into Qp and sTT before the 3x3 product so that each
  // entry is one chain of fused multiply-adds. a2, a1 and b4 come from
  // s24 = inv_det/24 (exactly inv_det/6 scaled by 1/4, so they equal
  // -(inv_det/6) (rho^2/4), -(inv_det/6) mu_eff and -(inv_det/6) (rho/4)).
  const R s24 = inv_det * (R)(1.0 / 24.0);
  const R a2 = s24 * -(P.rho * P.rho);
  const R a1 = s24 * ((R)-4 * mu_eff);
  const R b4 = s24 * -P.rho;
  const R Qp[3][3] = {{fmac(a2, Q00, a1), a2 * Q01, a2 * Q02},
                      {a2 * Q01, fmac(a2, Q11, a1), a2 * Q12},
                      {a2 * Q02, a2 * Q12, fmac(a2, Q22, a1)}};
  const R pb6 = psum * (R)(1.0 / 24.0);
  const R Pm[3][3] = {{P00, P01, P02}, {P01, P11, P12}, {P02, P12, P22}};
  const R r48 = P.rho * (R)(1.0 / 48.0);
  // sTT = (inv_det/24) rho T = -b4 T serves both the continuity's Rs and
  // K's b4 gph T^T term (as -gph sTT^T)
  R sTT[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) sTT[j] = -b4 * T[j];
  R K[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      R acc = (i == j) ? fmac(-gp[i], sTT[j], pb6) : -gp[i] * sTT[j];
      if constexpr (SKEW) acc = fmac(r48, Pm[i][j], acc);
      acc = fmac(G[i][0], Qp[0][j], acc);
      acc = fmac(G[i][1], Qp[1][j], acc);
      K[i][j] = fmac(G[i][2], Qp[2][j], acc);
    }
  }
  // Rs = inv_det/24 (rho Gh T + stau gph)
  const R sg = s24 * stau;
  R Rs[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R acc = sg * gp[i];
    acc = fmac(sTT[0], G[i][0], acc);
    acc = fmac(sTT[1], G[i][1], acc);
    Rs[i] = fmac(sTT[2], G[i][2], acc);
  }
  const R cont0 = trG * (R)(-1.0 / 24.0);
  // Galerkin convection -(rho/120) Gh (S_u + u_a) = Gh v_a, v_a = m120 u_a + m120 S_u
  // (halved in the skew-symmetric form)
  const R m120 = P.rho * (R)(SKEW ? -1.0 / 240.0 : -1.0 / 120.0);
  R mS[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) mS[i] = m120 * S[i];
  R ysum[3] = {(R)0, (R)0, (R)0};
  R csum = (R)0;
#pragma unroll
  for (int a = 1; a < 4; ++a) {
    const R* ca = c[a - 1];
    R v[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i] = fmac(m120, u[a][i], mS[i]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const R y = fmac(K[i][2], ca[2], fmac(K[i][1], ca[1], K[i][0] * ca[0]));
      ysum[i] += y;
      F[a][i] = fmac(G[i][2], v[2], fmac(G[i][1], v[1], fmac(G[i][0], v[0], y)));
    }
    F[a][3] = fmac(-ca[2], Rs[2], fmac(-ca[1], Rs[1], fmac(-ca[0], Rs[0], cont0)));
    csum += F[a][3];
  }
  {
    R v[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i] = fmac(m120, u[0][i], mS[i]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
      F[0][i] = fmac(G[i][2], v[2], fmac(G[i][1], v[1], fmac(G[i][0], v[0], -ysum[i])));
    // sum_a c_a = 0: the continuity entries sum to 4 cont0
    F[0][3] = fmac((R)4, cont0, -csum);
  }
}

// Where an element routine takes the nodal velocities u (and, in the
// reverse sweep, the cotangent w) from again at its phase boundaries:
// NoReload keeps the values it was given; a caller that holds them in shared
// memory can re-read them there instead, so that they are not live in
// registers across the whole routine (the block kernels fit their register
// caps that way). f: where the one-pass routine hands its element RHS once
// it is complete (before the reverse part); NoReload leaves it in F for the
// caller, a block kernel stores it to shared memory at once so that F is
// not live across the reverse sweep.
struct NoReload {
  template <class R>
  __device__ __forceinline__ void u(R (&)[4][3]) const {}
  template <class R>
  __device__ __forceinline__ void w(R (&)[4][4]) const {}
  template <class R>
  __device__ __forceinline__ void f(const R (*)[4]) const {}
};

// Forward element RHS. u[a][i], p[a] nodal values; F[a][0..2] momentum,
// F[a][3] continuity. FLAGS: kVreman | kSkew | kTauElem.
// Skew-symmetric variant: the Galerkin convection becomes
// -rho/2 int[N_a (u.grad)u_i - (u.grad N_a) u_i]: half the convective term plus
// (rho/48) P c_a with P = sum_g u_g u_g^T, folded into K.
// Per-element tau: tau from |S_u/4|; then sum_g tau = 4 tau, T = tau S_u
// (sum_g u_g = S_u) and Q = tau P.
// RL: u again before the element outputs (see NoReload).
template <class R, int FLAGS, class RL = NoReload>
__device__ __forceinline__ void element_rhs(const R c[3][3], R inv_det, R rh, const R u_in[4][3],
                                            const R p[4], const ElemParams<R>& P, R F[4][4],
                                            const RL& rl = RL()) {
  R u[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) u[a][i] = u_in[a][i];
  using M = MathOps<R>;
  constexpr bool VREMAN = (FLAGS & kVreman) != 0;
  constexpr bool SKEW = (FLAGS & kSkew) != 0;
  constexpr bool TAUE = (FLAGS & kTauElem) != 0;
  // Gh = sum_k (u_k - u_0) c_k^T, gph = sum_k (p_k - p_0) c_k
  R G[3][3], gp[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const R d1 = u[1][i] - u[0][i], d2 = u[2][i] - u[0][i], d3 = u[3][i] - u[0][i];
#pragma unroll
    for (int j = 0; j < 3; ++j) G[i][j] = fmac(d3, c[2][j], fmac(d2, c[1][j], d1 * c[0][j]));
  }
  {
    const R d1 = p[1] - p[0], d2 = p[2] - p[0], d3 = p[3] - p[0];
#pragma unroll
    for (int j = 0; j < 3; ++j) gp[j] = fmac(d3, c[2][j], fmac(d2, c[1][j], d1 * c[0][j]));
  }
  R S[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) S[i] = (u[0][i] + u[1][i]) + (u[2][i] + u[3][i]);
  const R psum = (p[0] + p[1]) + (p[2] + p[3]);
  const R trG = G[0][0] + G[1][1] + G[2][2];

  R mu_eff = P.mu;
  if constexpr (VREMAN) {
    // alpha = G^T, beta = h^2 G G^T; B and A from Gh, rescaled by detJ and h.
    R bm[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j)
        bm[i][j] = fmac(G[i][2], G[j][2], fmac(G[i][1], G[j][1], G[i][0] * G[j][0]));
    const R A = (bm[0][0] + bm[1][1]) + bm[2][2];
    R B = fmac(bm[1][1], bm[2][2], -(bm[1][2] * bm[1][2]));
    B = fmac(bm[0][0], bm[2][2], fmac(-bm[0][2], bm[0][2], B));
    B = fmac(bm[0][0], bm[1][1], fmac(-bm[0][1], bm[0][1], B));
    if (A > (R)0 && B > (R)0) {
      // nu_t = c h^2 sqrt(B_G/A_G) = c h^2 inv_det sqrt(B/A), and with
      // h = detJ^(1/3), h^2 inv_det = detJ^(-1/3) = rh
      mu_eff = fmac(P.rho * P.c_vreman, rh * M::sqrt_(B * M::rcp(A)), P.mu);
    }
  }
  const R k1 = (P.c1 * mu_eff) * (rh * rh);
  const R k2 = (P.c2 * P.rho) * rh;

  // Gauss points: u_g = QB S_u + (QA - QB) u_g-node.
  R stau = (R)0, T[3] = {(R)0, (R)0, (R)0};
  R Q00 = 0, Q11 = 0, Q22 = 0, Q01 = 0, Q02 = 0, Q12 = 0;
  R P00 = 0, P11 = 0, P22 = 0, P01 = 0, P02 = 0, P12 = 0;  // sum_g u_g u_g^T
  R bS[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) bS[i] = (R)kQB * S[i];
  R tau_e = (R)0;
  if constexpr (TAUE) {
    const R sm = fmac(S[2], S[2], fmac(S[1], S[1], S[0] * S[0])) * (R)0.0625;
    tau_e = M::rcp(fmac(k2, M::sqrt_(sm), k1));
  }
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    R ug[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) ug[i] = fmac((R)(kQA - kQB), u[g][i], bS[i]);
    if constexpr (!TAUE) {
      const R s = fmac(ug[2], ug[2], fmac(ug[1], ug[1], ug[0] * ug[0]));
      const R tau = M::rcp(fmac(k2, M::sqrt_(s), k1));
      stau += tau;
      R tu[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        tu[i] = tau * ug[i];
        T[i] += tu[i];
      }
      Q00 = fmac(tu[0], ug[0], Q00);
      Q11 = fmac(tu[1], ug[1], Q11);
      Q22 = fmac(tu[2], ug[2], Q22);
      Q01 = fmac(tu[0], ug[1], Q01);
      Q02 = fmac(tu[0], ug[2], Q02);
      Q12 = fmac(tu[1], ug[2], Q12);
    }
    if constexpr (SKEW || TAUE) {
      P00 = fmac(ug[0], ug[0], P00);
      P11 = fmac(ug[1], ug[1], P11);
      P22 = fmac(ug[2], ug[2], P22);
      P01 = fmac(ug[0], ug[1], P01);
      P02 = fmac(ug[0], ug[2], P02);
      P12 = fmac(ug[1], ug[2], P12);
    }
  }
  if constexpr (TAUE) {
    stau = (R)4 * tau_e;
#pragma unroll
    for (int i = 0; i < 3; ++i) T[i] = tau_e * S[i];
    Q00 = tau_e * P00;
    Q11 = tau_e * P11;
    Q22 = tau_e * P22;
    Q01 = tau_e * P01;
    Q02 = tau_e * P02;
    Q12 = tau_e * P12;
  }
  const R Qv[6] = {Q00, Q11, Q22, Q01, Q02, Q12};
  const R Pv[6] = {P00, P11, P22, P01, P02, P12};
  rl.u(u);
  element_outputs<R, FLAGS>(c, inv_det, u, G, gp, S, psum, trG, mu_eff, stau, T, Qv, Pv, P, F);
}

// Reverse sweep: given w[a][0..3] (cotangent of F[a][0..3]), returns
// gu[a][i] = sum_{b,k} w[b][k] dF[b][k]/du[a][i] and gpo[a] likewise for p.
// It differentiates exactly the sequence of element_rhs (same intermediates),
// recomputing the forward quantities; every product is written as a chain of
// fused multiply-adds.
//
// WITH_F: also write the element's forward outputs F (element_outputs) from
// the recomputed intermediates, so that one pass yields the RHS entries and
// the vector-Jacobian product at the same state.
//
// RL: where the nodal velocities u and the cotangent w come from again at
// three points of the sweep (before the reverse part, before Gbar, before the
// final gradient; see NoReload).

template <class R, int FLAGS, bool WITH_F, class RL = NoReload>
__device__ __forceinline__ void element_vjp_impl(const R c[3][3], R inv_det, R rh,
                                                 const R u_in[4][3], const R p[4],
                                                 const R w_in[4][4], const ElemParams<R>& P,
                                                 R gu[4][3], R gpo[4], R (*F)[4],
                                                 const RL& rl = RL()) {
  R u[4][3], w[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int i = 0; i < 3; ++i) u[a][i] = u_in[a][i];
#pragma unroll
    for (int k = 0; k < 4; ++k) w[a][k] = w_in[a][k];
  }
  using M = MathOps<R>;
  constexpr bool VREMAN = (FLAGS & kVreman) != 0;
  constexpr bool SKEW = (FLAGS & kSkew) != 0;
  constexpr bool TAUE = (FLAGS & kTauElem) != 0;
  // ---- forward recompute ----
  R G[3][3], gp[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const R d1 = u[1][i] - u[0][i], d2 = u[2][i] - u[0][i], d3 = u[3][i] - u[0][i];
#pragma unroll
    for (int j = 0; j < 3; ++j) G[i][j] = fmac(d3, c[2][j], fmac(d2, c[1][j], d1 * c[0][j]));
  }
  {
    const R d1 = p[1] - p[0], d2 = p[2] - p[0], d3 = p[3] - p[0];
#pragma unroll
    for (int j = 0; j < 3; ++j) gp[j] = fmac(d3, c[2][j], fmac(d2, c[1][j], d1 * c[0][j]));
  }
  R S[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) S[i] = (u[0][i] + u[1][i]) + (u[2][i] + u[3][i]);

  R mu_eff = P.mu;
  R vA = (R)0, vphi = (R)0, vscale = (R)0;  // Vreman intermediates
  R b00 = (R)0, b11 = (R)0, b22 = (R)0, b01 = (R)0, b02 = (R)0, b12 = (R)0;
  bool vactive = false;
  if constexpr (VREMAN) {
    b00 = G[0][0] * G[0][0] + G[0][1] * G[0][1] + G[0][2] * G[0][2];
    b11 = G[1][0] * G[1][0] + G[1][1] * G[1][1] + G[1][2] * G[1][2];
    b22 = G[2][0] * G[2][0] + G[2][1] * G[2][1] + G[2][2] * G[2][2];
    b01 = G[0][0] * G[1][0] + G[0][1] * G[1][1] + G[0][2] * G[1][2];
    b02 = G[0][0] * G[2][0] + G[0][1] * G[2][1] + G[0][2] * G[2][2];
    b12 = G[1][0] * G[2][0] + G[1][1] * G[2][1] + G[1][2] * G[2][2];
    vA = (b00 + b11) + b22;
    R vB = b00 * b11 - b01 * b01 + b00 * b22 - b02 * b02 + b11 * b22 - b12 * b12;
    if (vA > (R)0 && vB > (R)0) {
      vactive = true;
      vscale = (P.rho * P.c_vreman) * rh;  // rho c h^2 inv_det = rho c detJ^(-1/3)
      vphi = M::sqrt_(vB * M::rcp(vA));
      mu_eff = P.mu + vscale * vphi;
    }
  }
  const R rh2 = rh * rh;
  const R k1 = (P.c1 * mu_eff) * rh2;
  const R k2 = (P.c2 * P.rho) * rh;
  R bS[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) bS[i] = (R)kQB * S[i];
  R tau[4], kyr[4];  // tau_g and k2/|u_g| (0 where u_g = 0)
  R stau = (R)0, T[3] = {(R)0, (R)0, (R)0};
  R Q00 = (R)0, Q11 = (R)0, Q22 = (R)0, Q01 = (R)0, Q02 = (R)0, Q12 = (R)0;
  R P00 = (R)0, P11 = (R)0, P22 = (R)0, P01 = (R)0, P02 = (R)0, P12 = (R)0;
  R tau_e = (R)0, yr_e = (R)0;  // per-element tau and 1/|S_u/4|
  if constexpr (TAUE) {
    const R sm = fmac(S[2], S[2], fmac(S[1], S[1], S[0] * S[0])) * (R)0.0625;
    yr_e = M::rsqrt_(sm);
    tau_e = M::rcp(fmac(k2, sm * yr_e, k1));
  }
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    R ug[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) ug[i] = fmac((R)(kQA - kQB), u[g][i], bS[i]);
    if constexpr (!TAUE) {
      const R s = fmac(ug[2], ug[2], fmac(ug[1], ug[1], ug[0] * ug[0]));
      // k2 |u_g| = (k2 / |u_g|) s: the reverse sweep reuses k2 / |u_g|
      kyr[g] = k2 * M::rsqrt_(s);
      tau[g] = M::rcp(fmac(kyr[g], s, k1));
      stau += tau[g];
      R tu[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        tu[i] = tau[g] * ug[i];
        T[i] += tu[i];
      }
      Q00 = fmac(tu[0], ug[0], Q00);
      Q11 = fmac(tu[1], ug[1], Q11);
      Q22 = fmac(tu[2], ug[2], Q22);
      Q01 = fmac(tu[0], ug[1], Q01);
      Q02 = fmac(tu[0], ug[2], Q02);
      Q12 = fmac(tu[1], ug[2], Q12);
    }
    if constexpr (TAUE || (WITH_F && SKEW)) {
      P00 = fmac(ug[0], ug[0], P00);
      P11 = fmac(ug[1], ug[1], P11);
      P22 = fmac(ug[2], ug[2], P22);
      P01 = fmac(ug[0], ug[1], P01);
      P02 = fmac(ug[0], ug[2], P02);
      P12 = fmac(ug[1], ug[2], P12);
    }
  }
  if constexpr (TAUE) {
    stau = (R)4 * tau_e;
#pragma unroll
    for (int i = 0; i < 3; ++i) T[i] = tau_e * S[i];
    Q00 = tau_e * P00;
    Q11 = tau_e * P11;
    Q22 = tau_e * P22;
    Q01 = tau_e * P01;
    Q02 = tau_e * P02;
    Q12 = tau_e * P12;
  }

  if constexpr (WITH_F) {
    const R Qv[6] = {Q00, Q11, Q22, Q01, Q02, Q12};
    const R Pv[6] = {P00, P11, P22, P01, P02, P12};
    const R psum = (p[0] + p[1]) + (p[2] + p[3]);
    const R trG = G[0][0] + G[1][1] + G[2][2];
    element_outputs<R, FLAGS>(c, inv_det, u, G, gp, S, psum, trG, mu_eff, stau, T, Qv, Pv, P, F);
    rl.f(F);
  }

  // ---- reverse ----
  rl.w(w);
  // Omega = sum_a wm_a c_a^T and cw = sum_a wc_a c_a, with c_0 = -(c_1 + c_2 + c_3)
  R Om[3][3], cw[3];
  {
    R dw[3][4];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int q = 0; q < 4; ++q) dw[k][q] = w[k + 1][q] - w[0][q];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        Om[i][j] = fmac(dw[2][i], c[2][j], fmac(dw[1][i], c[1][j], dw[0][i] * c[0][j]));
#pragma unroll
    for (int j = 0; j < 3; ++j)
      cw[j] = fmac(dw[2][3], c[2][j], fmac(dw[1][3], c[1][j], dw[0][3] * c[0][j]));
  }
  const R wcs = (w[0][3] + w[1][3]) + (w[2][3] + w[3][3]);
  const R s24 = inv_det * (R)(1.0 / 24.0);
  const R s6 = (R)4 * s24;  // = inv_det/6 exactly
  const R a1 = s24 * ((R)-4 * mu_eff);
  const R a2 = s24 * -(P.rho * P.rho);
  const R b4 = s24 * -P.rho;
  // Rbar = -(inv_det/24) cw is not formed: it enters as stau Rbar
  // (-s24 stau cw), Rbar . gph, rho G^T Rbar = b4 G^T cw and rho Rbar T^T =
  // cw (b4 T)^T, since b4 = -rho inv_det/24
  // pressure mean: pbar-bar / 4 = tr(Omega)/24
  const R pq = (Om[0][0] + Om[1][1] + Om[2][2]) * (R)(1.0 / 24.0);
  // mu_eff-bar = <Wbar, G> with Wbar = -(inv_det/6) Omega
  R mub;
  {
    R acc = Om[0][0] * G[0][0];
#pragma unroll
    for (int q = 1; q < 9; ++q) acc = fmac(Om[q / 3][q % 3], G[q / 3][q % 3], acc);
    mub = -s6 * acc;
  }
  // Qbar = a2 G^T Omega; Qh = (Qbar + Qbar^T)/2, its symmetric part, built
  // entry by entry (Q is symmetric, so only Qh matters)
  R Qh[3][3];
  {
    const R a2h = (R)0.5 * a2;
#pragma unroll
    for (int i = 0; i < 3; ++i)
      Qh[i][i] = a2 * fmac(G[2][i], Om[2][i], fmac(G[1][i], Om[1][i], G[0][i] * Om[0][i]));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i + 1; j < 3; ++j) {
        R acc = G[0][i] * Om[0][j];
        acc = fmac(G[0][j], Om[0][i], acc);
        acc = fmac(G[1][i], Om[1][j], acc);
        acc = fmac(G[1][j], Om[1][i], acc);
        acc = fmac(G[2][i], Om[2][j], acc);
        acc = fmac(G[2][j], Om[2][i], acc);
        Qh[i][j] = Qh[j][i] = a2h * acc;
      }
  }
  // Tbar = b4 (Omega^T gph + G^T cw) ; staubar = Rbar . gph ; gpbar = Omega (b4 T) + stau Rbar
  R Tb[3], gpb[3], bT[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) bT[i] = b4 * T[i];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    R acc = Om[0][j] * gp[0];
    acc = fmac(Om[1][j], gp[1], acc);
    acc = fmac(Om[2][j], gp[2], acc);
    acc = fmac(G[0][j], cw[0], acc);
    acc = fmac(G[1][j], cw[1], acc);
    Tb[j] = b4 * fmac(G[2][j], cw[2], acc);
  }
  {
    const R sRb = -s24 * stau;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      R acc = sRb * cw[i];
      acc = fmac(Om[i][0], bT[0], acc);
      acc = fmac(Om[i][1], bT[1], acc);
      gpb[i] = fmac(Om[i][2], bT[2], acc);
    }
  }
  const R staub = -s24 * fmac(cw[2], gp[2], fmac(cw[1], gp[1], cw[0] * gp[0]));
  // Gbar = Omega Qp' + rho Rbar T^T + sum_a wm_a v_a^T - (sum_a wc_a)/24 I,
  // Qp' = a2 Q + a1 I, v_a = -(rho/120)(u_a + S_u)
  rl.u(u);
  rl.w(w);
  R Gb[3][3];
  {
    const R Qp[3][3] = {{fmac(a2, Q00, a1), a2 * Q01, a2 * Q02},
                        {a2 * Q01, fmac(a2, Q11, a1), a2 * Q12},
                        {a2 * Q02, a2 * Q12, fmac(a2, Q22, a1)}};
    const R m120 = P.rho * (R)(SKEW ? -1.0 / 240.0 : -1.0 / 120.0);
    R v[4][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const R mS = m120 * S[j];
#pragma unroll
      for (int a = 0; a < 4; ++a) v[a][j] = fmac(m120, u[a][j], mS);
    }
    const R wc24 = wcs * (R)(1.0 / 24.0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        R acc = (i == j) ? fmac(cw[i], bT[j], -wc24) : cw[i] * bT[j];
        acc = fmac(Om[i][0], Qp[0][j], acc);
        acc = fmac(Om[i][1], Qp[1][j], acc);
        acc = fmac(Om[i][2], Qp[2][j], acc);
        acc = fmac(w[0][i], v[0][j], acc);
        acc = fmac(w[1][i], v[1][j], acc);
        acc = fmac(w[2][i], v[2][j], acc);
        Gb[i][j] = fmac(w[3][i], v[3][j], acc);
      }
  }
  // Gauss points in reverse: ugb_g = dL/du_g
  R ugb[4][3];
  R Usum[3] = {(R)0, (R)0, (R)0};
  const R crh2 = P.c1 * rh2;
  // skew-symmetric convection: K += (rho/48) P, P = sum_g u_g u_g^T, so
  // d/du_g <Omega, (rho/48) P> = (rho/48) (Omega + Omega^T) u_g
  R Os[3][3];
  if constexpr (SKEW) {
    const R r48 = P.rho * (R)(1.0 / 48.0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Os[i][j] = r48 * (Om[i][j] + Om[j][i]);
  }
  R Sb_tau[3] = {(R)0, (R)0, (R)0};  // S_u-bar from the per-element tau
  if constexpr (TAUE) {
    // tau-bar = 4 staub + Tb . S + <Qbar, P> ; T = tau S ; Q = tau P
    const R Pm[3][3] = {{P00, P01, P02}, {P01, P11, P12}, {P02, P12, P22}};
    R taub = (R)4 * staub;
#pragma unroll
    for (int i = 0; i < 3; ++i) taub = Tb[i] * S[i] + taub;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) taub = fmac(Qh[i][j], Pm[i][j], taub);
    const R db = -(tau_e * tau_e) * taub;
    mub = crh2 * db + mub;
    // |S_u/4| = sqrt(S.S/16): d/dS = S / (16 |S_u/4|)
    const R sc = (k2 * db) * (yr_e * (R)0.0625);
#pragma unroll
    for (int i = 0; i < 3; ++i) Sb_tau[i] = tau_e * Tb[i] + sc * S[i];
  }
  const R te2 = (R)2 * tau_e;
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    R ug[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) ug[i] = fmac((R)(kQA - kQB), u[g][i], bS[i]);
    if constexpr (!TAUE) {
      // T and Q enter as tau (Tb . u_g + u_g^T Qh u_g): with QT = Tb + Qh u_g,
      // tau-bar = staub + u_g . QT and the tau-weighted part of u_g-bar is
      // tau (Tb + 2 Qh u_g) = tau (2 QT - Tb)
      R QT[3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
        QT[i] = fmac(Qh[i][2], ug[2], fmac(Qh[i][1], ug[1], fmac(Qh[i][0], ug[0], Tb[i])));
      const R taub = fmac(ug[2], QT[2], fmac(ug[1], QT[1], fmac(ug[0], QT[0], staub)));
      const R db = -(tau[g] * tau[g]) * taub;  // d(1/d)
      mub = fmac(crh2, db, mub);
      const R sc = kyr[g] * db;                 // d|u_g| / du_g = u_g / |u_g|
#pragma unroll
      for (int i = 0; i < 3; ++i)
        ugb[g][i] = fmac(tau[g], fmac((R)2, QT[i], -Tb[i]), sc * ug[i]);
    } else {
      // Q = tau P: d/du_g <Qbar, tau P> = 2 tau Qh u_g
#pragma unroll
      for (int i = 0; i < 3; ++i)
        ugb[g][i] = te2 * fmac(Qh[i][2], ug[2], fmac(Qh[i][1], ug[1], Qh[i][0] * ug[0]));
    }
    if constexpr (SKEW) {
#pragma unroll
      for (int i = 0; i < 3; ++i)
        ugb[g][i] = Os[i][0] * ug[0] + (Os[i][1] * ug[1] + (Os[i][2] * ug[2] + ugb[g][i]));
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) Usum[i] += ugb[g][i];
  }
  // Vreman: mu_eff = mu + vscale phi, phi = sqrt(B/A):
  // d phi / d Gh = (P - phi^2 I) Gh / (phi A), P = tr(beta) I - beta, tr(beta) = A;
  // Gbar += f (P - phi^2 I) Gh with f = mub vscale / (phi A) folded into the
  // matrix, so that each entry is one FMA chain
  if (VREMAN && vactive) {
    const R f = mub * vscale * M::rcp(vphi * vA);
    const R t = f * (vA - vphi * vphi);
    const R fb01 = -f * b01, fb02 = -f * b02, fb12 = -f * b12;
    const R fP[3][3] = {{fmac(-f, b00, t), fb01, fb02},
                        {fb01, fmac(-f, b11, t), fb12},
                        {fb02, fb12, fmac(-f, b22, t)}};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        Gb[i][j] = fmac(fP[i][2], G[2][j], fmac(fP[i][1], G[1][j], fmac(fP[i][0], G[0][j], Gb[i][j])));
  }
  // Gh = sum_a u_a c_a^T, S = sum_a u_a, u_g = QB S + (QA - QB) u_g, and the
  // convection's -(rho/120) Gh (S + u_a): gu_a = Gb c_a + Sbar + Hm^T wm_a + (QA-QB) ugb_a
  // with Hm = -(rho/120) Gh and Sbar = Hm^T sum_a wm_a + QB sum_g ugb_g.
  rl.w(w);
  {
    const R m120 = P.rho * (R)(SKEW ? -1.0 / 240.0 : -1.0 / 120.0);
    R Hm[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Hm[i][j] = m120 * G[i][j];
    R Sb[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      R acc = (R)kQB * Usum[j];
      if constexpr (TAUE) acc = acc + Sb_tau[j];
#pragma unroll
      for (int i = 0; i < 3; ++i) acc = fmac(Hm[i][j], (w[0][i] + w[1][i]) + (w[2][i] + w[3][i]), acc);
      Sb[j] = acc;
    }
    // Gb c_a as a chain from Sb; c_0 = -(c_1 + c_2 + c_3)
    R cs[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) cs[j] = (c[0][j] + c[1][j]) + c[2][j];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        R acc = fmac(Gb[i][2], c[k][2], fmac(Gb[i][1], c[k][1], fmac(Gb[i][0], c[k][0], Sb[i])));
        acc = fmac((R)(kQA - kQB), ugb[k + 1][i], acc);
        acc = fmac(Hm[0][i], w[k + 1][0], acc);
        acc = fmac(Hm[1][i], w[k + 1][1], acc);
        gu[k + 1][i] = fmac(Hm[2][i], w[k + 1][2], acc);
      }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      R acc = fmac(-Gb[i][2], cs[2], fmac(-Gb[i][1], cs[1], fmac(-Gb[i][0], cs[0], Sb[i])));
      acc = fmac((R)(kQA - kQB), ugb[0][i], acc);
      acc = fmac(Hm[0][i], w[0][0], acc);
      acc = fmac(Hm[1][i], w[0][1], acc);
      gu[0][i] = fmac(Hm[2][i], w[0][2], acc);
    }
  }
  // gph = sum_a p_a c_a, p_bar = sum_a p_a / 4
  R gsum = (R)0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    R acc = fmac(gpb[0], c[k][0], pq);
    acc = fmac(gpb[1], c[k][1], acc);
    gpo[k + 1] = fmac(gpb[2], c[k][2], acc);
    gsum += gpo[k + 1];
  }
  gpo[0] = fmac((R)4, pq, -gsum);
}

template <class R, int FLAGS, class RL = NoReload>
__device__ __forceinline__ void element_vjp(const R c[3][3], R inv_det, R rh, const R u[4][3],
                                            const R p[4], const R w[4][4], const ElemParams<R>& P,
                                            R gu[4][3], R gpo[4], const RL& rl = RL()) {
  element_vjp_impl<R, FLAGS, false, RL>(c, inv_det, rh, u, p, w, P, gu, gpo, nullptr, rl);
}

// The element RHS F and the vector-Jacobian product (gu, gpo) of w at the
// same state in one pass: the forward intermediates are computed once.
template <class R, int FLAGS, class RL = NoReload>
__device__ __forceinline__ void element_rhs_vjp(const R c[3][3], R inv_det, R rh,
                                                const R u[4][3], const R p[4], const R w[4][4],
                                                const ElemParams<R>& P, R F[4][4], R gu[4][3],
                                                R gpo[4], const RL& rl = RL()) {
  element_vjp_impl<R, FLAGS, true, RL>(c, inv_det, rh, u, p, w, P, gu, gpo, F, rl);
}

}  // namespace nsrhs
