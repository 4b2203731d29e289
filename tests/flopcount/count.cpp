// Flop census of the element kernels: instantiate the device arithmetic with a
// scalar that counts every operation whose operands are not both uniform
// (uniform = derived only from the launch parameters and literals, i.e. work
// the compiler hoists out of the element loop).
// Convention: add/sub/mul = 1, fused multiply-add = 2 (it appears here as a
// mul and an add), reciprocal / sqrt / reciprocal cube root = 1 each.
#include <cstdio>

struct Cnt {
  double v = 0.0;
  bool uni = true;
  bool prod = false;  // a counted product not yet consumed by an addition
  Cnt() = default;
  Cnt(double x) : v(x), uni(true) {}
  Cnt(double x, bool u, bool pr = false) : v(x), uni(u), prod(pr) {}
  explicit operator double() const { return v; }
};
static long g_add = 0, g_mul = 0, g_sfu = 0;
// Instruction estimate (not a flop count): an addition that consumes a fresh
// product is taken as fused with it (one FMA instruction).
static long g_fused = 0;
inline Cnt op(double r, const Cnt& a, const Cnt& b, long& c, bool is_mul) {
  bool u = a.uni && b.uni;
  if (!u) ++c;
  if (!u && !is_mul && (a.prod || b.prod)) ++g_fused;
  return Cnt(r, u, !u && is_mul);
}
inline Cnt operator+(const Cnt& a, const Cnt& b) { return op(a.v + b.v, a, b, g_add, false); }
inline Cnt operator-(const Cnt& a, const Cnt& b) { return op(a.v - b.v, a, b, g_add, false); }
inline Cnt operator*(const Cnt& a, const Cnt& b) { return op(a.v * b.v, a, b, g_mul, true); }
inline Cnt operator-(const Cnt& a) { return Cnt(-a.v, a.uni, a.prod); }  // folds into its consumer
inline Cnt& operator+=(Cnt& a, const Cnt& b) { return a = a + b; }
inline Cnt& operator-=(Cnt& a, const Cnt& b) { return a = a - b; }
inline bool operator>(const Cnt& a, const Cnt& b) { return a.v > b.v; }

#include "../../paper_2403_08777_gb300/csrc/element.cuh"

namespace nsrhs {
template <>
struct MathOps<Cnt> {
  static Cnt sfu(double r, const Cnt& a) {
    if (!a.uni) ++g_sfu;
    return Cnt(r, a.uni);
  }
  static Cnt rcp(const Cnt& x) { return sfu(1.0 / x.v, x); }
  static Cnt sqrt_(const Cnt& x) { return sfu(std::sqrt(x.v), x); }
  static Cnt rcbrt_(const Cnt& x) { return sfu(1.0 / std::cbrt(x.v), x); }
  static Cnt rsqrt_(const Cnt& x) { return sfu(1.0 / std::sqrt(x.v), x); }
};
}  // namespace nsrhs

using namespace nsrhs;

static void reset() { g_add = g_mul = g_sfu = g_fused = 0; }
static long total() { return g_add + g_mul + g_sfu; }

int main() {
  // A generic element; the values only steer the Vreman branch (taken).
  const double Xd[4][3] = {{0.1, 0.0, 0.05}, {1.0, 0.1, 0.0}, {0.0, 1.1, 0.2}, {0.1, 0.2, 0.9}};
  Cnt X[4][3], u[4][3], p[4], w[4][4];
  for (int a = 0; a < 4; ++a) {
    for (int d = 0; d < 3; ++d) X[a][d] = Cnt(Xd[a][d], false);
    for (int i = 0; i < 3; ++i) u[a][i] = Cnt(0.3 * a - 0.2 * i + 0.1 * a * i + 0.05, false);
    p[a] = Cnt(0.7 - 0.3 * a, false);
    for (int k = 0; k < 4; ++k) w[a][k] = Cnt(0.2 * a + 0.1 * k - 0.3, false);
  }
  ElemParams<Cnt> P{Cnt(1.0), Cnt(1e-3), Cnt(0.07), Cnt(4.0), Cnt(2.0)};
  for (int vreman = 0; vreman < 2; ++vreman) {
    Cnt c[3][3], inv_det, rh, F[4][4], gu[4][3], gp[4];
    reset();
    element_geometry<Cnt, Cnt, Cnt>(X, c, inv_det, rh);
    long geo = total(), geo_sfu = g_sfu;
    reset();
    if (vreman) element_rhs<Cnt, kVreman>(c, inv_det, rh, u, p, P, F);
    else element_rhs<Cnt, 0>(c, inv_det, rh, u, p, P, F);
    long fwd = total(), fwd_sfu = g_sfu, fwd_inst = total() - g_fused;
    reset();
    if (vreman) element_vjp<Cnt, kVreman>(c, inv_det, rh, u, p, w, P, gu, gp);
    else element_vjp<Cnt, 0>(c, inv_det, rh, u, p, w, P, gu, gp);
    long vjp = total(), vjp_sfu = g_sfu, vjp_inst = total() - g_fused;
    // per call: the geometry is computed once per mesh and cached
    std::printf("%s fwd %ld sfu %ld vjp %ld sfu %ld geometry %ld sfu %ld\n",
                vreman ? "vreman" : "plain", fwd, fwd_sfu, vjp, vjp_sfu, geo, geo_sfu);
    std::printf("%s instructions (FMA-contracted estimate): fwd %ld vjp %ld\n",
                vreman ? "vreman" : "plain", fwd_inst, vjp_inst);
    {
      Cnt F3[4][4], gu3[4][3], gp3[4];
      reset();
      if (vreman) element_rhs_vjp<Cnt, kVreman>(c, inv_det, rh, u, p, w, P, F3, gu3, gp3);
      else element_rhs_vjp<Cnt, 0>(c, inv_det, rh, u, p, w, P, F3, gu3, gp3);
      std::printf("%s rhs+vjp %ld sfu %ld instructions %ld\n", vreman ? "vreman" : "plain",
                  total(), g_sfu, total() - g_fused);
    }
    {
      Cnt F2[4][4];
      reset();
      if (vreman) element_rhs<Cnt, kVreman>(c, inv_det, rh, u, p, P, F2);
      else element_rhs<Cnt, 0>(c, inv_det, rh, u, p, P, F2);
      std::printf("%s fwd detail: add %ld mul %ld fused %ld sfu %ld -> fma %ld, lone mul %ld, "
                  "lone add %ld\n", vreman ? "vreman" : "plain", g_add, g_mul, g_fused, g_sfu,
                  g_fused, g_mul - g_fused, g_add - g_fused);
    }
  }
  return 0;
}
