// Operation count of the METHOD (the oracle's definition of the element RHS),
// as opposed to count.cpp, which counts the kernels' restructured algebra.
//
// The oracle's element routine is compiled here with a recording scalar: its
// arithmetic is put on a tape as an expression DAG in which constants are
// folded (operations on literals and parameters only cost nothing; x + 0,
// x * 1 and x * 0 are not operations) and a repeated operation on the same
// operands is the same node (common subexpressions count once). Forward
// count = the DAG's arithmetic nodes: add/sub/mul/div/sqrt/cbrt = 1 each (a
// multiply-add written as such is 2). Nodes that depend on the coordinates
// only form the geometry; the rest depend on the nodal (u, p).
//
// Adjoint count = the forward's (u, p)-dependent nodes (recomputed) plus one
// reverse-mode sweep over the DAG for the vector-Jacobian product with
// respect to (u, p): for c = a * b, abar += cbar * b (1 mul); for c = a / b,
// t = cbar / b (1), abar += t, bbar -= t * c (1 mul); for c = sqrt(a),
// abar += (cbar / c) * 0.5 (2); every node's adjoint is the sum of its
// consumers' contributions (contributions - 1 additions; sign changes are
// free). The seed (the cotangent) costs nothing.
//
// The oracle's element code is included from a header the test writes from
// oracle/nsrhs_oracle.cpp (its parameter struct, constants and element
// routine, with its double type replaced by the recording scalar GT).
#include <cmath>
#include <cstdio>
#include <map>
#include <tuple>
#include <vector>

struct Node {
  char op;     // 'x' coordinate leaf, 'u' nodal-field leaf, + - * / n(negate) s(sqrt) c(cbrt)
  int a, b;    // operand node ids (-1: a folded constant)
  double ca, cb;
  bool active;  // depends on the nodal fields
  double val;
};
static std::vector<Node> g_tape;
static std::map<std::tuple<char, int, int, double, double>, int> g_cse;

struct MC {
  double v = 0.0;
  int id = -1;  // -1: folded constant
  MC() = default;
  MC(double x) : v(x), id(-1) {}
  MC(double x, int i) : v(x), id(i) {}
  bool uni() const { return id < 0; }
};

static MC leaf(double v, char kind) {
  g_tape.push_back(Node{kind, -1, -1, 0.0, 0.0, kind == 'u', v});
  return MC(v, (int)g_tape.size() - 1);
}

static MC node(char op, const MC& a, const MC& b, double r) {
  int ia = a.id, ib = b.id;
  double ca = a.uni() ? a.v : 0.0, cb = b.uni() ? b.v : 0.0;
  if ((op == '+' || op == '*') && (ia > ib || (ia == ib && ca > cb))) {
    std::swap(ia, ib);
    std::swap(ca, cb);
  }
  auto key = std::make_tuple(op, ia, ib, ca, cb);
  auto it = g_cse.find(key);
  if (it != g_cse.end()) return MC(g_tape[it->second].val, it->second);
  bool act = (ia >= 0 && g_tape[ia].active) || (ib >= 0 && g_tape[ib].active);
  g_tape.push_back(Node{op, ia, ib, ca, cb, act, r});
  int id = (int)g_tape.size() - 1;
  g_cse[key] = id;
  return MC(r, id);
}

inline MC operator-(const MC& a) { return a.uni() ? MC(-a.v) : node('n', a, MC(0.0), -a.v); }
inline MC operator+(const MC& a, const MC& b) {
  if (a.uni() && b.uni()) return MC(a.v + b.v);
  if (a.uni() && a.v == 0.0) return b;
  if (b.uni() && b.v == 0.0) return a;
  return node('+', a, b, a.v + b.v);
}
inline MC operator-(const MC& a, const MC& b) {
  if (a.uni() && b.uni()) return MC(a.v - b.v);
  if (b.uni() && b.v == 0.0) return a;
  if (a.uni() && a.v == 0.0) return -b;
  return node('-', a, b, a.v - b.v);
}
inline MC operator*(const MC& a, const MC& b) {
  if (a.uni() && b.uni()) return MC(a.v * b.v);
  if ((a.uni() && a.v == 0.0) || (b.uni() && b.v == 0.0)) return MC(0.0);
  if (a.uni() && a.v == 1.0) return b;
  if (b.uni() && b.v == 1.0) return a;
  if (a.uni() && a.v == -1.0) return -b;
  if (b.uni() && b.v == -1.0) return -a;
  return node('*', a, b, a.v * b.v);
}
inline MC operator/(const MC& a, const MC& b) {
  if (a.uni() && b.uni()) return MC(a.v / b.v);
  if (b.uni() && b.v == 1.0) return a;
  if (a.uni() && a.v == 0.0) return MC(0.0);
  return node('/', a, b, a.v / b.v);
}
inline MC& operator+=(MC& a, const MC& b) { return a = a + b; }
inline MC& operator-=(MC& a, const MC& b) { return a = a - b; }
inline bool operator>(const MC& a, const MC& b) { return a.v > b.v; }
inline bool operator!=(const MC& a, const MC& b) { return a.v != b.v; }
inline bool operator==(const MC& a, const MC& b) { return a.v == b.v; }
inline MC re(const MC& x) { return x; }

namespace std {
inline MC sqrt(const MC& a) { return a.uni() ? MC(std::sqrt(a.v)) : node('s', a, MC(0.0), std::sqrt(a.v)); }
inline MC cbrt(const MC& a) { return a.uni() ? MC(std::cbrt(a.v)) : node('c', a, MC(0.0), std::cbrt(a.v)); }
}  // namespace std

typedef MC GT;
#include "oracle_element.inc"

static bool counted(char op) {
  return op == '+' || op == '-' || op == '*' || op == '/' || op == 's' || op == 'c';
}

struct Counts {
  long fwd_total = 0, fwd_geometry = 0, reverse = 0;
};

static Counts count_element(double c_vreman, double tau_elem, double skew) {
  g_tape.clear();
  g_cse.clear();
  const double Xd[4][3] = {{0.1, 0.0, 0.05}, {1.0, 0.1, 0.0}, {0.0, 1.1, 0.2}, {0.1, 0.2, 0.9}};
  GT X[4][3];
  MC U[4][4], F[4][4];
  for (int a = 0; a < 4; ++a) {
    for (int d = 0; d < 3; ++d) X[a][d] = leaf(Xd[a][d], 'x');
    for (int k = 0; k < 3; ++k) U[a][k] = leaf(0.3 * a - 0.2 * k + 0.1 * a * k + 0.05, 'u');
    U[a][3] = leaf(0.7 - 0.3 * a, 'u');
  }
  Params P{MC(1.0), MC(1e-3), MC(c_vreman), MC(4.0), MC(2.0), MC(skew), MC(tau_elem)};
  element_rhs<MC>(X, U, P, T_ALL, F);
  Counts c;
  for (const Node& n : g_tape)
    if (counted(n.op)) {
      ++c.fwd_total;
      if (!n.active) ++c.fwd_geometry;
    }
  // reverse sweep from the 16 outputs
  std::vector<int> contrib(g_tape.size(), 0);
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 4; ++k)
      if (F[a][k].id >= 0) contrib[F[a][k].id] += 1;  // the seed
  auto give = [&](int id) {
    if (id >= 0 && g_tape[id].active) contrib[id] += 1;
  };
  for (int i = (int)g_tape.size() - 1; i >= 0; --i) {
    const Node& n = g_tape[i];
    if (!n.active || contrib[i] == 0) continue;
    c.reverse += contrib[i] - 1;  // summing the contributions
    const bool aa = n.a >= 0 && g_tape[n.a].active, ba = n.b >= 0 && g_tape[n.b].active;
    switch (n.op) {
      case '+': case '-': give(n.a); give(n.b); break;
      case 'n': give(n.a); break;
      case '*':
        if (aa) { ++c.reverse; give(n.a); }
        if (ba) { ++c.reverse; give(n.b); }
        break;
      case '/':
        ++c.reverse;  // t = cbar / b
        if (aa) give(n.a);
        if (ba) { ++c.reverse; give(n.b); }
        break;
      case 's': c.reverse += 2; give(n.a); break;
      case 'c': c.reverse += 3; give(n.a); break;
      default: break;
    }
  }
  // the gradient entries (leaves) sum their contributions too
  for (size_t i = 0; i < g_tape.size(); ++i)
    if (g_tape[i].op == 'u' && contrib[i] > 1) c.reverse += contrib[i] - 1;
  return c;
}

int main() {
  for (int vreman = 0; vreman < 2; ++vreman) {
    Counts c = count_element(vreman ? 0.07 : 0.0, 0.0, 0.0);
    const long per_call = c.fwd_total - c.fwd_geometry;
    std::printf("%s method fwd_total %ld geometry %ld per_call %ld vjp_per_call %ld\n",
                vreman ? "vreman" : "plain", c.fwd_total, c.fwd_geometry, per_call,
                per_call + c.reverse);
  }
  return 0;
}
