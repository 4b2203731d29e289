// Seeded synthetic inputs for the tetrahedral Navier-Stokes RHS assembly.
//
// This file generates INPUTS only: a jittered Kuhn (Freudenthal) tetrahedral
// mesh of the unit cube, nodal velocity/pressure fields, random vectors and node
// renumberings (random, reverse Cuthill-McKee). It contains none of the
// assembly arithmetic. Both the CPU oracle and the CUDA path consume what it
// produces; neither is linked into it.
//
// The paper's workload is a 32M-tet LES mesh of the Bolund cliff (Sec. III-A);
// that mesh is not available, so these structured-but-jittered meshes of
// linear tetrahedra (Sec. II restricts the study to tets) stand in for it.
//
// Random numbers: counter-based SplitMix64 keyed by (seed, stream, index), so
// every value is a pure function of its key and the output does not depend on
// thread count or visiting order.
//
// Host code only; portable C++17 (builds on x86-64 and aarch64).

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>
#include <memory>
#include <thread>
#include <vector>

namespace {

inline uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Counter-based draw: a pure function of (seed, stream, index).
inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t index) {
  return splitmix64(splitmix64(splitmix64(seed) ^ (stream * 0xD1B54A32D192ED03ull)) + index);
}

// Uniform in [0, 1) with 53 random bits.
inline double unif(uint64_t seed, uint64_t stream, uint64_t index) {
  return (double)(draw(seed, stream, index) >> 11) * 0x1.0p-53;
}

// Standard normal by Box-Muller from two counter draws.
inline double normal(uint64_t seed, uint64_t stream, uint64_t index) {
  double u1 = unif(seed, stream, 2 * index);
  double u2 = unif(seed, stream, 2 * index + 1);
  u1 = 1.0 - u1;  // (0, 1]
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
}

int n_threads() {
  unsigned t = std::thread::hardware_concurrency();
  if (t == 0) t = 1;
  if (t > 64) t = 64;
  return (int)t;
}

// Static block partition of [0, n) over threads.
void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& body) {
  int nt = n_threads();
  if (n < 65536 || nt == 1) {
    body(0, n);
    return;
  }
  std::vector<std::thread> th;
  int64_t chunk = (n + nt - 1) / nt;
  for (int t = 0; t < nt; ++t) {
    int64_t b = t * chunk, e = std::min(n, b + chunk);
    if (b >= e) break;
    th.emplace_back(body, b, e);
  }
  for (auto& x : th) x.join();
}

// Signed 6*volume of the tet (a, b, c, d): det[b-a, c-a, d-a].
inline double det6(const double* X, const double* Y, const double* Z, int64_t a, int64_t b,
                   int64_t c, int64_t d) {
  double e1x = X[b] - X[a], e1y = Y[b] - Y[a], e1z = Z[b] - Z[a];
  double e2x = X[c] - X[a], e2y = Y[c] - Y[a], e2z = Z[c] - Z[a];
  double e3x = X[d] - X[a], e3y = Y[d] - Y[a], e3z = Z[d] - Z[a];
  return e1x * (e2y * e3z - e2z * e3y) - e1y * (e2x * e3z - e2z * e3x) +
         e1z * (e2x * e3y - e2y * e3x);
}

}  // namespace

extern "C" {

// Kuhn mesh of the unit cube with n^3 hexes, 6 tets per hex.
//   node (i,j,k), 0<=i,j,k<=n, has id i + (n+1)*(j + (n+1)*k)  (lexicographic)
//   hex (i,j,k) has id i + n*(j + n*k); its tets are elements 6*hex .. 6*hex+5
//   tet for the axis order (a,b,c): (v0, v0+e_a, v0+e_a+e_b, v0+e_a+e_b+e_c=v7);
//   for odd permutations local nodes 1 and 2 are swapped so that detJ > 0.
// Interior nodes move by independent U(-jitter*h, jitter*h) per component
// (seed, stream 0); boundary nodes stay on the cube. Tets whose detJ falls below
// min_det_frac * h^3 have the jitter of their interior nodes halved, pass after
// pass, until none remain.
// coords: [3][N] f64, conn: [4][E] int32, hex_colour: [n^3] int8 (parity
// colour (i&1) + 2(j&1) + 4(k&1)) or NULL.
// Returns the number of nodes whose jitter was reduced (0 if none), -1 on error.
int64_t mg_box_mesh(int32_t n, double jitter, uint64_t seed, double min_det_frac, double* coords,
                    int32_t* conn, int8_t* hex_colour) {
  if (n < 1 || n > 1024 || !coords || !conn) return -1;
  const int64_t n1 = (int64_t)n + 1;
  const int64_t N = n1 * n1 * n1;
  const int64_t H = (int64_t)n * n * n;
  const int64_t E = 6 * H;
  const double h = 1.0 / n;
  double* X = coords;
  double* Y = coords + N;
  double* Z = coords + 2 * N;
  std::vector<double> off(3 * (size_t)N, 0.0);
  parallel_for(N, [&](int64_t b, int64_t e) {
    for (int64_t v = b; v < e; ++v) {
      int64_t i = v % n1, j = (v / n1) % n1, k = v / (n1 * n1);
      bool interior = i > 0 && i < n && j > 0 && j < n && k > 0 && k < n;
      for (int c = 0; c < 3; ++c)
        off[3 * v + c] =
            interior ? (2.0 * unif(seed, 0, 3 * (uint64_t)v + c) - 1.0) * jitter * h : 0.0;
    }
  });
  // Local corner index b = bx + 2 by + 4 bz.
  static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  static const int parity[6] = {0, 1, 1, 0, 0, 1};
  parallel_for(H, [&](int64_t b0, int64_t e0) {
    for (int64_t hx = b0; hx < e0; ++hx) {
      int64_t i = hx % n, j = (hx / n) % n, k = hx / ((int64_t)n * n);
      int64_t base = i + n1 * (j + n1 * k);
      auto corner = [&](int c) -> int64_t {
        return base + (c & 1) + n1 * ((c >> 1) & 1) + n1 * n1 * ((c >> 2) & 1);
      };
      if (hex_colour) hex_colour[hx] = (int8_t)((i & 1) + 2 * (j & 1) + 4 * (k & 1));
      for (int t = 0; t < 6; ++t) {
        int c1 = 1 << perms[t][0];
        int c2 = c1 | (1 << perms[t][1]);
        int64_t v[4] = {corner(0), corner(c1), corner(c2), corner(7)};
        if (parity[t]) std::swap(v[1], v[2]);
        int64_t el = 6 * hx + t;
        for (int a = 0; a < 4; ++a) conn[a * E + el] = (int32_t)v[a];
      }
    }
  });
  // Jitter + repair of inverted / nearly flat tets.
  std::unique_ptr<std::atomic<uint8_t>[]> bad(new std::atomic<uint8_t>[N]);
  int64_t n_reduced = 0;
  const double min_det = min_det_frac * h * h * h;
  for (int pass = 0; pass < 64; ++pass) {
    parallel_for(N, [&](int64_t b, int64_t e) {
      for (int64_t v = b; v < e; ++v) {
        int64_t i = v % n1, j = (v / n1) % n1, k = v / (n1 * n1);
        X[v] = (double)i * h + off[3 * v + 0];
        Y[v] = (double)j * h + off[3 * v + 1];
        Z[v] = (double)k * h + off[3 * v + 2];
      }
    });
    for (int64_t v = 0; v < N; ++v) bad[v].store(0, std::memory_order_relaxed);
    std::atomic<int64_t> nbad{0};
    parallel_for(E, [&](int64_t b, int64_t e) {
      int64_t local = 0;
      for (int64_t el = b; el < e; ++el) {
        int64_t v0 = conn[el], v1 = conn[E + el], v2 = conn[2 * E + el], v3 = conn[3 * E + el];
        if (det6(X, Y, Z, v0, v1, v2, v3) < min_det) {
          bad[v0].store(1, std::memory_order_relaxed);
          bad[v1].store(1, std::memory_order_relaxed);
          bad[v2].store(1, std::memory_order_relaxed);
          bad[v3].store(1, std::memory_order_relaxed);
          ++local;
        }
      }
      nbad += local;
    });
    if (nbad.load() == 0) break;
    if (pass == 63) return -2;
    for (int64_t v = 0; v < N; ++v) {
      if (bad[v].load(std::memory_order_relaxed) && (off[3 * v] != 0.0 || off[3 * v + 1] != 0.0 || off[3 * v + 2] != 0.0)) {
        off[3 * v] *= 0.5;
        off[3 * v + 1] *= 0.5;
        off[3 * v + 2] *= 0.5;
        ++n_reduced;
      }
    }
  }
  return n_reduced;
}

// Nodal (u, v, w, p) as [4][N] f64.
//   u = (sin X cos Y cos Z, -cos X sin Y cos Z, 0), X = 2 pi x (Taylor-Green),
//   + N(0, noise_sigma^2) per component (stream 1),
//   + m * d with m ~ U(0, mag_max) and d uniform on the sphere (streams 2, 3)
//     when mag_max > 0,
//   p ~ U(-1, 1) (stream 4).
void mg_fields(int64_t N, const double* coords, uint64_t seed, double noise_sigma, double mag_max,
               double* up) {
  const double* X = coords;
  const double* Y = coords + N;
  const double* Z = coords + 2 * N;
  parallel_for(N, [&](int64_t b, int64_t e) {
    for (int64_t v = b; v < e; ++v) {
      double x = 2.0 * M_PI * X[v], y = 2.0 * M_PI * Y[v], z = 2.0 * M_PI * Z[v];
      double u[3] = {std::sin(x) * std::cos(y) * std::cos(z), -std::cos(x) * std::sin(y) * std::cos(z),
                     0.0};
      for (int c = 0; c < 3; ++c) u[c] += noise_sigma * normal(seed, 1, 3 * (uint64_t)v + c);
      if (mag_max > 0.0) {
        double m = mag_max * unif(seed, 2, (uint64_t)v);
        double d[3], nn = 0.0;
        for (int c = 0; c < 3; ++c) {
          d[c] = normal(seed, 3, 3 * (uint64_t)v + c);
          nn += d[c] * d[c];
        }
        nn = std::sqrt(nn);
        if (nn > 0.0)
          for (int c = 0; c < 3; ++c) u[c] += m * d[c] / nn;
      }
      for (int c = 0; c < 3; ++c) up[c * N + v] = u[c];
      up[3 * N + v] = 2.0 * unif(seed, 4, (uint64_t)v) - 1.0;
    }
  });
}

// out[i] ~ N(0, 1), i < n (seed, stream 5).
void mg_normal(int64_t n, uint64_t seed, double* out) {
  parallel_for(n, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) out[i] = normal(seed, 5, (uint64_t)i);
  });
}

// Random node order: order[new] = old, sorted by a counter-based 64-bit key
// (seed, stream 6); ties (probability ~0) broken by the old id.
void mg_random_order(int64_t N, uint64_t seed, int64_t* order) {
  std::vector<std::pair<uint64_t, int64_t>> key(N);
  parallel_for(N, [&](int64_t b, int64_t e) {
    for (int64_t v = b; v < e; ++v) key[v] = {draw(seed, 6, (uint64_t)v), v};
  });
  std::sort(key.begin(), key.end());
  for (int64_t v = 0; v < N; ++v) order[v] = key[v].second;
}

// Reverse Cuthill-McKee order of the node graph of a tet mesh
// (nodes adjacent when they share an element): order[new] = old.
// Start node: pseudo-peripheral node found by repeated BFS (George-Liu),
// starting from the lowest-degree node. Neighbours are visited by increasing
// (degree, id). Disconnected pieces are appended one after another.
// Returns 0, or -1 on bad input.
int mg_rcm_order(int64_t N, int64_t E, const int32_t* conn, int64_t* order) {
  if (N <= 0 || N > INT32_MAX || E < 0 || !conn || !order) return -1;
  for (int64_t i = 0; i < 4 * E; ++i)
    if (conn[i] < 0 || conn[i] >= N) return -1;
  // node -> element incidence (CSR)
  std::vector<int64_t> start(N + 1, 0);
  for (int64_t i = 0; i < 4 * E; ++i) start[conn[i] + 1]++;
  for (int64_t v = 0; v < N; ++v) start[v + 1] += start[v];
  std::vector<int32_t> inc(start[N]);
  {
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (int64_t a = 0; a < 4; ++a)
      for (int64_t el = 0; el < E; ++el) inc[fill[conn[a * E + el]]++] = (int32_t)el;
  }
  auto neighbours = [&](int64_t v, std::vector<int32_t>& out) {
    out.clear();
    for (int64_t q = start[v]; q < start[v + 1]; ++q) {
      int64_t el = inc[q];
      for (int a = 0; a < 4; ++a) {
        int32_t w = conn[a * E + el];
        if (w != v) out.push_back(w);
      }
    }
    std::sort(out.begin(), out.end());
    out.erase(std::unique(out.begin(), out.end()), out.end());
  };
  // Deduplicated adjacency (CSR), built in two parallel passes.
  std::vector<int64_t> astart(N + 1, 0);
  parallel_for(N, [&](int64_t b, int64_t e) {
    std::vector<int32_t> nb;
    for (int64_t v = b; v < e; ++v) {
      neighbours(v, nb);
      astart[v + 1] = (int64_t)nb.size();
    }
  });
  for (int64_t v = 0; v < N; ++v) astart[v + 1] += astart[v];
  std::vector<int32_t> adj(astart[N]);
  parallel_for(N, [&](int64_t b, int64_t e) {
    std::vector<int32_t> nb;
    for (int64_t v = b; v < e; ++v) {
      neighbours(v, nb);
      std::copy(nb.begin(), nb.end(), adj.begin() + astart[v]);
    }
  });
  std::vector<int32_t>().swap(inc);
  auto deg = [&](int64_t v) -> int64_t { return astart[v + 1] - astart[v]; };

  std::vector<uint8_t> visited(N, 0);
  std::vector<int32_t> level(N, -1);
  std::vector<int32_t> queue;
  queue.reserve(N);
  // BFS from s over the piece of s (nodes not yet placed); returns the
  // eccentricity of s and the lowest (degree, id) node of the last level.
  auto bfs = [&](int64_t s, int64_t& far) -> int32_t {
    std::vector<int32_t> q;
    q.push_back((int32_t)s);
    level[s] = 0;
    size_t head = 0;
    int32_t ecc = 0;
    while (head < q.size()) {
      int32_t v = q[head++];
      for (int64_t t = astart[v]; t < astart[v + 1]; ++t) {
        int32_t w = adj[t];
        if (level[w] < 0 && !visited[w]) {
          level[w] = level[v] + 1;
          ecc = std::max(ecc, level[w]);
          q.push_back(w);
        }
      }
    }
    far = -1;
    for (int32_t v : q)
      if (level[v] == ecc && (far < 0 || deg(v) < deg(far) || (deg(v) == deg(far) && v < far)))
        far = v;
    for (int32_t v : q) level[v] = -1;
    return ecc;
  };
  int64_t scan = 0;
  while ((int64_t)queue.size() < N) {
    while (visited[scan]) ++scan;
    // lowest-degree node of the piece containing `scan` as the initial guess
    int64_t s = scan;
    {
      std::vector<int32_t> q{(int32_t)scan};
      level[scan] = 0;
      for (size_t head = 0; head < q.size(); ++head) {
        int32_t v = q[head];
        if (deg(v) < deg(s) || (deg(v) == deg(s) && v < s)) s = v;
        for (int64_t t = astart[v]; t < astart[v + 1]; ++t)
          if (level[adj[t]] < 0 && !visited[adj[t]]) {
            level[adj[t]] = 0;
            q.push_back(adj[t]);
          }
      }
      for (int32_t v : q) level[v] = -1;
    }
    int64_t far;
    int32_t ecc = bfs(s, far);
    for (int it = 0; it < 8; ++it) {
      int64_t far2;
      int32_t ecc2 = bfs(far, far2);
      if (ecc2 <= ecc) break;
      s = far;
      ecc = ecc2;
      far = far2;
    }
    // Cuthill-McKee
    size_t head = queue.size();
    queue.push_back((int32_t)s);
    visited[s] = 1;
    while (head < queue.size()) {
      int32_t v = queue[head++];
      size_t first = queue.size();
      for (int64_t t = astart[v]; t < astart[v + 1]; ++t) {
        int32_t w = adj[t];
        if (!visited[w]) {
          visited[w] = 1;
          queue.push_back(w);
        }
      }
      std::sort(queue.begin() + first, queue.end(), [&](int32_t a, int32_t b) {
        return deg(a) != deg(b) ? deg(a) < deg(b) : a < b;
      });
    }
  }
  for (int64_t i = 0; i < N; ++i) order[i] = queue[N - 1 - i];
  return 0;
}

// Semi-bandwidth of the nodal graph: max over elements of (max id - min id).
int64_t mg_bandwidth(int64_t E, const int32_t* conn) {
  int64_t bw = 0;
  for (int64_t el = 0; el < E; ++el) {
    int32_t lo = conn[el], hi = conn[el];
    for (int a = 1; a < 4; ++a) {
      lo = std::min(lo, conn[a * E + el]);
      hi = std::max(hi, conn[a * E + el]);
    }
    bw = std::max<int64_t>(bw, hi - lo);
  }
  return bw;
}

}  // extern "C"
