// nsrhs: C-ABI library for the element-by-element Navier-Stokes RHS assembly
// on linear tetrahedra (arXiv 2403.08777, Sec. II and V), GB300 / sm_103a.
//
// Host side: mesh objects (device copies of coordinates and connectivity,
// validation, aspect-ratio classification, Morton element order, cached
// geometry, element blocks, optional colourings), argument checking and
// kernel launches. Device side: the element kernels (element.cuh holds the
// per-element arithmetic, blocks.cuh the block-staged kernels, colour.cuh
// the colourings). One thread assembles one element, with every
// intermediate in registers (the paper's specialisation + privatisation,
// Sec. V-B/V-C), and scatters its 16 entries as soon as they are computed
// (immediate scatter, Sec. V-D): by double-precision atomic adds (the FP64
// default), by per-block sums staged in shared memory (the mixed default),
// or in coloured launches, whose atomics never meet at one address, so that
// their order (colour after colour) is fixed. Atomics resolve the write
// conflicts that the paper's CPU path avoids with a separate serial scatter
// loop (Sec. V-C); colouring also fixes the order of the sums.
//
// Aspect ratio: mesh creation classifies elements by aspect ratio against
// opts.ar_threshold, but only to report the count (n_high_ar). The threshold
// changes no arithmetic: every element's determinant and inverse are computed
// in double once per mesh, and the mixed form reads their float rounding.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <new>
#include <unordered_set>
#include <vector>

#include <cub/cub.cuh>

#include "../../include/nsrhs.h"
#include "blocks.cuh"
#include "colour.cuh"
#include "element.cuh"
#include "elmat.cuh"

struct nsrhs_mesh {
  int64_t n_nodes = 0, n_elems = 0;
  int device = 0;
  double* coords = nullptr;   // [3][N]
  int32_t* conn = nullptr;    // [4][E], caller's element order
  // Element geometry computed once in double precision (cofactor vectors
  // c[k][d] at rows 3k+d, then 1/detJ, then detJ^(-1/3)), [kGeomRows][E]:
  // it depends on the mesh only, and one streamed 88-byte record costs far
  // less on GB300 than the ~40 FP64 instructions that recompute it.
  double* geom = nullptr;
  // Per-element records (blocks.cuh; chunk-major per block of elements): the
  // same geometry rounded to float (the mixed form) and the block map of the
  // block kernels.
  nsrhs::RecChunk* rec = nullptr;
  // Element blocks (blocks.cuh): elements are stored in Morton order of
  // their centroids; per block of kBlockElems elements its distinct nodes,
  // their contribution runs and the local connectivity.
  int64_t n_blocks = 0;
  int64_t* blk_node_off = nullptr;  // [n_blocks + 1]
  int32_t* blk_nodes = nullptr;     // [blk_node_off[n_blocks]]
  uint32_t* blk_runs = nullptr;     // [blk_node_off[n_blocks]] (first position << 16) | length
  int blk_cap = 0;                  // staging capacity: the largest block's distinct nodes, rounded up
  double* inv_mass = nullptr;       // [N] 1 / lumped mass
  double* mass = nullptr;           // [N] lumped mass sum_e V_e / 4
  // Colour-major copy for the COLOUR scatter (colour.cuh), built when the
  // mesh options ask for it: the elements stably sorted by colour, colour k
  // at [col_off[k], col_off[k + 1]).
  std::vector<int64_t> col_off;
  int32_t* col_conn = nullptr;      // [4][E]
  double* col_geom = nullptr;       // [kGeomRows][E]
  nsrhs::RecChunk* col_rec = nullptr;  // the records of the colour-major order
  uint8_t* colour = nullptr;        // [E] colour of each element (Morton order)
  int32_t* elem_order = nullptr;    // [E] caller's index of each element (Morton order)
  // Block colouring for the BLOCK_COLOUR scatter: block colour k is the
  // blocks bcol_order[bcol_off[k] .. bcol_off[k + 1]).
  std::vector<int64_t> bcol_off;
  int32_t* bcol_order = nullptr;    // [n_blocks]
  uint8_t* bcolour = nullptr;       // [n_blocks] colour of each block
  nsrhs_mesh_info info{};
  std::vector<void*> allocations;
};

namespace {

using nsrhs::ElemParams;

std::mutex g_registry_mutex;
std::unordered_set<const nsrhs_mesh*> g_registry;

bool is_live(const nsrhs_mesh* m) {
  std::lock_guard<std::mutex> lock(g_registry_mutex);
  return m != nullptr && g_registry.count(m) != 0;
}

constexpr int kThreads = 128;
constexpr int kGeomRows = 11;
// Block-kernel grids: at most a full SM's worth of threads (2048) per SM.
constexpr int kBlockCtasPerSm = 2048 / nsrhs::kBlockElems > 0 ? 2048 / nsrhs::kBlockElems : 1;

// Minimum resident CTAs per SM requested from the compiler (register cap) for
// the FP64 element kernels; measured choices, overridable at build time.
#ifndef NSRHS_FWD_MIN_CTAS
#define NSRHS_FWD_MIN_CTAS 1
#endif
#ifndef NSRHS_VJP_MIN_CTAS
#define NSRHS_VJP_MIN_CTAS 1
#endif
// The coloured FP64 kernels: capped so that as many CTAs fit per SM as for
// the atomic kernels.
#ifndef NSRHS_FWD_COLOUR_MIN_CTAS
#define NSRHS_FWD_COLOUR_MIN_CTAS 3
#endif
#ifndef NSRHS_VJP_COLOUR_MIN_CTAS
#define NSRHS_VJP_COLOUR_MIN_CTAS 2
#endif

int sm_count(int device) {
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n <= 0)
    n = 152;
  return n;
}

// The largest dynamic shared memory one CTA may use on `device`.
size_t smem_limit(int device) {
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
      v <= 0)
    v = 48 * 1024;
  return (size_t)v;
}

// Grid for a grid-stride loop over n items: a whole number of waves of
// `per_sm` blocks on every SM, no more blocks than items need.
unsigned grid_for(int64_t n, int device, int per_sm) {
  int64_t need = (n + kThreads - 1) / kThreads;
  int64_t cap = (int64_t)sm_count(device) * per_sm;
  return (unsigned)std::max<int64_t>(1, std::min(need, cap));
}

// ---------------------------------------------------------------------------
// Mesh validation and classification (setup).

struct ValidateOut {
  unsigned long long bad_index;
  unsigned long long bad_det;
  unsigned long long n_high_ar;
  unsigned long long min_det_bits;  // positive doubles order like their bit patterns
  unsigned long long max_ar_bits;
};

__global__ void validate_kernel(int64_t N, int64_t E, const double* __restrict__ coords,
                                const int32_t* __restrict__ conn, double ar_threshold,
                                uint8_t* __restrict__ high_ar, ValidateOut* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t v[4];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      v[a] = conn[a * E + e];
      ok = ok && v[a] >= 0 && (int64_t)v[a] < N;
    }
    high_ar[e] = 0;
    if (!ok) {
      atomicAdd(&out->bad_index, 1ull);
      continue;
    }
    double X[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int d = 0; d < 3; ++d) X[a][d] = coords[d * N + v[a]];
    double ed[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int d = 0; d < 3; ++d) ed[k][d] = X[k + 1][d] - X[0][d];
    double det = ed[0][0] * (ed[1][1] * ed[2][2] - ed[1][2] * ed[2][1]) -
                 ed[0][1] * (ed[1][0] * ed[2][2] - ed[1][2] * ed[2][0]) +
                 ed[0][2] * (ed[1][0] * ed[2][1] - ed[1][1] * ed[2][0]);
    if (!(det > 0.0)) {
      atomicAdd(&out->bad_det, 1ull);
      continue;
    }
    // aspect ratio l_max * S / (6 sqrt(6) V), V = det / 6
    double lmax2 = 0.0;
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b) {
        double dx = X[b][0] - X[a][0], dy = X[b][1] - X[a][1], dz = X[b][2] - X[a][2];
        lmax2 = fmax(lmax2, dx * dx + dy * dy + dz * dz);
      }
    double S = 0.0;
    const int fc[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
    for (int f = 0; f < 4; ++f) {
      const double* A = X[fc[f][0]];
      const double* B = X[fc[f][1]];
      const double* C = X[fc[f][2]];
      double ab[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
      double ac[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
      double cx = ab[1] * ac[2] - ab[2] * ac[1];
      double cy = ab[2] * ac[0] - ab[0] * ac[2];
      double cz = ab[0] * ac[1] - ab[1] * ac[0];
      S += 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
    }
    double ar = sqrt(lmax2) * S / (sqrt(6.0) * det);
    if (ar > ar_threshold) {
      high_ar[e] = 1;
      atomicAdd(&out->n_high_ar, 1ull);
    }
    atomicMin(&out->min_det_bits, (unsigned long long)__double_as_longlong(det));
    atomicMax(&out->max_ar_bits, (unsigned long long)__double_as_longlong(ar));
  }
}

// ---------------------------------------------------------------------------
// Mesh check without allocation (nsrhs_mesh_check_noalloc). The same
// per-element checks as validate_kernel; partial results per block go to a
// static device array instead of cudaMalloc'd memory, and a one-block kernel
// reduces them into the caller's result.

struct CheckPartial {
  unsigned long long bad_index, bad_det, n_high_ar;
  double min_det, max_ar;
  double pad[3];  // 64 bytes
};
static_assert(sizeof(CheckPartial) == 64, "CheckPartial layout");

// One slot per block of check_partials_kernel (64 KiB). Host code must not
// pass this symbol to a kernel: it uses the address from cudaGetSymbolAddress.
static __device__ __align__(256) CheckPartial g_check_scratch[NSRHS_CHECK_SCRATCH_BLOCKS];

constexpr int kCheckThreads = 256;

__global__ void __launch_bounds__(kCheckThreads)
    check_partials_kernel(int64_t N, int64_t E, const double* __restrict__ coords,
                          const int32_t* __restrict__ conn, double ar_threshold,
                          CheckPartial* __restrict__ partials) {
  unsigned long long bad_index = 0, bad_det = 0, n_high = 0;
  double min_det = __longlong_as_double(0x7FF0000000000000ll), max_ar = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t v[4];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      v[a] = conn[a * E + e];
      ok = ok && v[a] >= 0 && (int64_t)v[a] < N;
    }
    if (!ok) {
      ++bad_index;
      continue;
    }
    double X[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int d = 0; d < 3; ++d) X[a][d] = coords[d * N + v[a]];
    double ed[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int d = 0; d < 3; ++d) ed[k][d] = X[k + 1][d] - X[0][d];
    double det = ed[0][0] * (ed[1][1] * ed[2][2] - ed[1][2] * ed[2][1]) -
                 ed[0][1] * (ed[1][0] * ed[2][2] - ed[1][2] * ed[2][0]) +
                 ed[0][2] * (ed[1][0] * ed[2][1] - ed[1][1] * ed[2][0]);
    if (!(det > 0.0)) {
      ++bad_det;
      continue;
    }
    double lmax2 = 0.0;
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b) {
        double dx = X[b][0] - X[a][0], dy = X[b][1] - X[a][1], dz = X[b][2] - X[a][2];
        lmax2 = fmax(lmax2, dx * dx + dy * dy + dz * dz);
      }
    double S = 0.0;
    const int fc[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
    for (int f = 0; f < 4; ++f) {
      const double* A = X[fc[f][0]];
      const double* B = X[fc[f][1]];
      const double* C = X[fc[f][2]];
      double ab[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
      double ac[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
      double cx = ab[1] * ac[2] - ab[2] * ac[1];
      double cy = ab[2] * ac[0] - ab[0] * ac[2];
      double cz = ab[0] * ac[1] - ab[1] * ac[0];
      S += 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
    }
    double ar = sqrt(lmax2) * S / (sqrt(6.0) * det);
    if (ar > ar_threshold) ++n_high;
    min_det = fmin(min_det, det);
    max_ar = fmax(max_ar, ar);
  }
  __shared__ CheckPartial red[kCheckThreads];
  red[threadIdx.x] = CheckPartial{bad_index, bad_det, n_high, min_det, max_ar, {0.0, 0.0, 0.0}};
  __syncthreads();
  for (int stride = kCheckThreads / 2; stride > 0; stride >>= 1) {
    if ((int)threadIdx.x < stride) {
      CheckPartial& a = red[threadIdx.x];
      const CheckPartial& b = red[threadIdx.x + stride];
      a.bad_index += b.bad_index;
      a.bad_det += b.bad_det;
      a.n_high_ar += b.n_high_ar;
      a.min_det = fmin(a.min_det, b.min_det);
      a.max_ar = fmax(a.max_ar, b.max_ar);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kCheckThreads)
    check_reduce_kernel(int n_partials, const CheckPartial* __restrict__ partials,
                        nsrhs_mesh_check_result* __restrict__ result) {
  CheckPartial acc{0ull, 0ull, 0ull, __longlong_as_double(0x7FF0000000000000ll), 0.0,
                   {0.0, 0.0, 0.0}};
  for (int i = threadIdx.x; i < n_partials; i += blockDim.x) {
    const CheckPartial& b = partials[i];
    acc.bad_index += b.bad_index;
    acc.bad_det += b.bad_det;
    acc.n_high_ar += b.n_high_ar;
    acc.min_det = fmin(acc.min_det, b.min_det);
    acc.max_ar = fmax(acc.max_ar, b.max_ar);
  }
  __shared__ CheckPartial red[kCheckThreads];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int stride = kCheckThreads / 2; stride > 0; stride >>= 1) {
    if ((int)threadIdx.x < stride) {
      CheckPartial& a = red[threadIdx.x];
      const CheckPartial& b = red[threadIdx.x + stride];
      a.bad_index += b.bad_index;
      a.bad_det += b.bad_det;
      a.n_high_ar += b.n_high_ar;
      a.min_det = fmin(a.min_det, b.min_det);
      a.max_ar = fmax(a.max_ar, b.max_ar);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    result->bad_index = (int64_t)red[0].bad_index;
    result->bad_det = (int64_t)red[0].bad_det;
    result->n_high_ar = (int64_t)red[0].n_high_ar;
    result->min_detj = red[0].min_det;
    result->max_ar = red[0].max_ar;
  }
}

constexpr int kMaxDevices = 64;
std::mutex g_check_mutex;
CheckPartial* g_check_addr[kMaxDevices] = {};

// Device address of g_check_scratch on the current device (looked up once per
// device with that device current).
nsrhs_status check_scratch_address(CheckPartial** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NSRHS_ECUDA;
  std::lock_guard<std::mutex> lock(g_check_mutex);
  if (g_check_addr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_check_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return NSRHS_ECUDA;
    }
    g_check_addr[dev] = (CheckPartial*)p;
  }
  *out = g_check_addr[dev];
  return NSRHS_OK;
}

// Cached element geometry (setup): double cofactors, 1/detJ and detJ^(-1/3)
// of every element, and their float roundings in the element records (whose
// block map the block planning fills in afterwards).
__global__ void geometry_kernel(int64_t N, int64_t E, const double* __restrict__ coords,
                                const int32_t* __restrict__ conn, double* __restrict__ geom,
                                nsrhs::RecChunk* __restrict__ rec) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    double X[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int64_t v = conn[a * E + e];
#pragma unroll
      for (int d = 0; d < 3; ++d) X[a][d] = coords[d * N + v];
    }
    double c[3][3], inv_det, rh;
    nsrhs::element_geometry<double, double>(X, c, inv_det, rh);
    double g[kGeomRows];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int d = 0; d < 3; ++d) g[3 * k + d] = c[k][d];
    g[9] = inv_det;
    g[10] = rh;
    float gf[12];
#pragma unroll
    for (int q = 0; q < kGeomRows; ++q) {
      geom[q * E + e] = g[q];
      gf[q] = __double2float_rn(g[q]);
    }
    gf[11] = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k)
      *reinterpret_cast<float4*>(rec + nsrhs::rec_index(e, k)) =
          make_float4(gf[4 * k], gf[4 * k + 1], gf[4 * k + 2], gf[4 * k + 3]);
    *reinterpret_cast<uint4*>(rec + nsrhs::rec_index(e, 3)) = make_uint4(0u, 0u, 0u, 0u);
  }
}

// Lumped mass: every element adds V/4 = 1 / (24 inv_det) to its 4 nodes.
__global__ void lumped_mass_kernel(int64_t E, const int32_t* __restrict__ conn,
                                   const double* __restrict__ geom, double* __restrict__ mass) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double v4 = 1.0 / (24.0 * geom[9 * E + e]);
#pragma unroll
    for (int a = 0; a < 4; ++a) atomicAdd(mass + conn[a * E + e], v4);
  }
}

__global__ void invert_kernel(int64_t n, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = 1.0 / x[i];
}

// Runge-Kutta stage combination on the velocity rows:
// out = a0 u0 + a1 (uin + dt/rho F / m); the pressure row of out is u0's.
__global__ void rk_combine_kernel(int64_t N, double a0, double a1, double dt_rho,
                                  const double* __restrict__ u0, const double* __restrict__ uin,
                                  const double* __restrict__ F,
                                  const double* __restrict__ inv_mass, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double s = dt_rho * inv_mass[i];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double stage = uin[k * N + i] + s * F[k * N + i];
      out[k * N + i] = a0 == 0.0 ? a1 * stage : a0 * u0[k * N + i] + a1 * stage;
    }
    out[3 * N + i] = u0[3 * N + i];
  }
}

// out = (float) in, [4][N] (the mixed form's explicit step assembles from a
// float copy of the double state).
__global__ void narrow_kernel(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __double2float_rn(in[i]);
}

// ---------------------------------------------------------------------------
// Assembly kernels.

template <class T>
__device__ __forceinline__ T ldg(const T* p) {
  return __ldg(p);
}

template <class R>
__device__ __forceinline__ void load_geometry(const R* __restrict__ geom, int64_t E, int64_t e,
                                              R c[3][3], R& inv_det, R& rh) {
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int d = 0; d < 3; ++d) c[k][d] = ldg(geom + (3 * k + d) * E + e);
  inv_det = ldg(geom + 9 * E + e);
  rh = ldg(geom + 10 * E + e);
}

// Where an element's geometry (cofactors, 1/detJ, detJ^(-1/3)) comes from:
// the per-mesh cache (an 88-byte streamed record), or the node coordinates
// gathered through the connectivity and formed into the Jacobian in the
// call itself (Sec. V-B's per-element constant gradients, 43 FP64 operations).
struct GeomCached {
  const double* __restrict__ geom;
  __device__ __forceinline__ void get(int64_t E, int64_t e, const int32_t v[4], double c[3][3],
                                      double& inv_det, double& rh) const {
    load_geometry(geom, E, e, c, inv_det, rh);
  }
};
struct GeomRecompute {
  const double* __restrict__ coords;  // [3][N]
  int64_t N;
  __device__ __forceinline__ void get(int64_t E, int64_t e, const int32_t v[4], double c[3][3],
                                      double& inv_det, double& rh) const {
    double X[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int d = 0; d < 3; ++d) X[a][d] = __ldg(coords + d * N + v[a]);
    nsrhs::element_geometry<double, double>(X, c, inv_det, rh);
  }
};

// A result entry as double: itself, or a float widened with integer
// operations (no FP64 instruction).
__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ double to_double(float x) { return nsrhs::widen_f32(x); }

// FP64 forward of element e: streamed connectivity and cached geometry,
// gathered nodal (u, p), register-resident element arithmetic, immediate
// scatter of the 16 entries.
template <int FLAGS, bool COLOUR, class GS = GeomCached>
__device__ __forceinline__ void fwd_fp64_element(int64_t N, int64_t E, int64_t e,
                                                 const int32_t* __restrict__ conn, const GS& gs,
                                                 const double* __restrict__ up,
                                                 const ElemParams<double>& P,
                                                 double* __restrict__ rhs) {
  int32_t v[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) v[a] = ldg(conn + a * E + e);
  double u[4][3], p[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int i = 0; i < 3; ++i) u[a][i] = ldg(up + i * N + v[a]);
    p[a] = ldg(up + 3 * N + v[a]);
  }
  double c[3][3], inv_det, rh;
  gs.get(E, e, v, c, inv_det, rh);
  double F[4][4];
  nsrhs::element_rhs<double, FLAGS>(c, inv_det, rh, u, p, P, F);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int k = 0; k < 4; ++k) atomicAdd(rhs + k * N + v[a], F[a][k]);
}

// FP64 forward, one element per thread over all elements, atomic scatter.
template <int FLAGS>
__global__ void __launch_bounds__(kThreads, NSRHS_FWD_MIN_CTAS)
    fwd_fp64_atomic_kernel(int64_t N, int64_t E, const int32_t* __restrict__ conn,
                           const double* __restrict__ geom, const double* __restrict__ up,
                           ElemParams<double> P, double* __restrict__ rhs) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x)
    fwd_fp64_element<FLAGS, false>(N, E, e, conn, GeomCached{geom}, up, P, rhs);
}

// FP64 forward with the element geometry formed from the gathered node
// coordinates in the call (no cached geometry read), atomic scatter.
template <int FLAGS>
__global__ void __launch_bounds__(kThreads, NSRHS_FWD_MIN_CTAS)
    fwd_fp64_recompute_kernel(int64_t N, int64_t E, const int32_t* __restrict__ conn,
                              const double* __restrict__ coords, const double* __restrict__ up,
                              ElemParams<double> P, double* __restrict__ rhs) {
  const GeomRecompute gs{coords, N};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x)
    fwd_fp64_element<FLAGS, false>(N, E, e, conn, gs, up, P, rhs);
}

// FP64 forward over the elements [e0, e1) of one colour of the colour-major
// copy (row stride E). No two elements of a colour share a node, so every
// address receives at most one atomic in the launch, and the colour order
// fixes the summation order: the result is bitwise reproducible.
template <int FLAGS>
__global__ void __launch_bounds__(kThreads, NSRHS_FWD_COLOUR_MIN_CTAS)
    fwd_fp64_colour_kernel(int64_t N, int64_t E, int64_t e0, int64_t e1,
                           const int32_t* __restrict__ conn, const double* __restrict__ geom,
                           const double* __restrict__ up, ElemParams<double> P,
                           double* __restrict__ rhs) {
  for (int64_t e = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < e1;
       e += (int64_t)gridDim.x * blockDim.x)
    fwd_fp64_element<FLAGS, true>(N, E, e, conn, GeomCached{geom}, up, P, rhs);
}

// Element-matrix comparison kernel: the same RHS through a full 16x16
// element matrix per tet (elmat.cuh), then the same atomic scatter.
template <bool VREMAN>
__global__ void __launch_bounds__(kThreads)
    fwd_fp64_elmat_kernel(int64_t N, int64_t E, const int32_t* __restrict__ conn,
                          const double* __restrict__ geom, const double* __restrict__ up,
                          ElemParams<double> P, double* __restrict__ rhs) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t v[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) v[a] = ldg(conn + a * E + e);
    double u[4][3], p[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
      for (int i = 0; i < 3; ++i) u[a][i] = ldg(up + i * N + v[a]);
      p[a] = ldg(up + 3 * N + v[a]);
    }
    double c[3][3], inv_det, rh;
    load_geometry(geom, E, e, c, inv_det, rh);
    double F[4][4];
    nsrhs::element_rhs_by_matrix<VREMAN>(c, inv_det, rh, u, p, P, F);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int k = 0; k < 4; ++k) atomicAdd(rhs + k * N + v[a], F[a][k]);
  }
}

// Mixed form of element e: float (u, p) and float element arithmetic on the
// cached geometry (computed in double for every element, so the determinant
// and inverse of high-aspect-ratio elements are double-accurate), double
// global accumulation; float results are widened to double with integer
// operations.
template <int FLAGS, bool COLOUR>
__device__ __forceinline__ void fwd_mixed_element(int64_t N, int64_t E, int64_t e,
                                                  const int32_t* __restrict__ conn,
                                                  const nsrhs::RecChunk* __restrict__ rec,
                                                  const float* __restrict__ up,
                                                  const ElemParams<float>& P,
                                                  double* __restrict__ rhs) {
  int32_t v[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) v[a] = ldg(conn + a * E + e);
  float u[4][3], p[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int i = 0; i < 3; ++i) u[a][i] = ldg(up + i * N + v[a]);
    p[a] = ldg(up + 3 * N + v[a]);
  }
  float c[3][3], inv_det, rh;
  nsrhs::load_rec_geometry(rec, e, c, inv_det, rh);
  float F[4][4];
  nsrhs::element_rhs<float, FLAGS>(c, inv_det, rh, u, p, P, F);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int k = 0; k < 4; ++k) atomicAdd(rhs + k * N + v[a], nsrhs::widen_f32(F[a][k]));
}

template <int FLAGS>
__global__ void __launch_bounds__(kThreads)
    fwd_mixed_atomic_kernel(int64_t N, int64_t E, const int32_t* __restrict__ conn,
                            const nsrhs::RecChunk* __restrict__ rec, const float* __restrict__ up,
                            ElemParams<float> P, double* __restrict__ rhs) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x)
    fwd_mixed_element<FLAGS, false>(N, E, e, conn, rec, up, P, rhs);
}

template <int FLAGS>
__global__ void __launch_bounds__(kThreads)
    fwd_mixed_colour_kernel(int64_t N, int64_t E, int64_t e0, int64_t e1,
                            const int32_t* __restrict__ conn,
                            const nsrhs::RecChunk* __restrict__ rec, const float* __restrict__ up,
                            ElemParams<float> P, double* __restrict__ rhs) {
  for (int64_t e = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < e1;
       e += (int64_t)gridDim.x * blockDim.x)
    fwd_mixed_element<FLAGS, true>(N, E, e, conn, rec, up, P, rhs);
}

// FP64 vector-Jacobian product of element e: gather the cotangent at the
// element's nodes (the reverse of the scatter), recompute the element, run
// the reverse sweep, scatter-add the gradient (the reverse of the gather).
template <int FLAGS, bool COLOUR, class GS = GeomCached>
__device__ __forceinline__ void vjp_fp64_element(int64_t N, int64_t E, int64_t e,
                                                 const int32_t* __restrict__ conn, const GS& gs,
                                                 const double* __restrict__ up,
                                                 const double* __restrict__ cot,
                                                 const ElemParams<double>& P,
                                                 double* __restrict__ grad) {
  int32_t v[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) v[a] = ldg(conn + a * E + e);
  double u[4][3], p[4], w[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int i = 0; i < 3; ++i) u[a][i] = ldg(up + i * N + v[a]);
    p[a] = ldg(up + 3 * N + v[a]);
#pragma unroll
    for (int k = 0; k < 4; ++k) w[a][k] = ldg(cot + k * N + v[a]);
  }
  double c[3][3], inv_det, rh;
  gs.get(E, e, v, c, inv_det, rh);
  double gu[4][3], gp[4];
  nsrhs::element_vjp<double, FLAGS>(c, inv_det, rh, u, p, w, P, gu, gp);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int i = 0; i < 3; ++i) atomicAdd(grad + i * N + v[a], gu[a][i]);
    atomicAdd(grad + 3 * N + v[a], gp[a]);
  }
}

template <int FLAGS>
__global__ void __launch_bounds__(kThreads, NSRHS_VJP_MIN_CTAS)
    vjp_fp64_atomic_kernel(int64_t N, int64_t E, const int32_t* __restrict__ conn,
                           const double* __restrict__ geom, const double* __restrict__ up,
                           const double* __restrict__ cot, ElemParams<double> P,
                           double* __restrict__ grad) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x)
    vjp_fp64_element<FLAGS, false>(N, E, e, conn, GeomCached{geom}, up, cot, P, grad);
}

// FP64 adjoint with the element geometry formed from the gathered node
// coordinates in the call, atomic scatter.
template <int FLAGS>
__global__ void __launch_bounds__(kThreads, NSRHS_VJP_MIN_CTAS)
    vjp_fp64_recompute_kernel(int64_t N, int64_t E, const int32_t* __restrict__ conn,
                              const double* __restrict__ coords, const double* __restrict__ up,
                              const double* __restrict__ cot, ElemParams<double> P,
                              double* __restrict__ grad) {
  const GeomRecompute gs{coords, N};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x)
    vjp_fp64_element<FLAGS, false>(N, E, e, conn, gs, up, cot, P, grad);
}

template <int FLAGS>
__global__ void __launch_bounds__(kThreads, NSRHS_VJP_COLOUR_MIN_CTAS)
    vjp_fp64_colour_kernel(int64_t N, int64_t E, int64_t e0, int64_t e1,
                           const int32_t* __restrict__ conn, const double* __restrict__ geom,
                           const double* __restrict__ up, const double* __restrict__ cot,
                           ElemParams<double> P, double* __restrict__ grad) {
  for (int64_t e = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < e1;
       e += (int64_t)gridDim.x * blockDim.x)
    vjp_fp64_element<FLAGS, true>(N, E, e, conn, GeomCached{geom}, up, cot, P, grad);
}

// Mixed-precision vector-Jacobian product of element e: float (u, p), float
// cotangent, float reverse sweep on the float geometry, double accumulation
// of the gradient.
template <int FLAGS, bool COLOUR>
__device__ __forceinline__ void vjp_mixed_element(int64_t N, int64_t E, int64_t e,
                                                  const int32_t* __restrict__ conn,
                                                  const nsrhs::RecChunk* __restrict__ rec,
                                                  const float* __restrict__ up,
                                                  const float* __restrict__ cot,
                                                  const ElemParams<float>& P,
                                                  double* __restrict__ grad) {
  int32_t v[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) v[a] = ldg(conn + a * E + e);
  float u[4][3], p[4], w[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int i = 0; i < 3; ++i) u[a][i] = ldg(up + i * N + v[a]);
    p[a] = ldg(up + 3 * N + v[a]);
#pragma unroll
    for (int k = 0; k < 4; ++k) w[a][k] = ldg(cot + k * N + v[a]);
  }
  float c[3][3], inv_det, rh;
  nsrhs::load_rec_geometry(rec, e, c, inv_det, rh);
  float gu[4][3], gp[4];
  nsrhs::element_vjp<float, FLAGS>(c, inv_det, rh, u, p, w, P, gu, gp);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
      atomicAdd(grad + i * N + v[a], nsrhs::widen_f32(gu[a][i]));
    atomicAdd(grad + 3 * N + v[a], nsrhs::widen_f32(gp[a]));
  }
}

template <int FLAGS>
__global__ void __launch_bounds__(kThreads)
    vjp_mixed_atomic_kernel(int64_t N, int64_t E, const int32_t* __restrict__ conn,
                            const nsrhs::RecChunk* __restrict__ rec, const float* __restrict__ up,
                            const float* __restrict__ cot, ElemParams<float> P,
                            double* __restrict__ grad) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x)
    vjp_mixed_element<FLAGS, false>(N, E, e, conn, rec, up, cot, P, grad);
}

template <int FLAGS>
__global__ void __launch_bounds__(kThreads)
    vjp_mixed_colour_kernel(int64_t N, int64_t E, int64_t e0, int64_t e1,
                            const int32_t* __restrict__ conn,
                            const nsrhs::RecChunk* __restrict__ rec, const float* __restrict__ up,
                            const float* __restrict__ cot, ElemParams<float> P,
                            double* __restrict__ grad) {
  for (int64_t e = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < e1;
       e += (int64_t)gridDim.x * blockDim.x)
    vjp_mixed_element<FLAGS, true>(N, E, e, conn, rec, up, cot, P, grad);
}

// The RHS and the vector-Jacobian product at the same state in one pass
// (element_rhs_vjp): one gather of (u, p) and the cotangent, one geometry
// read, the forward intermediates computed once; R = double (FP64) or float
// (mixed: float arithmetic, double accumulation by integer widening).
template <class R, int FLAGS, class G>
__global__ void __launch_bounds__(kThreads, NSRHS_VJP_MIN_CTAS)
    rhs_vjp_atomic_kernel(int64_t N, int64_t E, const int32_t* __restrict__ conn,
                          const G* __restrict__ geom, const R* __restrict__ up,
                          const R* __restrict__ cot, ElemParams<R> P, double* __restrict__ rhs,
                          double* __restrict__ grad) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t v[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) v[a] = ldg(conn + a * E + e);
    R u[4][3], p[4], w[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
      for (int i = 0; i < 3; ++i) u[a][i] = ldg(up + i * N + v[a]);
      p[a] = ldg(up + 3 * N + v[a]);
#pragma unroll
      for (int k = 0; k < 4; ++k) w[a][k] = ldg(cot + k * N + v[a]);
    }
    R c[3][3], inv_det, rh;
    nsrhs::block_geometry(reinterpret_cast<const nsrhs::RecChunk*>(geom),
                          reinterpret_cast<const double*>(geom), E, e, c, inv_det, rh);
    R F[4][4], gu[4][3], gp[4];
    nsrhs::element_rhs_vjp<R, FLAGS>(c, inv_det, rh, u, p, w, P, F, gu, gp);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
      for (int k = 0; k < 4; ++k) atomicAdd(rhs + k * N + v[a], to_double(F[a][k]));
#pragma unroll
      for (int i = 0; i < 3; ++i) atomicAdd(grad + i * N + v[a], to_double(gu[a][i]));
      atomicAdd(grad + 3 * N + v[a], to_double(gp[a]));
    }
  }
}

// ---------------------------------------------------------------------------

// Makes the mesh's device current for the duration of a call and restores
// the caller's device afterwards (launches and pointers belong to one device).
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int device) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      ok = false;
      prev = -1;
      return;
    }
    if (prev != device) ok = cudaSetDevice(device) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Calls f(std::integral_constant<int, FLAGS>) for the runtime formulation flags.
template <class Fn>
void with_flags(int flags, Fn&& f) {
  switch (flags & 7) {
    case 0: f(std::integral_constant<int, 0>{}); break;
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 5: f(std::integral_constant<int, 5>{}); break;
    case 6: f(std::integral_constant<int, 6>{}); break;
    default: f(std::integral_constant<int, 7>{}); break;
  }
}

int formulation_flags(const nsrhs_params* p) {
  return (p->c_vreman != 0.0 ? nsrhs::kVreman : 0) |
         (p->convection == NSRHS_SKEW ? nsrhs::kSkew : 0) |
         (p->tau_mode == NSRHS_TAU_ELEMENT ? nsrhs::kTauElem : 0);
}

nsrhs_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return NSRHS_OK;
  if (e == cudaErrorMemoryAllocation) return NSRHS_ENOMEM;
  return NSRHS_ECUDA;
}

#define NSRHS_TRY(expr)                              \
  do {                                               \
    nsrhs_status _s = cuda_status(expr);             \
    if (_s != NSRHS_OK) return _s;                   \
  } while (0)

nsrhs_status check_params(const nsrhs_params* p) {
  if (!p) return NSRHS_EINVAL;
  if (!(p->rho >= 0.0) || !(p->mu > 0.0) || !(p->c_vreman >= 0.0) || !(p->c1 > 0.0) ||
      !(p->c2 >= 0.0) || !std::isfinite(p->rho) || !std::isfinite(p->mu) ||
      !std::isfinite(p->c_vreman) || !std::isfinite(p->c1) || !std::isfinite(p->c2))
    return NSRHS_EINVAL;
  if (p->precision != NSRHS_FP64 && p->precision != NSRHS_MIXED) return NSRHS_EINVAL;
  if (p->scatter < NSRHS_SCATTER_AUTO || p->scatter > NSRHS_SCATTER_BLOCK_COLOUR)
    return NSRHS_EINVAL;
  if (p->convection != NSRHS_CONVECTIVE && p->convection != NSRHS_SKEW) return NSRHS_EINVAL;
  if (p->tau_mode != NSRHS_TAU_GAUSS && p->tau_mode != NSRHS_TAU_ELEMENT) return NSRHS_EINVAL;
  if (p->geometry != NSRHS_GEOM_CACHED && p->geometry != NSRHS_GEOM_RECOMPUTE) return NSRHS_EINVAL;
  if (p->reserved != 0) return NSRHS_EINVAL;
  return NSRHS_OK;
}

// Whether the block kernels' shared memory (W values per staged node: 4 for
// the forward, 8 for the adjoint) fits one CTA on the mesh's device; a mesh
// whose largest block touches very many distinct nodes may not fit the FP64
// adjoint's pipeline (NSRHS_EUNSUPPORTED).
bool block_smem_fits(const nsrhs_mesh* m, const nsrhs_params* p, int W, int entry_buffers = 1) {
  size_t need;
  if (p->precision == NSRHS_FP64)
    need = W == 4 ? nsrhs::block_smem_bytes<double, 4>(m->blk_cap, entry_buffers)
                  : nsrhs::block_smem_bytes<double, 8>(m->blk_cap, entry_buffers);
  else
    need = W == 4 ? nsrhs::block_smem_bytes<float, 4>(m->blk_cap, entry_buffers)
                  : nsrhs::block_smem_bytes<float, 8>(m->blk_cap, entry_buffers);
  return need <= smem_limit(m->device);
}

// The geometry-recompute path exists for the FP64 atomic forward and adjoint.
bool recompute_supported(const nsrhs_params* p) {
  return p->precision == NSRHS_FP64 &&
         (p->scatter == NSRHS_SCATTER_AUTO || p->scatter == NSRHS_SCATTER_ATOMIC);
}

template <class R>
ElemParams<R> elem_params(const nsrhs_params* p) {
  return ElemParams<R>{(R)p->rho, (R)p->mu, (R)p->c_vreman, (R)p->c1, (R)p->c2};
}

void free_mesh(nsrhs_mesh* m) {
  if (!m) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(m->device);
  for (void* ptr : m->allocations) cudaFree(ptr);
  cudaSetDevice(prev);
  delete m;
}

template <class T>
nsrhs_status mesh_alloc(nsrhs_mesh* m, T** ptr, size_t count) {
  *ptr = nullptr;
  if (count == 0) return NSRHS_OK;
  cudaError_t e = cudaMalloc((void**)ptr, count * sizeof(T));
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? NSRHS_ENOMEM : NSRHS_ECUDA;
  }
  m->allocations.push_back(*ptr);
  m->info.device_bytes += (int64_t)(count * sizeof(T));
  return NSRHS_OK;
}

// Scoped device buffer for setup temporaries.
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes ? bytes : 1); }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

// Sorts the elements by the Morton code of their centroids (conn is permuted
// in place); if keep_order is not NULL it receives the caller's index of
// each element in the new order.
nsrhs_status morton_reorder(nsrhs_mesh* m, int32_t* keep_order, cudaStream_t s) {
  const int64_t N = m->n_nodes, E = m->n_elems;
  DevBuf box, keys, keys2, ids, ids2, tmp, conn2;
  NSRHS_TRY(box.alloc(6 * sizeof(unsigned long long)));
  const unsigned long long init[6] = {~0ull, ~0ull, ~0ull, 0ull, 0ull, 0ull};
  NSRHS_TRY(cudaMemcpyAsync(box.p, init, sizeof(init), cudaMemcpyHostToDevice, s));
  nsrhs::bbox_kernel<<<grid_for(N, m->device, 4), kThreads, 0, s>>>(N, m->coords,
                                                                    box.as<unsigned long long>());
  NSRHS_TRY(cudaGetLastError());
  unsigned long long hb[6];
  NSRHS_TRY(cudaMemcpyAsync(hb, box.p, sizeof(hb), cudaMemcpyDeviceToHost, s));
  NSRHS_TRY(cudaStreamSynchronize(s));
  double lo[3], sc[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = nsrhs::from_ordered_bits(hb[d]);
    const double ext = nsrhs::from_ordered_bits(hb[3 + d]) - lo[d];
    sc[d] = ext > 0.0 ? 2097151.0 / ext : 0.0;
  }
  NSRHS_TRY(keys.alloc(E * sizeof(unsigned long long)));
  NSRHS_TRY(keys2.alloc(E * sizeof(unsigned long long)));
  NSRHS_TRY(ids.alloc(E * sizeof(int32_t)));
  NSRHS_TRY(ids2.alloc(E * sizeof(int32_t)));
  nsrhs::morton_kernel<<<grid_for(E, m->device, 8), kThreads, 0, s>>>(
      N, E, m->coords, m->conn, lo[0], lo[1], lo[2], sc[0], sc[1], sc[2],
      keys.as<unsigned long long>(), ids.as<int32_t>());
  NSRHS_TRY(cudaGetLastError());
  size_t tmp_bytes = 0;
  NSRHS_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, keys.as<unsigned long long>(),
                                            keys2.as<unsigned long long>(), ids.as<int32_t>(),
                                            ids2.as<int32_t>(), (int)E, 0, 63, s));
  NSRHS_TRY(tmp.alloc(tmp_bytes));
  NSRHS_TRY(cub::DeviceRadixSort::SortPairs(tmp.p, tmp_bytes, keys.as<unsigned long long>(),
                                            keys2.as<unsigned long long>(), ids.as<int32_t>(),
                                            ids2.as<int32_t>(), (int)E, 0, 63, s));
  NSRHS_TRY(conn2.alloc(4 * E * sizeof(int32_t)));
  nsrhs::permute_conn_kernel<<<grid_for(E, m->device, 8), kThreads, 0, s>>>(
      E, m->conn, ids2.as<int32_t>(), conn2.as<int32_t>());
  NSRHS_TRY(cudaGetLastError());
  NSRHS_TRY(cudaMemcpyAsync(m->conn, conn2.p, 4 * E * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  if (keep_order)
    NSRHS_TRY(cudaMemcpyAsync(keep_order, ids2.p, E * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  NSRHS_TRY(cudaStreamSynchronize(s));
  return NSRHS_OK;
}

nsrhs_status build_blocks(nsrhs_mesh* m, cudaStream_t s) {
  const int64_t E = m->n_elems;
  const int64_t nb = (E + nsrhs::kBlockElems - 1) / nsrhs::kBlockElems;
  if (nb > INT32_MAX) return NSRHS_EINVAL;
  m->n_blocks = nb;
  nsrhs_status st;
  DevBuf counts, tmp;
  NSRHS_TRY(counts.alloc((nb + 1) * sizeof(int64_t)));
  if ((st = mesh_alloc(m, &m->blk_node_off, (size_t)nb + 1)) != NSRHS_OK) return st;
  // pass 0: distinct nodes per block
  nsrhs::block_plan_kernel<<<(unsigned)nb, nsrhs::kBlockElems, 0, s>>>(
      0, E, m->conn, counts.as<int64_t>(), nullptr, nullptr, nullptr, nullptr);
  NSRHS_TRY(cudaGetLastError());
  // node_off = exclusive prefix sum of the counts (counts[nb] = 0)
  {
    NSRHS_TRY(cudaMemsetAsync(counts.as<int64_t>() + nb, 0, sizeof(int64_t), s));
    size_t tmp_bytes = 0;
    NSRHS_TRY(cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, counts.as<int64_t>(),
                                            m->blk_node_off, (int)nb + 1, s));
    NSRHS_TRY(tmp.alloc(tmp_bytes));
    NSRHS_TRY(cub::DeviceScan::ExclusiveSum(tmp.p, tmp_bytes, counts.as<int64_t>(),
                                            m->blk_node_off, (int)nb + 1, s));
  }
  // the largest block's distinct-node count sizes the staging buffers
  DevBuf dmax, tmp2;
  NSRHS_TRY(dmax.alloc(sizeof(int64_t)));
  {
    size_t tmp_bytes = 0;
    NSRHS_TRY(cub::DeviceReduce::Max(nullptr, tmp_bytes, counts.as<int64_t>(), dmax.as<int64_t>(),
                                     (int)nb, s));
    NSRHS_TRY(tmp2.alloc(tmp_bytes));
    NSRHS_TRY(cub::DeviceReduce::Max(tmp2.p, tmp_bytes, counts.as<int64_t>(), dmax.as<int64_t>(),
                                     (int)nb, s));
  }
  int64_t total = 0, max_distinct = 0;
  NSRHS_TRY(cudaMemcpyAsync(&total, m->blk_node_off + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  NSRHS_TRY(cudaMemcpyAsync(&max_distinct, dmax.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  NSRHS_TRY(cudaStreamSynchronize(s));
  if (max_distinct < 1 || max_distinct > nsrhs::kBlockSlots) return NSRHS_ECUDA;
  m->blk_cap = (int)std::min<int64_t>(nsrhs::kBlockSlots, (max_distinct + 31) / 32 * 32);
  if ((st = mesh_alloc(m, &m->blk_nodes, (size_t)total)) != NSRHS_OK) return st;
  if ((st = mesh_alloc(m, &m->blk_runs, (size_t)total)) != NSRHS_OK) return st;
  nsrhs::block_plan_kernel<<<(unsigned)nb, nsrhs::kBlockElems, 0, s>>>(
      1, E, m->conn, nullptr, m->blk_node_off, m->blk_nodes, m->blk_runs, m->rec);
  NSRHS_TRY(cudaGetLastError());
  return NSRHS_OK;
}

// Colours the elements (colour.cuh), checks the colouring independently and
// builds the colour-major copy of the connectivity and cached geometry.
nsrhs_status build_colouring(nsrhs_mesh* m, cudaStream_t s) {
  using ull = unsigned long long;
  const int64_t N = m->n_nodes, E = m->n_elems;
  nsrhs_status st;
  if ((st = mesh_alloc(m, &m->colour, (size_t)E)) != NSRHS_OK) return st;
  DevBuf claim, used, counters, counts, ids, ids_sorted, keys_sorted, tmp;
  NSRHS_TRY(claim.alloc(N * sizeof(ull)));
  NSRHS_TRY(used.alloc(2 * N * sizeof(ull)));
  NSRHS_TRY(counters.alloc(2 * sizeof(ull)));
  NSRHS_TRY(cudaMemsetAsync(m->colour, nsrhs::kUncoloured, (size_t)E, s));
  NSRHS_TRY(cudaMemsetAsync(used.p, 0, 2 * N * sizeof(ull), s));
  NSRHS_TRY(cudaMemsetAsync(counters.p, 0, 2 * sizeof(ull), s));
  const unsigned grid = grid_for(E, m->device, 8);
  ull hc[2] = {0, 0};
  while (hc[0] < (ull)E) {
    const ull before = hc[0];
    NSRHS_TRY(cudaMemsetAsync(claim.p, 0xFF, N * sizeof(ull), s));
    nsrhs::colour_claim_kernel<<<grid, kThreads, 0, s>>>(E, m->conn, m->colour, claim.as<ull>());
    NSRHS_TRY(cudaGetLastError());
    nsrhs::colour_accept_kernel<<<grid, kThreads, 0, s>>>(E, m->conn, claim.as<ull>(),
                                                          used.as<ull>(), m->colour,
                                                          counters.as<ull>());
    NSRHS_TRY(cudaGetLastError());
    NSRHS_TRY(cudaMemcpyAsync(hc, counters.p, sizeof(hc), cudaMemcpyDeviceToHost, s));
    NSRHS_TRY(cudaStreamSynchronize(s));
    if (hc[1] != 0) return NSRHS_EUNSUPPORTED;  // needs more than kMaxColours colours
    if (hc[0] == before) return NSRHS_ECUDA;    // no progress: cannot happen
  }
  // independent check: no colour twice at a node
  NSRHS_TRY(cudaMemsetAsync(used.p, 0, 2 * N * sizeof(ull), s));
  NSRHS_TRY(cudaMemsetAsync(counters.p, 0, 2 * sizeof(ull), s));
  nsrhs::colour_check_kernel<<<grid, kThreads, 0, s>>>(E, m->conn, m->colour, used.as<ull>(),
                                                       counters.as<ull>());
  NSRHS_TRY(cudaGetLastError());
  NSRHS_TRY(counts.alloc(nsrhs::kMaxColours * sizeof(ull)));
  NSRHS_TRY(cudaMemsetAsync(counts.p, 0, nsrhs::kMaxColours * sizeof(ull), s));
  nsrhs::colour_count_kernel<<<grid, kThreads, 0, s>>>(E, m->colour, counts.as<ull>());
  NSRHS_TRY(cudaGetLastError());
  ull hcount[nsrhs::kMaxColours];
  NSRHS_TRY(cudaMemcpyAsync(hc, counters.p, sizeof(hc), cudaMemcpyDeviceToHost, s));
  NSRHS_TRY(cudaMemcpyAsync(hcount, counts.p, sizeof(hcount), cudaMemcpyDeviceToHost, s));
  NSRHS_TRY(cudaStreamSynchronize(s));
  if (hc[0] != 0) return NSRHS_ECUDA;
  int n_col = 0;
  for (int k = 0; k < nsrhs::kMaxColours; ++k)
    if (hcount[k]) n_col = k + 1;
  m->col_off.assign(n_col + 1, 0);
  for (int k = 0; k < n_col; ++k) m->col_off[k + 1] = m->col_off[k] + (int64_t)hcount[k];
  if (m->col_off[n_col] != E) return NSRHS_ECUDA;
  // colour-major order: a stable sort of the element indices by colour
  NSRHS_TRY(ids.alloc(E * sizeof(int32_t)));
  NSRHS_TRY(ids_sorted.alloc(E * sizeof(int32_t)));
  NSRHS_TRY(keys_sorted.alloc((size_t)E));
  nsrhs::iota_kernel<<<grid, kThreads, 0, s>>>(E, ids.as<int32_t>());
  NSRHS_TRY(cudaGetLastError());
  size_t tmp_bytes = 0;
  NSRHS_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, m->colour, keys_sorted.as<uint8_t>(),
                                            ids.as<int32_t>(), ids_sorted.as<int32_t>(), (int)E, 0,
                                            8, s));
  NSRHS_TRY(tmp.alloc(tmp_bytes));
  NSRHS_TRY(cub::DeviceRadixSort::SortPairs(tmp.p, tmp_bytes, m->colour, keys_sorted.as<uint8_t>(),
                                            ids.as<int32_t>(), ids_sorted.as<int32_t>(), (int)E, 0,
                                            8, s));
  if ((st = mesh_alloc(m, &m->col_conn, 4 * (size_t)E)) != NSRHS_OK) return st;
  if ((st = mesh_alloc(m, &m->col_geom, kGeomRows * (size_t)E)) != NSRHS_OK) return st;
  if ((st = mesh_alloc(m, &m->col_rec, (size_t)nsrhs::rec_chunks(E))) != NSRHS_OK) return st;
  const int32_t* perm = ids_sorted.as<int32_t>();
  nsrhs::permute_rows_kernel<int32_t><<<grid, kThreads, 0, s>>>(4, E, perm, m->conn, m->col_conn);
  NSRHS_TRY(cudaGetLastError());
  nsrhs::permute_rows_kernel<double><<<grid, kThreads, 0, s>>>(kGeomRows, E, perm, m->geom,
                                                               m->col_geom);
  NSRHS_TRY(cudaGetLastError());
  nsrhs::permute_records_kernel<<<grid, kThreads, 0, s>>>(E, perm, m->rec, m->col_rec);
  NSRHS_TRY(cudaGetLastError());
  NSRHS_TRY(cudaStreamSynchronize(s));
  m->info.n_colours = n_col;
  return NSRHS_OK;
}

// Colours the element blocks (colour.cuh), checks the colouring and lists the
// blocks of each colour.
nsrhs_status build_block_colouring(nsrhs_mesh* m, cudaStream_t s) {
  using ull = unsigned long long;
  const int64_t N = m->n_nodes, nb = m->n_blocks;
  nsrhs_status st;
  if ((st = mesh_alloc(m, &m->bcolour, (size_t)nb)) != NSRHS_OK) return st;
  DevBuf claim, used, counters, counts, ids, keys_sorted, tmp;
  NSRHS_TRY(claim.alloc(N * sizeof(ull)));
  NSRHS_TRY(used.alloc(2 * N * sizeof(ull)));
  NSRHS_TRY(counters.alloc(2 * sizeof(ull)));
  NSRHS_TRY(cudaMemsetAsync(m->bcolour, nsrhs::kUncoloured, (size_t)nb, s));
  NSRHS_TRY(cudaMemsetAsync(used.p, 0, 2 * N * sizeof(ull), s));
  NSRHS_TRY(cudaMemsetAsync(counters.p, 0, 2 * sizeof(ull), s));
  // one warp per block
  const unsigned grid = grid_for(32 * nb, m->device, 8);
  ull hc[2] = {0, 0};
  while (hc[0] < (ull)nb) {
    const ull before = hc[0];
    NSRHS_TRY(cudaMemsetAsync(claim.p, 0xFF, N * sizeof(ull), s));
    nsrhs::block_colour_claim_kernel<<<grid, kThreads, 0, s>>>(
        nb, m->blk_node_off, m->blk_nodes, m->bcolour, claim.as<ull>());
    NSRHS_TRY(cudaGetLastError());
    nsrhs::block_colour_accept_kernel<<<grid, kThreads, 0, s>>>(
        nb, m->blk_node_off, m->blk_nodes, claim.as<ull>(), used.as<ull>(), m->bcolour,
        counters.as<ull>());
    NSRHS_TRY(cudaGetLastError());
    NSRHS_TRY(cudaMemcpyAsync(hc, counters.p, sizeof(hc), cudaMemcpyDeviceToHost, s));
    NSRHS_TRY(cudaStreamSynchronize(s));
    if (hc[1] != 0) return NSRHS_EUNSUPPORTED;  // needs more than kMaxColours colours
    if (hc[0] == before) return NSRHS_ECUDA;    // no progress: cannot happen
  }
  NSRHS_TRY(cudaMemsetAsync(used.p, 0, 2 * N * sizeof(ull), s));
  NSRHS_TRY(cudaMemsetAsync(counters.p, 0, 2 * sizeof(ull), s));
  nsrhs::block_colour_check_kernel<<<grid, kThreads, 0, s>>>(
      nb, m->blk_node_off, m->blk_nodes, m->bcolour, used.as<ull>(), counters.as<ull>());
  NSRHS_TRY(cudaGetLastError());
  NSRHS_TRY(counts.alloc(nsrhs::kMaxColours * sizeof(ull)));
  NSRHS_TRY(cudaMemsetAsync(counts.p, 0, nsrhs::kMaxColours * sizeof(ull), s));
  const unsigned grid1 = grid_for(nb, m->device, 8);
  nsrhs::colour_count_kernel<<<grid1, kThreads, 0, s>>>(nb, m->bcolour, counts.as<ull>());
  NSRHS_TRY(cudaGetLastError());
  ull hcount[nsrhs::kMaxColours];
  NSRHS_TRY(cudaMemcpyAsync(hc, counters.p, sizeof(hc), cudaMemcpyDeviceToHost, s));
  NSRHS_TRY(cudaMemcpyAsync(hcount, counts.p, sizeof(hcount), cudaMemcpyDeviceToHost, s));
  NSRHS_TRY(cudaStreamSynchronize(s));
  if (hc[0] != 0) return NSRHS_ECUDA;
  int n_col = 0;
  for (int k = 0; k < nsrhs::kMaxColours; ++k)
    if (hcount[k]) n_col = k + 1;
  m->bcol_off.assign(n_col + 1, 0);
  for (int k = 0; k < n_col; ++k) m->bcol_off[k + 1] = m->bcol_off[k] + (int64_t)hcount[k];
  if (m->bcol_off[n_col] != nb) return NSRHS_ECUDA;
  if ((st = mesh_alloc(m, &m->bcol_order, (size_t)nb)) != NSRHS_OK) return st;
  NSRHS_TRY(ids.alloc(nb * sizeof(int32_t)));
  NSRHS_TRY(keys_sorted.alloc((size_t)nb));
  nsrhs::iota_kernel<<<grid1, kThreads, 0, s>>>(nb, ids.as<int32_t>());
  NSRHS_TRY(cudaGetLastError());
  size_t tmp_bytes = 0;
  NSRHS_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, m->bcolour,
                                            keys_sorted.as<uint8_t>(), ids.as<int32_t>(),
                                            m->bcol_order, (int)nb, 0, 8, s));
  NSRHS_TRY(tmp.alloc(tmp_bytes));
  NSRHS_TRY(cub::DeviceRadixSort::SortPairs(tmp.p, tmp_bytes, m->bcolour,
                                            keys_sorted.as<uint8_t>(), ids.as<int32_t>(),
                                            m->bcol_order, (int)nb, 0, 8, s));
  NSRHS_TRY(cudaStreamSynchronize(s));
  m->info.n_block_colours = n_col;
  return NSRHS_OK;
}

nsrhs_status mesh_build(nsrhs_mesh* m, const double* coords, const int32_t* conn,
                        const nsrhs_mesh_opts& opts, cudaStream_t s) {
  const int64_t N = m->n_nodes, E = m->n_elems;
  nsrhs_status st;
  if ((st = mesh_alloc(m, &m->coords, 3 * (size_t)N)) != NSRHS_OK) return st;
  if ((st = mesh_alloc(m, &m->conn, 4 * (size_t)E)) != NSRHS_OK) return st;
  NSRHS_TRY(cudaMemcpyAsync(m->coords, coords, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s));
  NSRHS_TRY(cudaMemcpyAsync(m->conn, conn, sizeof(int32_t) * 4 * E, cudaMemcpyDeviceToDevice, s));

  // Validation scratch (freed before returning).
  uint8_t* high_ar = nullptr;
  ValidateOut* vout = nullptr;
  NSRHS_TRY(cudaMalloc((void**)&high_ar, (size_t)E));
  cudaError_t ce = cudaMalloc((void**)&vout, sizeof(ValidateOut));
  if (ce != cudaSuccess) {
    cudaFree(high_ar);
    return cuda_status(ce);
  }
  ValidateOut init{};
  init.min_det_bits = (unsigned long long)0x7FF0000000000000ull;  // +inf
  init.max_ar_bits = 0ull;
  ValidateOut res{};
  ce = cudaMemcpyAsync(vout, &init, sizeof(init), cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) {
    validate_kernel<<<grid_for(E, m->device, 8), kThreads, 0, s>>>(N, E, m->coords, m->conn,
                                                                  opts.ar_threshold, high_ar, vout);
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(&res, vout, sizeof(res), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  cudaFree(high_ar);
  cudaFree(vout);
  if (ce != cudaSuccess) return cuda_status(ce);
  if (res.bad_index != 0 || res.bad_det != 0) return NSRHS_EMESH;

  double min_det, max_ar;
  std::memcpy(&min_det, &res.min_det_bits, sizeof(double));
  std::memcpy(&max_ar, &res.max_ar_bits, sizeof(double));
  m->info.min_detj = min_det;
  m->info.max_ar = max_ar;
  m->info.n_high_ar = (int64_t)res.n_high_ar;

  // Morton order of the element centroids (the RHS does not depend on the
  // element order, up to rounding).
  if (opts.colour && (st = mesh_alloc(m, &m->elem_order, (size_t)E)) != NSRHS_OK) return st;
  if ((st = morton_reorder(m, m->elem_order, s)) != NSRHS_OK) return st;
  // Cached geometry (double and float) of every element.
  if ((st = mesh_alloc(m, &m->geom, kGeomRows * (size_t)E)) != NSRHS_OK) return st;
  if ((st = mesh_alloc(m, &m->rec, (size_t)nsrhs::rec_chunks(E))) != NSRHS_OK) return st;
  geometry_kernel<<<grid_for(E, m->device, 8), kThreads, 0, s>>>(N, E, m->coords, m->conn,
                                                                 m->geom, m->rec);
  NSRHS_TRY(cudaGetLastError());
  if ((st = build_blocks(m, s)) != NSRHS_OK) return st;
  if (opts.colour && (st = build_colouring(m, s)) != NSRHS_OK) return st;
  if (opts.colour && (st = build_block_colouring(m, s)) != NSRHS_OK) return st;
  // Lumped mass and its inverse (explicit time stepping).
  if ((st = mesh_alloc(m, &m->mass, (size_t)N)) != NSRHS_OK) return st;
  if ((st = mesh_alloc(m, &m->inv_mass, (size_t)N)) != NSRHS_OK) return st;
  NSRHS_TRY(cudaMemsetAsync(m->mass, 0, sizeof(double) * N, s));
  lumped_mass_kernel<<<grid_for(E, m->device, 8), kThreads, 0, s>>>(E, m->conn, m->geom, m->mass);
  NSRHS_TRY(cudaGetLastError());
  invert_kernel<<<grid_for(N, m->device, 8), kThreads, 0, s>>>(N, m->mass, m->inv_mass);
  NSRHS_TRY(cudaGetLastError());
  NSRHS_TRY(cudaStreamSynchronize(s));
  m->info.n_nodes = N;
  m->info.n_elems = E;
  m->info.n_blocks = m->n_blocks;
  m->info.block_elems = nsrhs::kBlockElems;
  return NSRHS_OK;
}

}  // namespace

extern "C" {

void nsrhs_params_default(nsrhs_params* p) {
  if (!p) return;
  p->rho = 1.0;
  p->mu = 1e-2;
  p->c_vreman = 0.0;
  p->c1 = 4.0;
  p->c2 = 2.0;
  p->precision = NSRHS_FP64;
  p->scatter = NSRHS_SCATTER_AUTO;
  p->convection = NSRHS_CONVECTIVE;
  p->tau_mode = NSRHS_TAU_GAUSS;
  p->geometry = NSRHS_GEOM_CACHED;
  p->reserved = 0;
}

void nsrhs_mesh_opts_default(nsrhs_mesh_opts* o) {
  if (!o) return;
  o->ar_threshold = 10.0;
  o->colour = 0;
  o->reserved = 0;
}

const char* nsrhs_status_string(nsrhs_status s) {
  switch (s) {
    case NSRHS_OK: return "ok";
    case NSRHS_EINVAL: return "invalid argument";
    case NSRHS_ENOMEM: return "device out of memory";
    case NSRHS_EMESH: return "invalid mesh (index out of range or detJ <= 0)";
    case NSRHS_ECUDA: return "CUDA error";
    case NSRHS_EUNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

nsrhs_status nsrhs_mesh_create(int64_t n_nodes, int64_t n_elems, const double* coords,
                               const int32_t* conn, const nsrhs_mesh_opts* opts, void* stream,
                               nsrhs_mesh** out) {
  if (!out) return NSRHS_EINVAL;
  *out = nullptr;
  if (!coords || !conn) return NSRHS_EINVAL;
  if (n_nodes < 1 || n_elems < 1 || n_nodes > INT32_MAX || n_elems > INT32_MAX) return NSRHS_EINVAL;
  nsrhs_mesh_opts o;
  nsrhs_mesh_opts_default(&o);
  if (opts) o = *opts;
  if (!(o.ar_threshold > 0.0) || (o.colour != 0 && o.colour != 1) || o.reserved != 0)
    return NSRHS_EINVAL;
  nsrhs_mesh* m = new (std::nothrow) nsrhs_mesh();
  if (!m) return NSRHS_ENOMEM;
  if (cudaGetDevice(&m->device) != cudaSuccess) {
    delete m;
    return NSRHS_ECUDA;
  }
  m->n_nodes = n_nodes;
  m->n_elems = n_elems;
  nsrhs_status st = mesh_build(m, coords, conn, o, (cudaStream_t)stream);
  if (st != NSRHS_OK) {
    free_mesh(m);
    return st;
  }
  {
    std::lock_guard<std::mutex> lock(g_registry_mutex);
    g_registry.insert(m);
  }
  *out = m;
  return NSRHS_OK;
}

nsrhs_status nsrhs_mesh_get_info(const nsrhs_mesh* m, nsrhs_mesh_info* info) {
  if (!is_live(m) || !info) return NSRHS_EINVAL;
  *info = m->info;
  return NSRHS_OK;
}

nsrhs_status nsrhs_assemble(const nsrhs_mesh* m, const nsrhs_params* p, const void* up,
                            double* rhs, void* stream) {
  if (!is_live(m) || !up || !rhs) return NSRHS_EINVAL;
  nsrhs_status st = check_params(p);
  if (st != NSRHS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard dg(m->device);
  if (!dg.ok) return NSRHS_ECUDA;
  const int64_t N = m->n_nodes, E = m->n_elems;
  const int flags = formulation_flags(p);
  if ((p->scatter == NSRHS_SCATTER_COLOUR && m->col_conn == nullptr) ||
      (p->scatter == NSRHS_SCATTER_BLOCK_COLOUR && m->bcol_order == nullptr))
    return NSRHS_EUNSUPPORTED;
  if (p->geometry == NSRHS_GEOM_RECOMPUTE && !recompute_supported(p)) return NSRHS_EUNSUPPORTED;
  const bool block_path = p->scatter == NSRHS_SCATTER_BLOCK ||
                          p->scatter == NSRHS_SCATTER_BLOCK_COLOUR ||
                          (p->scatter == NSRHS_SCATTER_AUTO && p->precision == NSRHS_MIXED);
  if (p->geometry == NSRHS_GEOM_CACHED && block_path && !block_smem_fits(m, p, 4))
    return NSRHS_EUNSUPPORTED;
  NSRHS_TRY(cudaMemsetAsync(rhs, 0, sizeof(double) * 4 * N, s));
  if (p->geometry == NSRHS_GEOM_RECOMPUTE) {
    auto P = elem_params<double>(p);
    with_flags(flags, [&](auto fl) {
      fwd_fp64_recompute_kernel<decltype(fl)::value><<<grid_for(E, m->device, 16), kThreads, 0,
                                                       s>>>(N, E, m->conn, m->coords,
                                                            (const double*)up, P, rhs);
    });
    return cuda_status(cudaGetLastError());
  }
  if (p->scatter == NSRHS_SCATTER_BLOCK_COLOUR) {
    // one launch per block colour, in colour order
    const int64_t nb = m->n_blocks;
    cudaError_t err = cudaSuccess;
    for (size_t k = 0; k + 1 < m->bcol_off.size() && err == cudaSuccess; ++k) {
      const int64_t i0 = m->bcol_off[k], i1 = m->bcol_off[k + 1];
      const unsigned grid = (unsigned)std::max<int64_t>(
          1, std::min<int64_t>(i1 - i0, (int64_t)sm_count(m->device) * kBlockCtasPerSm));
      if (p->precision == NSRHS_FP64) {
        auto P = elem_params<double>(p);
        const size_t smem = nsrhs::block_smem_bytes<double, 4>(m->blk_cap);
        with_flags(flags, [&](auto fl) {
          auto kern = nsrhs::fwd_block_kernel<double, decltype(fl)::value, true>;
          err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
          if (err == cudaSuccess)
            kern<<<grid, nsrhs::kBlockElems, smem, s>>>(
                N, E, nb, m->blk_node_off, m->blk_nodes, m->blk_runs, m->blk_cap, m->rec,
                m->geom, (const double*)up, P, rhs, m->bcol_order, i0, i1);
        });
      } else {
        auto P = elem_params<float>(p);
        const size_t smem = nsrhs::block_smem_bytes<float, 4>(m->blk_cap);
        with_flags(flags, [&](auto fl) {
          auto kern = nsrhs::fwd_block_kernel<float, decltype(fl)::value, true>;
          err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
          if (err == cudaSuccess)
            kern<<<grid, nsrhs::kBlockElems, smem, s>>>(
                N, E, nb, m->blk_node_off, m->blk_nodes, m->blk_runs, m->blk_cap, m->rec,
                nullptr, (const float*)up, P, rhs, m->bcol_order, i0, i1);
        });
      }
      if (err == cudaSuccess) err = cudaGetLastError();
    }
    return cuda_status(err);
  }
  if (p->scatter == NSRHS_SCATTER_COLOUR) {
    // one launch per colour, in colour order
    for (size_t k = 0; k + 1 < m->col_off.size(); ++k) {
      const int64_t e0 = m->col_off[k], e1 = m->col_off[k + 1];
      const unsigned grid = grid_for(e1 - e0, m->device, 16);
      if (p->precision == NSRHS_FP64) {
        auto P = elem_params<double>(p);
        with_flags(flags, [&](auto fl) {
          fwd_fp64_colour_kernel<decltype(fl)::value><<<grid, kThreads, 0, s>>>(
              N, E, e0, e1, m->col_conn, m->col_geom, (const double*)up, P, rhs);
        });
      } else {
        auto P = elem_params<float>(p);
        with_flags(flags, [&](auto fl) {
          fwd_mixed_colour_kernel<decltype(fl)::value><<<grid, kThreads, 0, s>>>(
              N, E, e0, e1, m->col_conn, m->col_rec, (const float*)up, P, rhs);
        });
      }
      NSRHS_TRY(cudaGetLastError());
    }
    return NSRHS_OK;
  }
  // AUTO: atomics for the FP64 form (its FP64 pipe, not the scatter, is the
  // limit, and the block sums would add FP64 work); blocks for the mixed form
  // (bound by L2 atomics and gathers).
  const bool block = p->scatter == NSRHS_SCATTER_BLOCK ||
                     (p->scatter == NSRHS_SCATTER_AUTO && p->precision == NSRHS_MIXED);
  if (block) {
    const int64_t nb = m->n_blocks;
    const unsigned grid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>(nb, (int64_t)sm_count(m->device) * kBlockCtasPerSm));
    cudaError_t err = cudaSuccess;
    if (p->precision == NSRHS_FP64) {
      auto P = elem_params<double>(p);
      const size_t smem = nsrhs::block_smem_bytes<double, 4>(m->blk_cap);
      with_flags(flags, [&](auto fl) {
        auto kern = nsrhs::fwd_block_kernel<double, decltype(fl)::value>;
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err == cudaSuccess)
          kern<<<grid, nsrhs::kBlockElems, smem, s>>>(N, E, nb, m->blk_node_off, m->blk_nodes,
                                                      m->blk_runs, m->blk_cap, m->rec,
                                                      m->geom, (const double*)up, P, rhs,
                                                      nullptr, 0, 0);
      });
    } else {
      auto P = elem_params<float>(p);
      const size_t smem = nsrhs::block_smem_bytes<float, 4>(m->blk_cap);
      with_flags(flags, [&](auto fl) {
        auto kern = nsrhs::fwd_block_kernel<float, decltype(fl)::value>;
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err == cudaSuccess)
          kern<<<grid, nsrhs::kBlockElems, smem, s>>>(N, E, nb, m->blk_node_off, m->blk_nodes,
                                                      m->blk_runs, m->blk_cap, m->rec,
                                                      nullptr, (const float*)up, P, rhs,
                                                      nullptr, 0, 0);
      });
    }
    if (err != cudaSuccess) return cuda_status(err);
    return cuda_status(cudaGetLastError());
  }
  const unsigned grid = grid_for(E, m->device, 16);
  if (p->precision == NSRHS_FP64) {
    auto P = elem_params<double>(p);
    with_flags(flags, [&](auto fl) {
      fwd_fp64_atomic_kernel<decltype(fl)::value>
          <<<grid, kThreads, 0, s>>>(N, E, m->conn, m->geom, (const double*)up, P, rhs);
    });
  } else {
    auto P = elem_params<float>(p);
    with_flags(flags, [&](auto fl) {
      fwd_mixed_atomic_kernel<decltype(fl)::value>
          <<<grid, kThreads, 0, s>>>(N, E, m->conn, m->rec, (const float*)up, P, rhs);
    });
  }
  return cuda_status(cudaGetLastError());
}

nsrhs_status nsrhs_assemble_vjp(const nsrhs_mesh* m, const nsrhs_params* p, const void* up,
                                const void* cot, double* grad, void* stream) {
  if (!is_live(m) || !up || !cot || !grad) return NSRHS_EINVAL;
  nsrhs_status st = check_params(p);
  if (st != NSRHS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard dg(m->device);
  if (!dg.ok) return NSRHS_ECUDA;
  const int64_t N = m->n_nodes, E = m->n_elems;
  if ((p->scatter == NSRHS_SCATTER_COLOUR && m->col_conn == nullptr) ||
      (p->scatter == NSRHS_SCATTER_BLOCK_COLOUR && m->bcol_order == nullptr))
    return NSRHS_EUNSUPPORTED;
  if (p->geometry == NSRHS_GEOM_RECOMPUTE && !recompute_supported(p)) return NSRHS_EUNSUPPORTED;
  const bool block_path = p->scatter == NSRHS_SCATTER_BLOCK ||
                          p->scatter == NSRHS_SCATTER_BLOCK_COLOUR ||
                          (p->scatter == NSRHS_SCATTER_AUTO && p->precision == NSRHS_MIXED);
  if (p->geometry == NSRHS_GEOM_CACHED && block_path && !block_smem_fits(m, p, 8))
    return NSRHS_EUNSUPPORTED;
  NSRHS_TRY(cudaMemsetAsync(grad, 0, sizeof(double) * 4 * N, s));
  const int flags = formulation_flags(p);
  if (p->geometry == NSRHS_GEOM_RECOMPUTE) {
    auto P = elem_params<double>(p);
    with_flags(flags, [&](auto fl) {
      vjp_fp64_recompute_kernel<decltype(fl)::value><<<grid_for(E, m->device, 16), kThreads, 0,
                                                       s>>>(N, E, m->conn, m->coords,
                                                            (const double*)up,
                                                            (const double*)cot, P, grad);
    });
    return cuda_status(cudaGetLastError());
  }
  // AUTO: atomics for the FP64 form (FP64-pipe-bound), blocks for the mixed
  // form (measured faster)
  const bool block = p->scatter == NSRHS_SCATTER_BLOCK ||
                     (p->scatter == NSRHS_SCATTER_AUTO && p->precision == NSRHS_MIXED);
  if (block || p->scatter == NSRHS_SCATTER_BLOCK_COLOUR) {
    // BLOCK: one grid over all blocks; BLOCK_COLOUR: one launch per block
    // colour (the atomics of a launch never meet at one address)
    const bool coloured = p->scatter == NSRHS_SCATTER_BLOCK_COLOUR;
    const int64_t nb = m->n_blocks;
    std::vector<int64_t> ranges = coloured ? m->bcol_off : std::vector<int64_t>{0, nb};
    cudaError_t err = cudaSuccess;
    for (size_t k = 0; k + 1 < ranges.size() && err == cudaSuccess; ++k) {
      const int64_t i0 = ranges[k], i1 = ranges[k + 1];
      const unsigned grid = (unsigned)std::max<int64_t>(
          1, std::min<int64_t>(i1 - i0, (int64_t)sm_count(m->device) * kBlockCtasPerSm));
      auto launch = [&](auto kern, size_t smem, const double* geom, const auto* u, const auto* c,
                        const auto& P) {
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err == cudaSuccess)
          kern<<<grid, nsrhs::kBlockElems, smem, s>>>(
              N, E, nb, m->blk_node_off, m->blk_nodes, m->blk_runs, m->blk_cap, m->rec,
              geom, u, c, P, grad, coloured ? m->bcol_order : nullptr, i0, i1);
      };
      if (p->precision == NSRHS_FP64) {
        auto P = elem_params<double>(p);
        with_flags(flags, [&](auto fl) {
          constexpr int F = decltype(fl)::value;
          if (coloured)
            launch(nsrhs::vjp_block_kernel<double, F, true>, nsrhs::block_smem_bytes<double, 8>(m->blk_cap),
                   m->geom, (const double*)up, (const double*)cot, P);
          else
            launch(nsrhs::vjp_block_kernel<double, F, false>,
                   nsrhs::block_smem_bytes<double, 8>(m->blk_cap), m->geom, (const double*)up,
                   (const double*)cot, P);
        });
      } else {
        auto P = elem_params<float>(p);
        with_flags(flags, [&](auto fl) {
          constexpr int F = decltype(fl)::value;
          if (coloured)
            launch(nsrhs::vjp_block_kernel<float, F, true>, nsrhs::block_smem_bytes<float, 8>(m->blk_cap),
                   nullptr, (const float*)up, (const float*)cot, P);
          else
            launch(nsrhs::vjp_block_kernel<float, F, false>, nsrhs::block_smem_bytes<float, 8>(m->blk_cap),
                   nullptr, (const float*)up, (const float*)cot, P);
        });
      }
      if (err == cudaSuccess) err = cudaGetLastError();
    }
    return cuda_status(err);
  }
  if (p->scatter == NSRHS_SCATTER_COLOUR) {
    for (size_t k = 0; k + 1 < m->col_off.size(); ++k) {
      const int64_t e0 = m->col_off[k], e1 = m->col_off[k + 1];
      const unsigned grid = grid_for(e1 - e0, m->device, 16);
      if (p->precision == NSRHS_FP64) {
        auto P = elem_params<double>(p);
        with_flags(formulation_flags(p), [&](auto fl) {
          vjp_fp64_colour_kernel<decltype(fl)::value><<<grid, kThreads, 0, s>>>(
              N, E, e0, e1, m->col_conn, m->col_geom, (const double*)up, (const double*)cot, P,
              grad);
        });
      } else {
        auto P = elem_params<float>(p);
        with_flags(formulation_flags(p), [&](auto fl) {
          vjp_mixed_colour_kernel<decltype(fl)::value><<<grid, kThreads, 0, s>>>(
              N, E, e0, e1, m->col_conn, m->col_rec, (const float*)up, (const float*)cot, P,
              grad);
        });
      }
      NSRHS_TRY(cudaGetLastError());
    }
    return NSRHS_OK;
  }
  const unsigned grid = grid_for(E, m->device, 16);
  if (p->precision == NSRHS_FP64) {
    auto P = elem_params<double>(p);
    with_flags(formulation_flags(p), [&](auto fl) {
      vjp_fp64_atomic_kernel<decltype(fl)::value><<<grid, kThreads, 0, s>>>(
          N, E, m->conn, m->geom, (const double*)up, (const double*)cot, P, grad);
    });
  } else {
    auto P = elem_params<float>(p);
    with_flags(formulation_flags(p), [&](auto fl) {
      vjp_mixed_atomic_kernel<decltype(fl)::value><<<grid, kThreads, 0, s>>>(
          N, E, m->conn, m->rec, (const float*)up, (const float*)cot, P, grad);
    });
  }
  return cuda_status(cudaGetLastError());
}

nsrhs_status nsrhs_assemble_rhs_vjp(const nsrhs_mesh* m, const nsrhs_params* p, const void* up,
                                    const void* cot, double* rhs, double* grad, void* stream) {
  if (!is_live(m) || !up || !cot || !rhs || !grad || rhs == grad) return NSRHS_EINVAL;
  nsrhs_status st = check_params(p);
  if (st != NSRHS_OK) return st;
  if (p->scatter == NSRHS_SCATTER_COLOUR) return NSRHS_EUNSUPPORTED;
  if (p->scatter == NSRHS_SCATTER_BLOCK_COLOUR && m->bcol_order == nullptr)
    return NSRHS_EUNSUPPORTED;
  if (p->geometry != NSRHS_GEOM_CACHED) return NSRHS_EUNSUPPORTED;
  // AUTO: atomics for the FP64 form, blocks for the mixed form (as for the
  // separate calls)
  const bool block = p->scatter == NSRHS_SCATTER_BLOCK ||
                     p->scatter == NSRHS_SCATTER_BLOCK_COLOUR ||
                     (p->scatter == NSRHS_SCATTER_AUTO && p->precision == NSRHS_MIXED);
  if (block && !block_smem_fits(m, p, 8, 2)) return NSRHS_EUNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard dg(m->device);
  if (!dg.ok) return NSRHS_ECUDA;
  const int64_t N = m->n_nodes, E = m->n_elems;
  NSRHS_TRY(cudaMemsetAsync(rhs, 0, sizeof(double) * 4 * N, s));
  NSRHS_TRY(cudaMemsetAsync(grad, 0, sizeof(double) * 4 * N, s));
  const int flags = formulation_flags(p);
  if (block) {
    const bool coloured = p->scatter == NSRHS_SCATTER_BLOCK_COLOUR;
    const int64_t nb = m->n_blocks;
    std::vector<int64_t> ranges = coloured ? m->bcol_off : std::vector<int64_t>{0, nb};
    cudaError_t err = cudaSuccess;
    for (size_t k = 0; k + 1 < ranges.size() && err == cudaSuccess; ++k) {
      const int64_t i0 = ranges[k], i1 = ranges[k + 1];
      const unsigned grid = (unsigned)std::max<int64_t>(
          1, std::min<int64_t>(i1 - i0, (int64_t)sm_count(m->device) * kBlockCtasPerSm));
      auto launch = [&](auto kern, size_t smem, const double* geom, const auto* u, const auto* c,
                        const auto& P) {
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err == cudaSuccess)
          kern<<<grid, nsrhs::kBlockElems, smem, s>>>(
              N, E, nb, m->blk_node_off, m->blk_nodes, m->blk_runs, m->blk_cap, m->rec, geom, u,
              c, P, rhs, grad, coloured ? m->bcol_order : nullptr, i0, i1);
      };
      if (p->precision == NSRHS_FP64) {
        auto P = elem_params<double>(p);
        const size_t smem = nsrhs::block_smem_bytes<double, 8>(m->blk_cap, 2);
        with_flags(flags, [&](auto fl) {
          constexpr int F = decltype(fl)::value;
          if (coloured)
            launch(nsrhs::rhs_vjp_block_kernel<double, F, true>, smem, m->geom, (const double*)up,
                   (const double*)cot, P);
          else
            launch(nsrhs::rhs_vjp_block_kernel<double, F, false>, smem, m->geom,
                   (const double*)up, (const double*)cot, P);
        });
      } else {
        auto P = elem_params<float>(p);
        const size_t smem = nsrhs::block_smem_bytes<float, 8>(m->blk_cap, 2);
        with_flags(flags, [&](auto fl) {
          constexpr int F = decltype(fl)::value;
          if (coloured)
            launch(nsrhs::rhs_vjp_block_kernel<float, F, true>, smem, nullptr, (const float*)up,
                   (const float*)cot, P);
          else
            launch(nsrhs::rhs_vjp_block_kernel<float, F, false>, smem, nullptr, (const float*)up,
                   (const float*)cot, P);
        });
      }
      if (err == cudaSuccess) err = cudaGetLastError();
    }
    return cuda_status(err);
  }
  const unsigned grid = grid_for(E, m->device, 16);
  if (p->precision == NSRHS_FP64) {
    auto P = elem_params<double>(p);
    with_flags(flags, [&](auto fl) {
      rhs_vjp_atomic_kernel<double, decltype(fl)::value, double><<<grid, kThreads, 0, s>>>(
          N, E, m->conn, m->geom, (const double*)up, (const double*)cot, P, rhs, grad);
    });
  } else {
    auto P = elem_params<float>(p);
    with_flags(flags, [&](auto fl) {
      rhs_vjp_atomic_kernel<float, decltype(fl)::value, nsrhs::RecChunk>
          <<<grid, kThreads, 0, s>>>(N, E, m->conn, m->rec, (const float*)up, (const float*)cot, P, rhs, grad);
    });
  }
  return cuda_status(cudaGetLastError());
}

nsrhs_status nsrhs_mesh_check_noalloc(int64_t n_nodes, int64_t n_elems, const double* coords,
                                      const int32_t* conn, double ar_threshold, void* stream,
                                      nsrhs_mesh_check_result* result_dev) {
  if (!coords || !conn || !result_dev) return NSRHS_EINVAL;
  if (n_nodes < 1 || n_elems < 1 || n_nodes > INT32_MAX || n_elems > INT32_MAX) return NSRHS_EINVAL;
  if (!(ar_threshold > 0.0)) return NSRHS_EINVAL;
  CheckPartial* scratch = nullptr;
  nsrhs_status st = check_scratch_address(&scratch);
  if (st != NSRHS_OK) return st;
  int dev = 0;
  cudaGetDevice(&dev);
  int64_t need = (n_elems + kCheckThreads - 1) / kCheckThreads;
  int64_t cap = std::min<int64_t>((int64_t)sm_count(dev) * 4, NSRHS_CHECK_SCRATCH_BLOCKS);
  int grid = (int)std::max<int64_t>(1, std::min(need, cap));
  cudaStream_t s = (cudaStream_t)stream;
  check_partials_kernel<<<grid, kCheckThreads, 0, s>>>(n_nodes, n_elems, coords, conn,
                                                       ar_threshold, scratch);
  NSRHS_TRY(cudaGetLastError());
  check_reduce_kernel<<<1, kCheckThreads, 0, s>>>(grid, scratch, result_dev);
  return cuda_status(cudaGetLastError());
}

nsrhs_status nsrhs_assemble_elmat(const nsrhs_mesh* m, const nsrhs_params* p, const double* up,
                                  double* rhs, void* stream) {
  if (!is_live(m) || !up || !rhs) return NSRHS_EINVAL;
  nsrhs_status st = check_params(p);
  if (st != NSRHS_OK) return st;
  if (p->precision != NSRHS_FP64 || p->convection != NSRHS_CONVECTIVE ||
      p->tau_mode != NSRHS_TAU_GAUSS || p->geometry != NSRHS_GEOM_CACHED)
    return NSRHS_EUNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard dg(m->device);
  if (!dg.ok) return NSRHS_ECUDA;
  const int64_t N = m->n_nodes, E = m->n_elems;
  NSRHS_TRY(cudaMemsetAsync(rhs, 0, sizeof(double) * 4 * N, s));
  auto P = elem_params<double>(p);
  const unsigned grid = grid_for(E, m->device, 16);
  if (p->c_vreman != 0.0)
    fwd_fp64_elmat_kernel<true><<<grid, kThreads, 0, s>>>(N, E, m->conn, m->geom, up, P, rhs);
  else
    fwd_fp64_elmat_kernel<false><<<grid, kThreads, 0, s>>>(N, E, m->conn, m->geom, up, P, rhs);
  return cuda_status(cudaGetLastError());
}

nsrhs_status nsrhs_mesh_element_colours(const nsrhs_mesh* m, int32_t which, int32_t* out_dev,
                                        void* stream) {
  if (!is_live(m) || !out_dev) return NSRHS_EINVAL;
  if (which < NSRHS_ELEMENT_COLOUR || which > NSRHS_ELEMENT_BLOCK) return NSRHS_EINVAL;
  if (m->colour == nullptr || m->bcolour == nullptr) return NSRHS_EUNSUPPORTED;
  DeviceGuard dg(m->device);
  if (!dg.ok) return NSRHS_ECUDA;
  const int64_t E = m->n_elems;
  nsrhs::colour_export_kernel<<<grid_for(E, m->device, 8), kThreads, 0, (cudaStream_t)stream>>>(
      E, which, nsrhs::kBlockElems, m->elem_order, m->colour, m->bcolour, out_dev);
  return cuda_status(cudaGetLastError());
}

nsrhs_status nsrhs_lumped_mass(const nsrhs_mesh* m, double* mass_dev, void* stream) {
  if (!is_live(m) || !mass_dev) return NSRHS_EINVAL;
  DeviceGuard dg(m->device);
  if (!dg.ok) return NSRHS_ECUDA;
  return cuda_status(cudaMemcpyAsync(mass_dev, m->mass, sizeof(double) * m->n_nodes,
                                     cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
}

nsrhs_status nsrhs_explicit_step(const nsrhs_mesh* m, const nsrhs_params* p, double dt,
                                 int32_t scheme, double* up_dev, double* work_dev, void* stream) {
  if (!is_live(m) || !up_dev || !work_dev) return NSRHS_EINVAL;
  nsrhs_status st = check_params(p);
  if (st != NSRHS_OK) return st;
  if (!(dt > 0.0) || !std::isfinite(dt) || !(p->rho > 0.0)) return NSRHS_EINVAL;
  if (scheme != NSRHS_EULER && scheme != NSRHS_SSPRK3) return NSRHS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard dg(m->device);
  if (!dg.ok) return NSRHS_ECUDA;
  const int64_t N = m->n_nodes;
  double* F = work_dev;              // [4][N] stage RHS
  double* stage = work_dev + 4 * N;  // [4][N] stage state
  float* narrow = reinterpret_cast<float*>(work_dev + 8 * N);  // MIXED: [4][N] float state
  const double dtr = dt / p->rho;
  const unsigned grid = grid_for(N, m->device, 8);
  // the stage RHS: FP64 from the double state; MIXED from its float copy
  // (float element arithmetic, double accumulation), the update in double
  auto rhs_of = [&](const double* u) {
    if (p->precision == NSRHS_FP64) return nsrhs_assemble(m, p, u, F, stream);
    narrow_kernel<<<grid_for(4 * N, m->device, 8), kThreads, 0, s>>>(4 * N, u, narrow);
    nsrhs_status st2 = cuda_status(cudaGetLastError());
    if (st2 != NSRHS_OK) return st2;
    return nsrhs_assemble(m, p, narrow, F, stream);
  };
  if (scheme == NSRHS_EULER) {
    if ((st = rhs_of(up_dev)) != NSRHS_OK) return st;
    rk_combine_kernel<<<grid, kThreads, 0, s>>>(N, 0.0, 1.0, dtr, up_dev, up_dev, F, m->inv_mass,
                                                up_dev);
    return cuda_status(cudaGetLastError());
  }
  // stage 1: stage = u + dt L(u)
  if ((st = rhs_of(up_dev)) != NSRHS_OK) return st;
  rk_combine_kernel<<<grid, kThreads, 0, s>>>(N, 0.0, 1.0, dtr, up_dev, up_dev, F, m->inv_mass,
                                              stage);
  NSRHS_TRY(cudaGetLastError());
  // stage 2: stage = 3/4 u + 1/4 (stage + dt L(stage))
  if ((st = rhs_of(stage)) != NSRHS_OK) return st;
  rk_combine_kernel<<<grid, kThreads, 0, s>>>(N, 0.75, 0.25, dtr, up_dev, stage, F, m->inv_mass,
                                              stage);
  NSRHS_TRY(cudaGetLastError());
  // stage 3: u = 1/3 u + 2/3 (stage + dt L(stage))
  if ((st = rhs_of(stage)) != NSRHS_OK) return st;
  rk_combine_kernel<<<grid, kThreads, 0, s>>>(N, 1.0 / 3.0, 2.0 / 3.0, dtr, up_dev, stage, F,
                                              m->inv_mass, up_dev);
  return cuda_status(cudaGetLastError());
}

void nsrhs_destroy(nsrhs_mesh* m) {
  if (!m) return;
  {
    std::lock_guard<std::mutex> lock(g_registry_mutex);
    if (g_registry.erase(m) == 0) return;  // not a live mesh: ignore
  }
  free_mesh(m);
}

}  // extern "C"
