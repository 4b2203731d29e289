// Element blocks for shared-memory staged gathers and scatters.
//
// Setup (once per mesh): elements are put in Morton order of their centroids,
// so that consecutive elements are close in space, and cut into blocks of
// kBlockElems elements. For every block the sorted list of the distinct nodes
// it touches is stored, and a run table: per distinct node, the run of its
// contributions in the block's contributions sorted by node, ranked longest
// run first; per element and local node, the node's index in the block's list
// and the position of its contribution in that sorted order (the block map,
// in the element's record).
//
// Assembly (per call): each CTA walks its blocks; the nodal values of a
// block's distinct nodes come into shared memory once (as cp.async copies
// issued three blocks ahead, through a 4-stage pipeline), each thread
// computes one element from shared memory and writes its 16 entries to
// shared memory at their sorted positions, and each distinct node's entries
// (a contiguous run) are summed in a fixed order and added to the global RHS
// with one atomic per component (for coloured blocks, launched colour by
// colour, these never meet at one address, so their order is fixed). The
// global atomics drop from 16 per element to 4 per (block, distinct node),
// and the sums inside a block do not depend on scheduling.
#pragma once

#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "element.cuh"

namespace nsrhs {

#ifndef NSRHS_BLOCK_ELEMS
#define NSRHS_BLOCK_ELEMS 256
#endif
#ifndef NSRHS_BLOCK_MIN_CTAS_F32
#define NSRHS_BLOCK_MIN_CTAS_F32 4
#endif
constexpr int kBlockElems = NSRHS_BLOCK_ELEMS;  // elements per block = threads per CTA
constexpr int kBlockSlots = 4 * kBlockElems;     // at most this many distinct nodes

// Per-element record of the block kernels and the mixed form, 64 bytes in
// four 16-byte chunks: chunks 0-2 the element geometry rounded to float
// (cofactor vectors c_k at words 3k + d, 1/detJ at word 9, detJ^(-1/3) at
// word 10, word 11 unused; computed in double once per mesh), chunk 3 the
// block map: per local node a, (index of the node among the block's distinct
// nodes << 16) | position of the element's contribution to it in the block's
// node-sorted order. Records are stored chunk-major within each block of
// kBlockElems elements, so that the threads of a warp, one element each, read
// chunk k of consecutive elements as one contiguous 512-byte access:
// element e's chunk k is RecChunk number rec_index(e, k).
struct __align__(16) RecChunk {
  uint32_t w[4];
};
__host__ __device__ __forceinline__ int64_t rec_index(int64_t e, int k) {
  return ((e / kBlockElems) * 4 + k) * kBlockElems + (e % kBlockElems);
}
// RecChunks to allocate for n elements (whole blocks)
inline int64_t rec_chunks(int64_t n) { return (n + kBlockElems - 1) / kBlockElems * 4 * kBlockElems; }

// Loads of one record: the float geometry (three 16-byte loads) and the
// block map (one).
__device__ __forceinline__ void load_rec_geometry(const RecChunk* __restrict__ rec, int64_t e,
                                                  float c[3][3], float& inv_det, float& rh) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(rec + rec_index(e, 0)));
  const float4 b = __ldg(reinterpret_cast<const float4*>(rec + rec_index(e, 1)));
  const float4 d = __ldg(reinterpret_cast<const float4*>(rec + rec_index(e, 2)));
  c[0][0] = a.x; c[0][1] = a.y; c[0][2] = a.z;
  c[1][0] = a.w; c[1][1] = b.x; c[1][2] = b.y;
  c[2][0] = b.z; c[2][1] = b.w; c[2][2] = d.x;
  inv_det = d.y;
  rh = d.z;
}
__device__ __forceinline__ uint4 load_rec_lmap(const RecChunk* __restrict__ rec, int64_t e) {
  return __ldg(reinterpret_cast<const uint4*>(rec + rec_index(e, 3)));
}

// ---- setup ----

// Order-preserving map of doubles to unsigned 64-bit integers.
__device__ __forceinline__ unsigned long long ordered_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__host__ __device__ __forceinline__ double from_ordered_bits(unsigned long long o) {
  const unsigned long long b = (o & 0x8000000000000000ull) ? (o & 0x7fffffffffffffffull) : ~o;
  double d;
  memcpy(&d, &b, sizeof(d));
  return d;
}

// box[0..2] = ordered min of x,y,z; box[3..5] = ordered max. Initialise box to
// (~0, ~0, ~0, 0, 0, 0).
__global__ void bbox_kernel(int64_t N, const double* __restrict__ coords,
                            unsigned long long* __restrict__ box) {
  unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const unsigned long long o = ordered_bits(coords[d * N + i]);
      lo[d] = o < lo[d] ? o : lo[d];
      hi[d] = o > hi[d] ? o : hi[d];
    }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    atomicMin(box + d, lo[d]);
    atomicMax(box + 3 + d, hi[d]);
  }
}

__device__ __forceinline__ unsigned long long spread3(unsigned long long v) {
  // 21 bits -> every third bit of 63
  v &= 0x1fffffull;
  v = (v | (v << 32)) & 0x1f00000000ffffull;
  v = (v | (v << 16)) & 0x1f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}

// key[e] = Morton code of the element centroid in the bounding box, id[e] = e.
__global__ void morton_kernel(int64_t N, int64_t E, const double* __restrict__ coords,
                              const int32_t* __restrict__ conn, double x0, double y0, double z0,
                              double sx, double sy, double sz,
                              unsigned long long* __restrict__ key, int32_t* __restrict__ id) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    double cx = 0.0, cy = 0.0, cz = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int64_t v = conn[a * E + e];
      cx += coords[v];
      cy += coords[N + v];
      cz += coords[2 * N + v];
    }
    const double q = 2097151.0;  // 2^21 - 1
    const unsigned long long ix = (unsigned long long)fmin(fmax((0.25 * cx - x0) * sx, 0.0), q);
    const unsigned long long iy = (unsigned long long)fmin(fmax((0.25 * cy - y0) * sy, 0.0), q);
    const unsigned long long iz = (unsigned long long)fmin(fmax((0.25 * cz - z0) * sz, 0.0), q);
    key[e] = spread3(ix) | (spread3(iy) << 1) | (spread3(iz) << 2);
    id[e] = (int32_t)e;
  }
}

// out[a][i] = in[a][perm[i]]
__global__ void permute_conn_kernel(int64_t E, const int32_t* __restrict__ in,
                                    const int32_t* __restrict__ perm, int32_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = perm[i];
#pragma unroll
    for (int a = 0; a < 4; ++a) out[a * E + i] = in[a * E + e];
  }
}

// Per block: sort its (node << 16 | slot) keys (slot = 4 * element-in-block
// + local node), find the distinct nodes.
// pass 0 writes counts[b] = number of distinct nodes;
// pass 1 (node_off = exclusive sum of counts) writes
//   nodes[node_off[b] + u]        the u-th distinct node in ascending order (the
//                                 staging order: neighbouring lanes gather
//                                 neighbouring ids)
//   runs[node_off[b] + r]         the run of the node of rank r, the nodes
//                                 ranked by the length of their run of
//                                 contributions, longest first (ties by node),
//                                 so that the per-node phase hands each warp
//                                 runs of similar length:
//                                 (first sorted position << 21) | (length << 10) | u
//   block map of (element e, local node a)   (u << 16) | its sorted position
__global__ void __launch_bounds__(kBlockElems)
    block_plan_kernel(int pass, int64_t E, const int32_t* __restrict__ conn,
                      int64_t* __restrict__ counts, const int64_t* __restrict__ node_off,
                      int32_t* __restrict__ nodes, uint32_t* __restrict__ runs,
                      RecChunk* __restrict__ rec) {
  __shared__ unsigned long long key[kBlockSlots];
  __shared__ int part[kBlockElems];
  __shared__ uint16_t start[kBlockSlots + 1];  // first sorted position of distinct node u
  __shared__ uint32_t order[kBlockSlots];      // (kBlockSlots - run length) << 16 | u
  const int tid = threadIdx.x;
  const int64_t b = blockIdx.x;
  const int64_t e0 = b * kBlockElems;
  for (int i = tid; i < kBlockSlots; i += kBlockElems) {
    const int64_t e = e0 + (i >> 2);
    key[i] = e < E ? (((unsigned long long)(uint32_t)conn[(int64_t)(i & 3) * E + e] << 16) |
                      (unsigned long long)i)
                   : ~0ull;
  }
  __syncthreads();
  // bitonic sort, ascending
  for (int k = 2; k <= kBlockSlots; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < kBlockSlots; i += kBlockElems) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long a = key[i], c = key[ixj];
          const bool up = (i & k) == 0;
          if ((a > c) == up) {
            key[i] = c;
            key[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  // distinct-node flags: thread tid owns sorted positions 4 tid .. 4 tid + 3
  int flag[4], local = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = 4 * tid + r;
    const unsigned long long kk = key[i];
    const bool valid = kk != ~0ull;
    flag[r] = valid && (i == 0 || (key[i - 1] >> 16) != (kk >> 16));
    local += flag[r];
  }
  part[tid] = local;
  __syncthreads();
  // inclusive scan of part[] (Hillis-Steele)
  for (int off = 1; off < kBlockElems; off <<= 1) {
    const int v = tid >= off ? part[tid - off] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  const int n_distinct = part[kBlockElems - 1];
  if (pass == 0) {
    if (tid == 0) counts[b] = n_distinct;
    return;
  }
  const int64_t off = node_off[b];
  // distinct index u in ascending node order, and each node's first position
  int u = part[tid] - local - 1;  // distinct index before this thread's first position
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = 4 * tid + r;
    if (key[i] == ~0ull) continue;
    u += flag[r];
    if (flag[r]) start[u] = (uint16_t)i;
  }
  if (tid == 0) {
    // the number of valid positions = elements in the block * 4
    const int64_t ne = (E - e0) < kBlockElems ? (E - e0) : kBlockElems;
    start[n_distinct] = (uint16_t)(4 * ne);
  }
  __syncthreads();
  for (int v = tid; v < kBlockSlots; v += kBlockElems)
    order[v] = v < n_distinct
                   ? ((uint32_t)(kBlockSlots - (start[v + 1] - start[v])) << 16) | (uint32_t)v
                   : 0xffffffffu;
  __syncthreads();
  // bitonic sort of order[], ascending: longest runs first
  for (int k = 2; k <= kBlockSlots; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < kBlockSlots; i += kBlockElems) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const uint32_t a = order[i], c = order[ixj];
          const bool up = (i & k) == 0;
          if ((a > c) == up) {
            order[i] = c;
            order[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  for (int r = tid; r < n_distinct; r += kBlockElems) {
    const int v = (int)(order[r] & 0xffffu);
    const int s0 = start[v], len = start[v + 1] - s0;
    nodes[off + v] = (int32_t)(key[s0] >> 16);
    runs[off + r] = ((uint32_t)s0 << 21) | ((uint32_t)len << 10) | (uint32_t)v;
  }
  u = part[tid] - local - 1;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = 4 * tid + r;
    const unsigned long long kk = key[i];
    if (kk == ~0ull) continue;
    u += flag[r];
    const int slot = (int)(kk & 0xffffull);
    rec[rec_index(e0 + (slot >> 2), 3)].w[slot & 3] = ((uint32_t)u << 16) | (uint32_t)i;
  }
}


// ---- assembly ----

// Sum of a node's contributions. double: plain double sum. float: compensated
// float sum (Knuth's TwoSum keeps the rounding error of every addition), which
// carries about 48 bits, widened and added in double at the end; this keeps
// the mixed form's accumulation double-accurate without FP64 instructions per
// contribution.
template <class R>
struct NodeSum;
template <>
struct NodeSum<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};

// Two floats in one 64-bit register (low word first), added or subtracted
// lane by lane in one instruction (the two-wide FP32 operations of sm_100
// and later).
__device__ __forceinline__ unsigned long long f32x2_add(unsigned long long a,
                                                        unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long f32x2_sub(unsigned long long a,
                                                        unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ float f32x2_lo(unsigned long long x) { return __uint_as_float((unsigned)x); }
__device__ __forceinline__ float f32x2_hi(unsigned long long x) {
  return __uint_as_float((unsigned)(x >> 32));
}

// The compensated float sum (TwoSum per addition) on two components at once.
struct NodeSumF32x2 {
  unsigned long long s = 0ull, c = 0ull;
  __device__ __forceinline__ void add(unsigned long long x) {
    const unsigned long long t = f32x2_add(s, x);
    const unsigned long long bp = f32x2_sub(t, s);
    c = f32x2_add(c, f32x2_add(f32x2_sub(s, f32x2_sub(t, bp)), f32x2_sub(x, bp)));
    s = t;
  }
  // the sum s + c in double: both widened exactly with integer operations,
  // one double addition (the FP64 pipe is 1/64 of the FP32 rate)
  __device__ __forceinline__ double lo() const {
    return widen_f32(f32x2_lo(s)) + widen_f32(f32x2_lo(c));
  }
  __device__ __forceinline__ double hi() const {
    return widen_f32(f32x2_hi(s)) + widen_f32(f32x2_hi(c));
  }
};

// Shared-memory layouts. Staged nodal values: one 4-component record per
// distinct node (u, v, w, p; the adjoint adds the cotangent's 4), so that an
// element reads each of its nodes with 128-bit loads. Element entries: one
// 4-component record per sorted position.
template <class R>
struct Smem;
template <>
struct Smem<float> {
  // the 4 values of node slot lc from a [slot][stride] float buffer
  static __device__ __forceinline__ void get4(const float* buf, int stride, int lc, float v[4]) {
    const float4 q = *reinterpret_cast<const float4*>(buf + stride * lc);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
  static __device__ __forceinline__ void put4(float* buf, int pos, const float f[4]) {
    *reinterpret_cast<float4*>(buf + 4 * pos) = make_float4(f[0], f[1], f[2], f[3]);
  }
  // sums of components 2h and 2h + 1 over the positions [r0, r1), in order
  static __device__ __forceinline__ void sum_pair(const float* buf, int h, int r0, int r1,
                                                  double& lo, double& hi) {
    const unsigned long long* e = reinterpret_cast<const unsigned long long*>(buf) + h;
    NodeSumF32x2 acc;
    // the next two entries are loaded ahead of the one being added
    unsigned long long x = r0 < r1 ? e[2 * r0] : 0ull;
    unsigned long long y = r0 + 1 < r1 ? e[2 * r0 + 2] : 0ull;
    for (int q = r0; q < r1; ++q) {
      const unsigned long long next = q + 2 < r1 ? e[2 * (q + 2)] : 0ull;
      acc.add(x);
      x = y;
      y = next;
    }
    lo = acc.lo();
    hi = acc.hi();
  }
};
template <>
struct Smem<double> {
  static __device__ __forceinline__ void get4(const double* buf, int stride, int lc, double v[4]) {
    const double2* q = reinterpret_cast<const double2*>(buf + stride * lc);
    const double2 a = q[0], b = q[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
  static __device__ __forceinline__ void put4(double* buf, int pos, const double f[4]) {
    double2* q = reinterpret_cast<double2*>(buf + 4 * pos);
    q[0] = make_double2(f[0], f[1]);
    q[1] = make_double2(f[2], f[3]);
  }
  static __device__ __forceinline__ void sum_pair(const double* buf, int h, int r0, int r1,
                                                  double& lo, double& hi) {
    const double2* e = reinterpret_cast<const double2*>(buf) + h;
    NodeSum<double> a, b;
    for (int q = r0; q < r1; ++q) {
      const double2 x = e[2 * q];
      a.add(x.x);
      b.add(x.y);
    }
    lo = a.value();
    hi = b.value();
  }
};

// Geometry of element e for the block kernels: float from the element record
// (mixed form), double from the cached [11][E] rows (FP64 form).
__device__ __forceinline__ void block_geometry(const RecChunk* __restrict__ rec,
                                               const double* __restrict__, int64_t, int64_t e,
                                               float c[3][3], float& inv_det, float& rh) {
  load_rec_geometry(rec, e, c, inv_det, rh);
}
__device__ __forceinline__ void block_geometry(const RecChunk* __restrict__,
                                               const double* __restrict__ geom, int64_t E,
                                               int64_t e, double c[3][3], double& inv_det,
                                               double& rh) {
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int d = 0; d < 3; ++d) c[k][d] = __ldg(geom + (3 * k + d) * E + e);
  inv_det = __ldg(geom + 9 * E + e);
  rh = __ldg(geom + 10 * E + e);
}

// A thread's element record for the block kernels, loaded one block ahead
// (issued before the per-node phase of the current block, so that its
// latency is hidden behind that phase and the barrier). AHEAD = 2: the whole
// float record (geometry and block map); AHEAD = 1: the block map only, the
// geometry read when the element is computed (measured: the mixed forward,
// whose element routine re-reads u from shared memory, is faster with 2; the
// mixed adjoint, capped at 80 registers, with 1). For R = double the FP64
// geometry always comes from the cached double rows.
template <class R, int AHEAD>
struct RecAhead;
template <>
struct RecAhead<float, 2> {
  float4 q0, q1, q2;
  uint4 lm;
  __device__ __forceinline__ void load(const RecChunk* __restrict__ rec, int64_t e) {
    q0 = __ldg(reinterpret_cast<const float4*>(rec + rec_index(e, 0)));
    q1 = __ldg(reinterpret_cast<const float4*>(rec + rec_index(e, 1)));
    q2 = __ldg(reinterpret_cast<const float4*>(rec + rec_index(e, 2)));
    lm = load_rec_lmap(rec, e);
  }
  __device__ __forceinline__ void geometry(const RecChunk* __restrict__, const double* __restrict__,
                                           int64_t, int64_t, float c[3][3], float& inv_det,
                                           float& rh) const {
    c[0][0] = q0.x; c[0][1] = q0.y; c[0][2] = q0.z;
    c[1][0] = q0.w; c[1][1] = q1.x; c[1][2] = q1.y;
    c[2][0] = q1.z; c[2][1] = q1.w; c[2][2] = q2.x;
    inv_det = q2.y;
    rh = q2.z;
  }
};
template <>
struct RecAhead<float, 1> {
  uint4 lm;
  __device__ __forceinline__ void load(const RecChunk* __restrict__ rec, int64_t e) {
    lm = load_rec_lmap(rec, e);
  }
  __device__ __forceinline__ void geometry(const RecChunk* __restrict__ rec,
                                           const double* __restrict__, int64_t, int64_t e,
                                           float c[3][3], float& inv_det, float& rh) const {
    load_rec_geometry(rec, e, c, inv_det, rh);
  }
};
template <int AHEAD>
struct RecAhead<double, AHEAD> {
  uint4 lm;
  __device__ __forceinline__ void load(const RecChunk* __restrict__ rec, int64_t e) {
    lm = load_rec_lmap(rec, e);
  }
  __device__ __forceinline__ void geometry(const RecChunk* __restrict__,
                                           const double* __restrict__ geom, int64_t E, int64_t e,
                                           double c[3][3], double& inv_det, double& rh) const {
    block_geometry(nullptr, geom, E, e, c, inv_det, rh);
  }
};

// The per-node phase of a block: each distinct node's entries (a contiguous
// run of sorted positions) summed in a fixed order and added to out [4][N]
// with one atomic per component. Work item i = (node of rank i / 2,
// component pair i % 2): two threads per node, so that twice as many threads
// share the runs and each sums one 64-bit pair; nodes come longest run
// first, so the lanes of a warp loop about equally long. The block's node
// ids (in staging order) and runs (in rank order, each naming its node's
// staging index) come from its pipeline stage (shared memory).
template <class R>
__device__ __forceinline__ void block_node_sums(int64_t N, int nb, const int32_t* ids,
                                                const uint32_t* rl, const R* buf,
                                                double* __restrict__ out) {
  for (int i = threadIdx.x; i < 2 * nb; i += kBlockElems) {
    const int j = i >> 1, h = i & 1;
    const uint32_t r = rl[j];
    const int r0 = (int)(r >> 21), r1 = r0 + (int)((r >> 10) & 0x7ffu);
    const int64_t v = ids[r & 0x3ffu];
    double lo, hi;
    Smem<R>::sum_pair(buf, h, r0, r1, lo, hi);
    atomicAdd(out + (2 * h) * N + v, lo);
    atomicAdd(out + (2 * h + 1) * N + v, hi);
  }
}

// The one-pass kernel's per-node sums: as block_node_sums for two entry
// buffers (the element RHS and its gradient) at once, so that each thread
// reads its node's run once and carries two independent summation chains.
template <class R>
__device__ __forceinline__ void block_node_sums2(int64_t N, int nb, const int32_t* ids,
                                                 const uint32_t* rl, const R* bufA,
                                                 double* __restrict__ outA, const R* bufB,
                                                 double* __restrict__ outB) {
  for (int i = threadIdx.x; i < 2 * nb; i += kBlockElems) {
    const int j = i >> 1, h = i & 1;
    const uint32_t r = rl[j];
    const int r0 = (int)(r >> 21), r1 = r0 + (int)((r >> 10) & 0x7ffu);
    const int64_t v = ids[r & 0x3ffu];
    double lo, hi, lo2, hi2;
    Smem<R>::sum_pair(bufA, h, r0, r1, lo, hi);
    Smem<R>::sum_pair(bufB, h, r0, r1, lo2, hi2);
    atomicAdd(outA + (2 * h) * N + v, lo);
    atomicAdd(outA + (2 * h + 1) * N + v, hi);
    atomicAdd(outB + (2 * h) * N + v, lo2);
    atomicAdd(outB + (2 * h + 1) * N + v, hi2);
  }
}

// The gather pipeline of the block kernels: kStages shared-memory stages per
// CTA, the copies of a block issued kStages - 1 blocks before it is computed
// (one block of lead left the staged gathers' latency exposed once the
// element arithmetic was cheap). A stage holds, for at most `cap` distinct
// nodes (the mesh's largest block, rounded up to a multiple of 32), the
// nodal records [cap][W] (W = 4: u, v, w, p; W = 8: and the cotangent), then
// the node ids [cap] and the runs [cap] of the block. After the stages, the
// element entries [kBlockSlots][4] by sorted position.
#ifndef NSRHS_BLOCK_STAGES
#define NSRHS_BLOCK_STAGES 4
#endif
constexpr int kStages = NSRHS_BLOCK_STAGES;

template <class R, int W>
__host__ __device__ constexpr size_t stage_bytes(int cap) {
  return (size_t)cap * (W * sizeof(R) + 2 * sizeof(uint32_t));
}
template <class R, int W>
__host__ __device__ constexpr size_t block_smem_bytes(int cap, int entry_buffers = 1) {
  return kStages * stage_bytes<R, W>(cap) + (size_t)entry_buffers * kBlockSlots * 4 * sizeof(R);
}

// Resident CTAs per SM the compiler must allow (register cap): the float
// kernels are latency-bound between their barrier-separated phases, so more
// CTAs per SM help; the double kernels are bound by the FP64 pipe.
template <class R>
constexpr int block_kernel_min_ctas() {
  return sizeof(R) == 4 ? NSRHS_BLOCK_MIN_CTAS_F32 : 2;
}
template <class R>
constexpr int block_vjp_min_ctas() {
  return sizeof(R) == 4 ? 3 : 1;
}

// Asynchronous global-to-shared copies (cp.async).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}

// Issues the copies of block b into one pipeline stage: its node ids (stored
// from the registers that address the gathers), runs, and nodal records
// (and, for W = 8, the cotangent at columns 4..7).
template <class R, int W>
__device__ __forceinline__ void stage_block(int64_t N, int64_t b,
                                            const int64_t* __restrict__ node_off,
                                            const int32_t* __restrict__ nodes,
                                            const uint32_t* __restrict__ runs,
                                            const R* __restrict__ up, const R* __restrict__ cot,
                                            unsigned char* stage, int cap) {
  const int64_t off = __ldg(node_off + b);
  const int nb = (int)(__ldg(node_off + b + 1) - off);
  R* vals = reinterpret_cast<R*>(stage);
  int32_t* ids = reinterpret_cast<int32_t*>(stage + (size_t)cap * W * sizeof(R));
  uint32_t* rl = reinterpret_cast<uint32_t*>(ids + cap);
  for (int j = threadIdx.x; j < nb; j += kBlockElems) {
    const int32_t v = __ldg(nodes + off + j);
    ids[j] = v;
    cp_async<4>(rl + j, runs + off + j);
    R* slot = vals + W * j;
#pragma unroll
    for (int k = 0; k < 4; ++k) cp_async<sizeof(R)>(slot + k, up + k * N + v);
    if constexpr (W == 8) {
#pragma unroll
      for (int k = 0; k < 4; ++k) cp_async<sizeof(R)>(slot + 4 + k, cot + k * N + v);
    }
  }
}

// The float element routines re-read an element's nodal velocities (and
// cotangent) from the staged [slot][W] records at their phase boundaries
// (the empty asm with a memory clobber keeps the compiler from reusing the
// first loads), so they are not held in registers across the routine: the
// mixed forward then takes the whole element record one block ahead within
// its 64 registers, and the mixed adjoint fits 3 CTAs per SM (80 registers)
// instead of 2 (128).
template <class R, int W>
struct StagedReload {
  const R* vals;
  const uint32_t* lmv;
  __device__ __forceinline__ void u(R (&uu)[4][3]) const {
    asm volatile("" ::: "memory");
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      R q[4];
      Smem<R>::get4(vals, W, (int)(lmv[a] >> 16), q);
      uu[a][0] = q[0];
      uu[a][1] = q[1];
      uu[a][2] = q[2];
    }
  }
  __device__ __forceinline__ void w(R (&ww)[4][4]) const {
    asm volatile("" ::: "memory");
#pragma unroll
    for (int a = 0; a < 4; ++a) Smem<R>::get4(vals + 4, W, (int)(lmv[a] >> 16), ww[a]);
  }
};

// Forward assembly with block-staged gathers and scatters; R is the element
// arithmetic type (float: mixed form, double: FP64 form). Dynamic shared
// memory: block_smem_bytes<R, 4>(cap) bytes.
//
// Per block: the block's stage has landed (wait + barrier); the copies of
// the block kStages - 1 ahead are issued into the stage the previous block
// used; each thread computes its element from the staged nodal records and
// writes its 16 entries at their sorted positions; barrier; the per-node
// sums and atomics.
//
// COLOUR: the CTAs process the blocks order[i0 .. i1) of one block colour (no
// two share a node, so every address receives at most one atomic in the
// launch and the colour order fixes the summation order: deterministic);
// otherwise blocks 0 .. n_blocks - 1.
template <class R, int FLAGS, bool COLOUR = false>
__global__ void __launch_bounds__(kBlockElems, block_kernel_min_ctas<R>())
    fwd_block_kernel(int64_t N, int64_t E, int64_t n_blocks, const int64_t* __restrict__ node_off,
                     const int32_t* __restrict__ nodes, const uint32_t* __restrict__ runs,
                     int cap, const RecChunk* __restrict__ rec, const double* __restrict__ geom64,
                     const R* __restrict__ up, ElemParams<R> P, double* __restrict__ rhs,
                     const int32_t* __restrict__ order = nullptr, int64_t i0 = 0,
                     int64_t i1 = 0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const size_t sbytes = stage_bytes<R, 4>(cap);
  R* sF = reinterpret_cast<R*>(smem_raw + kStages * sbytes);  // [kBlockSlots][4] entries
  const int tid = threadIdx.x;
  const int64_t first = COLOUR ? i0 : 0, last = COLOUR ? i1 : n_blocks;
  auto block_at = [&](int64_t i) -> int64_t { return COLOUR ? (int64_t)__ldg(order + i) : i; };
  int64_t i = first + blockIdx.x;
#pragma unroll 1
  for (int k = 0; k < kStages - 1; ++k) {
    const int64_t ik = i + (int64_t)k * gridDim.x;
    if (ik < last)
      stage_block<R, 4>(N, block_at(ik), node_off, nodes, runs, up, nullptr,
                        smem_raw + k * sbytes, cap);
    cp_async_commit();
  }
  RecAhead<R, 2> ra;
  if (i < last && block_at(i) * kBlockElems + tid < E) ra.load(rec, block_at(i) * kBlockElems + tid);
  for (int step = 0; i < last; i += gridDim.x, ++step) {
    const int64_t b = block_at(i);
    const int64_t bn = i + gridDim.x < last ? block_at(i + gridDim.x) : -1;
    unsigned char* st = smem_raw + (step % kStages) * sbytes;
    cp_async_wait<kStages - 2>();  // this block's copies (the oldest pending group) have landed
    __syncthreads();               // ... for every thread; the previous block's sums are done
    {
      const int64_t ia = i + (int64_t)(kStages - 1) * gridDim.x;
      if (ia < last)
        stage_block<R, 4>(N, block_at(ia), node_off, nodes, runs, up, nullptr,
                          smem_raw + ((step + kStages - 1) % kStages) * sbytes, cap);
      cp_async_commit();
    }
    const int64_t e = b * kBlockElems + tid;
    if (e < E) {
      const RecAhead<R, 2> cur = ra;
      const uint32_t lmv[4] = {cur.lm.x, cur.lm.y, cur.lm.z, cur.lm.w};
      const R* vals = reinterpret_cast<const R*>(st);
      R u[4][3], p[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        R q[4];
        Smem<R>::get4(vals, 4, (int)(lmv[a] >> 16), q);
        u[a][0] = q[0];
        u[a][1] = q[1];
        u[a][2] = q[2];
        p[a] = q[3];
      }
      R c[3][3], inv_det, rh;
      cur.geometry(rec, geom64, E, e, c, inv_det, rh);
      R F[4][4];
      if constexpr (sizeof(R) == 4)
        element_rhs<R, FLAGS>(c, inv_det, rh, u, p, P, F, StagedReload<R, 4>{vals, lmv});
      else
        element_rhs<R, FLAGS>(c, inv_det, rh, u, p, P, F);
#pragma unroll
      for (int a = 0; a < 4; ++a) Smem<R>::put4(sF, (int)(lmv[a] & 0xffffu), F[a]);
    }
    if (bn >= 0 && bn * kBlockElems + tid < E) ra.load(rec, bn * kBlockElems + tid);
    const int nb = (int)(__ldg(node_off + b + 1) - __ldg(node_off + b));
    __syncthreads();
    const int32_t* ids = reinterpret_cast<const int32_t*>(st + (size_t)cap * 4 * sizeof(R));
    block_node_sums<R>(N, nb, ids, reinterpret_cast<const uint32_t*>(ids + cap), sF, rhs);
  }
  cp_async_wait<0>();
}

// The one-pass kernel's element policy: Base's re-reads, and the element
// RHS stored at its sorted positions in the RHS entry buffer as soon as the
// routine has it, before the reverse part.
template <class R, class Base>
struct PutRhs : Base {
  R* sFr;
  const uint32_t* lm;
  __device__ __forceinline__ void f(const R (*F)[4]) const {
#pragma unroll
    for (int a = 0; a < 4; ++a) Smem<R>::put4(sFr, (int)(lm[a] & 0xffffu), F[a]);
  }
};

// Adjoint with block-staged gathers and scatters: the reverse of the forward
// block kernel. Per block the nodal (u, p) and the cotangent of its distinct
// nodes come through the same pipeline (W = 8), each thread runs one
// element's reverse sweep, the 16 gradient entries go to shared memory at
// their sorted positions, and each node's entries are summed in a fixed
// order and added with one atomic per component (COLOUR: blocks of one
// colour per launch, so that the summation order is fixed).
//
// WITH_F: the one-pass form; the element routine also yields the element
// RHS, which goes to a second entry buffer and is summed per node into rhs
// by the same runs (block_node_sums2). Dynamic shared memory: block_smem_bytes<R, 8>(cap, 1 +
// WITH_F) bytes.
template <class R, int FLAGS, bool COLOUR, bool WITH_F>
__device__ __forceinline__ void vjp_block_body(
    int64_t N, int64_t E, int64_t n_blocks, const int64_t* __restrict__ node_off,
    const int32_t* __restrict__ nodes, const uint32_t* __restrict__ runs, int cap,
    const RecChunk* __restrict__ rec, const double* __restrict__ geom64,
    const R* __restrict__ up, const R* __restrict__ cot, const ElemParams<R>& P,
    double* __restrict__ rhs, double* __restrict__ grad, const int32_t* __restrict__ order,
    int64_t i0, int64_t i1) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const size_t sbytes = stage_bytes<R, 8>(cap);
  R* sG = reinterpret_cast<R*>(smem_raw + kStages * sbytes);  // [kBlockSlots][4] gradient entries
  R* sFr = sG + kBlockSlots * 4;                                // [kBlockSlots][4] RHS entries (WITH_F)
  const int tid = threadIdx.x;
  const int64_t first = COLOUR ? i0 : 0, last = COLOUR ? i1 : n_blocks;
  auto block_at = [&](int64_t i) -> int64_t { return COLOUR ? (int64_t)__ldg(order + i) : i; };
  int64_t i = first + blockIdx.x;
#pragma unroll 1
  for (int k = 0; k < kStages - 1; ++k) {
    const int64_t ik = i + (int64_t)k * gridDim.x;
    if (ik < last)
      stage_block<R, 8>(N, block_at(ik), node_off, nodes, runs, up, cot, smem_raw + k * sbytes,
                        cap);
    cp_async_commit();
  }
  RecAhead<R, 1> ra;
  if (i < last && block_at(i) * kBlockElems + tid < E) ra.load(rec, block_at(i) * kBlockElems + tid);
  for (int step = 0; i < last; i += gridDim.x, ++step) {
    const int64_t b = block_at(i);
    const int64_t bn = i + gridDim.x < last ? block_at(i + gridDim.x) : -1;
    unsigned char* st = smem_raw + (step % kStages) * sbytes;
    cp_async_wait<kStages - 2>();
    __syncthreads();
    {
      const int64_t ia = i + (int64_t)(kStages - 1) * gridDim.x;
      if (ia < last)
        stage_block<R, 8>(N, block_at(ia), node_off, nodes, runs, up, cot,
                          smem_raw + ((step + kStages - 1) % kStages) * sbytes, cap);
      cp_async_commit();
    }
    const int64_t e = b * kBlockElems + tid;
    if (e < E) {
      const RecAhead<R, 1> cur = ra;
      const uint32_t lmv[4] = {cur.lm.x, cur.lm.y, cur.lm.z, cur.lm.w};
      const R* vals = reinterpret_cast<const R*>(st);
      R u[4][3], p[4], w[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int lc = (int)(lmv[a] >> 16);
        R q[4];
        Smem<R>::get4(vals, 8, lc, q);
        u[a][0] = q[0];
        u[a][1] = q[1];
        u[a][2] = q[2];
        p[a] = q[3];
        Smem<R>::get4(vals + 4, 8, lc, w[a]);
      }
      R c[3][3], inv_det, rh;
      cur.geometry(rec, geom64, E, e, c, inv_det, rh);
      R gu[4][3], gp[4];
      if constexpr (WITH_F) {
        R F[4][4];
        if constexpr (sizeof(R) == 4)
          element_rhs_vjp<R, FLAGS>(c, inv_det, rh, u, p, w, P, F, gu, gp,
                                    PutRhs<R, StagedReload<R, 8>>{{vals, lmv}, sFr, lmv});
        else
          element_rhs_vjp<R, FLAGS>(c, inv_det, rh, u, p, w, P, F, gu, gp,
                                    PutRhs<R, NoReload>{{}, sFr, lmv});
      } else {
        if constexpr (sizeof(R) == 4)
          element_vjp<R, FLAGS>(c, inv_det, rh, u, p, w, P, gu, gp, StagedReload<R, 8>{vals, lmv});
        else
          element_vjp<R, FLAGS>(c, inv_det, rh, u, p, w, P, gu, gp);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const R g4[4] = {gu[a][0], gu[a][1], gu[a][2], gp[a]};
        Smem<R>::put4(sG, (int)(lmv[a] & 0xffffu), g4);
      }
    }
    if (bn >= 0 && bn * kBlockElems + tid < E) ra.load(rec, bn * kBlockElems + tid);
    const int nb = (int)(__ldg(node_off + b + 1) - __ldg(node_off + b));
    __syncthreads();
    const int32_t* ids = reinterpret_cast<const int32_t*>(st + (size_t)cap * 8 * sizeof(R));
    const uint32_t* rl = reinterpret_cast<const uint32_t*>(ids + cap);
    if constexpr (WITH_F)
      block_node_sums2<R>(N, nb, ids, rl, sFr, rhs, sG, grad);
    else
      block_node_sums<R>(N, nb, ids, rl, sG, grad);
  }
  cp_async_wait<0>();
}

template <class R, int FLAGS, bool COLOUR = false>
__global__ void __launch_bounds__(kBlockElems, block_vjp_min_ctas<R>())
    vjp_block_kernel(int64_t N, int64_t E, int64_t n_blocks, const int64_t* __restrict__ node_off,
                     const int32_t* __restrict__ nodes, const uint32_t* __restrict__ runs,
                     int cap, const RecChunk* __restrict__ rec, const double* __restrict__ geom64,
                     const R* __restrict__ up, const R* __restrict__ cot, ElemParams<R> P,
                     double* __restrict__ grad, const int32_t* __restrict__ order, int64_t i0,
                     int64_t i1) {
  vjp_block_body<R, FLAGS, COLOUR, false>(N, E, n_blocks, node_off, nodes, runs, cap, rec, geom64,
                                          up, cot, P, nullptr, grad, order, i0, i1);
}

// The RHS and the adjoint at the same state in one pass (see vjp_block_body).
template <class R, int FLAGS, bool COLOUR = false>
__global__ void __launch_bounds__(kBlockElems, block_vjp_min_ctas<R>())
    rhs_vjp_block_kernel(int64_t N, int64_t E, int64_t n_blocks,
                         const int64_t* __restrict__ node_off, const int32_t* __restrict__ nodes,
                         const uint32_t* __restrict__ runs, int cap,
                         const RecChunk* __restrict__ rec, const double* __restrict__ geom64,
                         const R* __restrict__ up, const R* __restrict__ cot, ElemParams<R> P,
                         double* __restrict__ rhs, double* __restrict__ grad,
                         const int32_t* __restrict__ order, int64_t i0, int64_t i1) {
  vjp_block_body<R, FLAGS, COLOUR, true>(N, E, n_blocks, node_off, nodes, runs, cap, rec, geom64,
                                         up, cot, P, rhs, grad, order, i0, i1);
}

}  // namespace nsrhs
