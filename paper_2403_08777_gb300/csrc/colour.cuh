// Element colouring for the deterministic scatter.
//
// Two elements that share a node get different colours. The elements of one
// colour then add their 16 entries into the global RHS with atomics that
// never meet at one address (no two of them touch the same node), one launch
// per colour in a fixed colour order, so every RHS entry is summed in the
// same order on every call: the result is bitwise reproducible, unlike the
// unordered atomic scatter, at almost no cost (the atomics stay
// fire-and-forget). The paper's CPU code keeps a separate scalar scatter
// loop to avoid lost updates (Sec. V-C); colouring is the GPU form of that
// guarantee, with a fixed order on top.
//
// Colours are chosen greedily in the Jones-Plassmann way. Every element has a
// fixed pseudo-random priority. In each round, an uncoloured element whose
// priority is the lowest among the uncoloured elements at each of its four
// nodes takes the smallest colour not yet used at those nodes. No two
// elements accepted in one round share a node, so a round colours its whole
// accepted set at once, and the element of lowest priority overall is always
// accepted, so every round makes progress. Rounds are driven from the host
// (no device-side waiting).
//
// Blocks are coloured the same way (colour.cuh's block_* kernels): two
// element blocks (blocks.cuh) that share a node get different colours, so the
// block scatter's per-node atomics never meet at one address within a launch
// and one launch per colour fixes their order, keeping the blocks' locality.
// One warp handles one block's node list.
//
// The colour-major copy: after colouring, the elements are stably sorted by
// colour (inside a colour they keep the Morton order) and the connectivity
// and cached geometry are copied in that order, so that each colour's launch
// streams a contiguous range.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include "blocks.cuh"

namespace nsrhs {

constexpr int kMaxColours = 128;         // two 64-bit masks per node
constexpr uint8_t kUncoloured = 0xFF;

// Unique pseudo-random priority of element e (< 2^31): the high 32 bits are
// the SplitMix64 finaliser of e, the low 32 bits e itself.
__device__ __forceinline__ unsigned long long colour_priority(int64_t e) {
  unsigned long long z = (unsigned long long)e + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (z & 0xFFFFFFFF00000000ull) | (unsigned long long)(uint32_t)e;
}

// Smallest colour whose bit is clear in the 128-bit mask (m1:m0); -1 if none.
__device__ __forceinline__ int first_free_colour(unsigned long long m0, unsigned long long m1) {
  if (~m0 != 0ull) return __ffsll((long long)~m0) - 1;
  if (~m1 != 0ull) return 64 + __ffsll((long long)~m1) - 1;
  return -1;
}

// claim[n] = min priority of the uncoloured elements at node n
// (claim initialised to all ones).
__global__ void colour_claim_kernel(int64_t E, const int32_t* __restrict__ conn,
                                    const uint8_t* __restrict__ colour,
                                    unsigned long long* __restrict__ claim) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (colour[e] != kUncoloured) continue;
    const unsigned long long key = colour_priority(e);
#pragma unroll
    for (int a = 0; a < 4; ++a) atomicMin(claim + conn[a * E + e], key);
  }
}

// An uncoloured element that holds the claim of all four of its nodes takes
// the smallest colour absent from their masks used[2n], used[2n+1].
// counters[0] += elements coloured; counters[1] += elements that found no
// free colour among kMaxColours.
__global__ void colour_accept_kernel(int64_t E, const int32_t* __restrict__ conn,
                                     const unsigned long long* __restrict__ claim,
                                     unsigned long long* __restrict__ used,
                                     uint8_t* __restrict__ colour,
                                     unsigned long long* __restrict__ counters) {
  unsigned long long coloured = 0, overflow = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (colour[e] != kUncoloured) continue;
    const unsigned long long key = colour_priority(e);
    int32_t v[4];
    bool mine = true;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      v[a] = conn[a * E + e];
      mine = mine && claim[v[a]] == key;
    }
    if (!mine) continue;
    unsigned long long m0 = 0, m1 = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      m0 |= used[2 * (int64_t)v[a]];
      m1 |= used[2 * (int64_t)v[a] + 1];
    }
    const int c = first_free_colour(m0, m1);
    if (c < 0) {
      ++overflow;
      continue;
    }
    colour[e] = (uint8_t)c;
    const unsigned long long bit = 1ull << (c & 63);
#pragma unroll
    for (int a = 0; a < 4; ++a) atomicOr(used + 2 * (int64_t)v[a] + (c >> 6), bit);
    ++coloured;
  }
  if (coloured) atomicAdd(counters, coloured);
  if (overflow) atomicAdd(counters + 1, overflow);
}

// counts[c] += elements of colour c (block-local histogram first).
__global__ void colour_count_kernel(int64_t E, const uint8_t* __restrict__ colour,
                                    unsigned long long* __restrict__ counts) {
  __shared__ unsigned int h[kMaxColours];
  for (int i = threadIdx.x; i < kMaxColours; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    const unsigned c = colour[e];
    if (c < (unsigned)kMaxColours) atomicAdd(h + c, 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kMaxColours; i += blockDim.x)
    if (h[i]) atomicAdd(counts + i, (unsigned long long)h[i]);
}

// Independent check of a colouring: seen[2n + c/64] collects the colours met
// at node n; a colour met twice at one node, or an element left uncoloured,
// increments *bad. seen must start at zero.
__global__ void colour_check_kernel(int64_t E, const int32_t* __restrict__ conn,
                                    const uint8_t* __restrict__ colour,
                                    unsigned long long* __restrict__ seen,
                                    unsigned long long* __restrict__ bad) {
  unsigned long long nbad = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = colour[e];
    if (c >= kMaxColours) {
      ++nbad;
      continue;
    }
    const unsigned long long bit = 1ull << (c & 63);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const unsigned long long old = atomicOr(seen + 2 * (int64_t)conn[a * E + e] + (c >> 6), bit);
      if (old & bit) ++nbad;
    }
  }
  if (nbad) atomicAdd(bad, nbad);
}

__global__ void iota_kernel(int64_t n, int32_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int32_t)i;
}

// dst[r][i] = src[r][perm[i]] for rows r < rows, rows of length E.
template <class T>
__global__ void permute_rows_kernel(int rows, int64_t E, const int32_t* __restrict__ perm,
                                    const T* __restrict__ src, T* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = perm[i];
    for (int r = 0; r < rows; ++r) dst[r * E + i] = src[r * E + e];
  }
}

// Element records in a permuted order: element i of out is element perm[i]
// of in (the four chunks of each, at their chunk-major places).
__global__ void permute_records_kernel(int64_t E, const int32_t* __restrict__ perm,
                                       const RecChunk* __restrict__ in,
                                       RecChunk* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = perm[i];
#pragma unroll
    for (int k = 0; k < 4; ++k) out[rec_index(i, k)] = in[rec_index(e, k)];
  }
}

// Per element e (Morton position) in the caller's order out[order[e]]:
// which 0 its colour, 1 its block's colour, 2 its block index.
__global__ void colour_export_kernel(int64_t E, int which, int block_elems,
                                     const int32_t* __restrict__ order,
                                     const uint8_t* __restrict__ colour,
                                     const uint8_t* __restrict__ block_colour,
                                     int32_t* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / block_elems;
    out[order[e]] = which == 0 ? (int32_t)colour[e]
                               : which == 1 ? (int32_t)block_colour[b] : (int32_t)b;
  }
}

// ---- block colouring (one warp per block, node lists in CSR form) ----

__global__ void block_colour_claim_kernel(int64_t nb, const int64_t* __restrict__ node_off,
                                          const int32_t* __restrict__ nodes,
                                          const uint8_t* __restrict__ colour,
                                          unsigned long long* __restrict__ claim) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; b < nb; b += nwarps) {
    if (colour[b] != kUncoloured) continue;
    const unsigned long long key = colour_priority(b);
    for (int64_t j = node_off[b] + lane; j < node_off[b + 1]; j += 32) atomicMin(claim + nodes[j], key);
  }
}

__global__ void block_colour_accept_kernel(int64_t nb, const int64_t* __restrict__ node_off,
                                           const int32_t* __restrict__ nodes,
                                           const unsigned long long* __restrict__ claim,
                                           unsigned long long* __restrict__ used,
                                           uint8_t* __restrict__ colour,
                                           unsigned long long* __restrict__ counters) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long coloured = 0, overflow = 0;
  for (int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; b < nb; b += nwarps) {
    if (colour[b] != kUncoloured) continue;
    const unsigned long long key = colour_priority(b);
    const int64_t j0 = node_off[b], j1 = node_off[b + 1];
    bool mine = true;
    unsigned long long m0 = 0, m1 = 0;
    for (int64_t j = j0 + lane; j < j1; j += 32) {
      const int64_t n = nodes[j];
      mine = mine && claim[n] == key;
      m0 |= used[2 * n];
      m1 |= used[2 * n + 1];
    }
    if (!__all_sync(0xffffffffu, mine)) continue;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      m0 |= __shfl_xor_sync(0xffffffffu, m0, o);
      m1 |= __shfl_xor_sync(0xffffffffu, m1, o);
    }
    const int c = first_free_colour(m0, m1);
    if (c < 0) {
      if (lane == 0) ++overflow;
      continue;
    }
    const unsigned long long bit = 1ull << (c & 63);
    for (int64_t j = j0 + lane; j < j1; j += 32) atomicOr(used + 2 * (int64_t)nodes[j] + (c >> 6), bit);
    if (lane == 0) {
      colour[b] = (uint8_t)c;
      ++coloured;
    }
  }
  if (coloured) atomicAdd(counters, coloured);
  if (overflow) atomicAdd(counters + 1, overflow);
}

// Independent check of a block colouring (seen starts at zero).
__global__ void block_colour_check_kernel(int64_t nb, const int64_t* __restrict__ node_off,
                                          const int32_t* __restrict__ nodes,
                                          const uint8_t* __restrict__ colour,
                                          unsigned long long* __restrict__ seen,
                                          unsigned long long* __restrict__ bad) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long nbad = 0;
  for (int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; b < nb; b += nwarps) {
    const int c = colour[b];
    if (c >= kMaxColours) {
      if (lane == 0) ++nbad;
      continue;
    }
    const unsigned long long bit = 1ull << (c & 63);
    for (int64_t j = node_off[b] + lane; j < node_off[b + 1]; j += 32) {
      const unsigned long long old = atomicOr(seen + 2 * (int64_t)nodes[j] + (c >> 6), bit);
      if (old & bit) ++nbad;
    }
  }
  if (nbad) atomicAdd(bad, nbad);
}

}  // namespace nsrhs
