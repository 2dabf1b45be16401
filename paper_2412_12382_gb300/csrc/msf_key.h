// Packed Boruvka offer key of the threshold sweep (sweep.cu).
//
// An offer is the pair (L, j): L = the edge's level (1..127, the number of
// sorted thresholds it survives) and j = its oriented edge index.  Heavier
// offers win a 64-bit atomicMax: a higher level first, then the lower edge
// index, so the forest is the unique maximum spanning forest under the total
// order (L, -j).  L takes the top 7 bits and j the low 57, so every edge index
// a graph can hold (m < 2^40) packs without loss; a packed key of a valid
// offer is never 0 because L >= 1.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define TEC_HD __host__ __device__ __forceinline__
#else
#define TEC_HD inline
#endif

namespace tec {

constexpr int MSF_EDGE_BITS = 57;
constexpr uint64_t MSF_EDGE_MASK = (uint64_t(1) << MSF_EDGE_BITS) - 1;

TEC_HD uint64_t msf_key_pack(uint8_t L, int64_t j) {
    return ((uint64_t)L << MSF_EDGE_BITS) | (MSF_EDGE_MASK - (uint64_t)j);
}

TEC_HD int64_t msf_key_edge(uint64_t key) { return (int64_t)(MSF_EDGE_MASK - (key & MSF_EDGE_MASK)); }

TEC_HD uint8_t msf_key_level(uint64_t key) { return (uint8_t)(key >> MSF_EDGE_BITS); }

}  // namespace tec
