// Index checks of the bounds-check build (compiled with -DCHAD_DEBUG_BOUNDS
// into libchad_debug.so).  A failed check ORs its code into a device status
// word of the translation unit and the access is skipped; nothing traps.
// In the normal build every check is the constant true.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#ifdef CHAD_DEBUG_BOUNDS
#define CHAD_BOUNDS_WORD(tu) static __device__ unsigned int chad_bounds_word_##tu = 0u;
#define CHAD_IN_BOUNDS(tu, cond, code) \
  ((cond) ? true : (atomicOr(&chad_bounds_word_##tu, (unsigned int)(code)), false))
// Host read (and reset) of the translation unit's word.
#define CHAD_BOUNDS_ACCESSOR(tu)                                                            \
  unsigned int bounds_status_##tu(bool reset) {                                            \
    unsigned int v = 0u;                                                                    \
    if (cudaMemcpyFromSymbol(&v, chad_bounds_word_##tu, sizeof(v)) != cudaSuccess) return ~0u; \
    if (reset) {                                                                            \
      const unsigned int z = 0u;                                                            \
      cudaMemcpyToSymbol(chad_bounds_word_##tu, &z, sizeof(z));                             \
    }                                                                                       \
    return v;                                                                               \
  }
#else
#define CHAD_BOUNDS_WORD(tu)
#define CHAD_IN_BOUNDS(tu, cond, code) true
#define CHAD_BOUNDS_ACCESSOR(tu) \
  unsigned int bounds_status_##tu(bool) { return 0u; }
#endif

namespace chad {
// Status codes, one bit per check site.
enum : unsigned int {
  kBoundsCell = 1u << 0,      // cell id outside the grid
  kBoundsScatter = 1u << 1,   // cell-list slot outside [0, n)
  kBoundsRange = 1u << 2,     // neighbour slot range beyond the slots
  kBoundsQueue = 1u << 3,     // per-warp candidate queue overflow
  kBoundsColumn = 1u << 4,    // stored neighbour column outside the slots
  kBoundsOrder = 1u << 5,     // ordering slot outside [0, n)
  kBoundsBucket = 1u << 6,    // ordering bucket outside [0, 16)
};
unsigned int bounds_status_diffusion(bool reset);
unsigned int bounds_status_aux(bool reset);
}  // namespace chad
