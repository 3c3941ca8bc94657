// Particle frames from an external CFD solver (frame_io.cu): the binary frame
// file, its host reader, and the scatter of frame-ordered positions into the
// library's particle order by particle id.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

namespace chad {

// The 64-byte header of a frame file (little-endian).  After it come the
// arrays, each n values, in this order: x, y, z (dtype), then u, v, w
// (dtype) when fields has bit 1, then the particle ids (uint32) when fields
// has bit 2.  Without ids the particles are in the library's order.
struct FrameHeader {
  char magic[8];      // "CHADFRM" and a NUL
  uint32_t version;   // 1
  uint32_t dtype;     // bytes per value of the position and velocity arrays: 4 or 8
  uint64_t n;         // particles
  uint64_t step;      // the CFD step the frame belongs to
  double time_s;      // its simulated time
  uint32_t fields;    // bit 0 positions (required), bit 1 velocities, bit 2 ids
  uint32_t reserved[5];
};
static_assert(sizeof(FrameHeader) == 64, "frame header is 64 bytes");

constexpr uint32_t kFramePos = 1u, kFrameVel = 2u, kFrameId = 4u;

// Reads and checks a frame file.  pos receives [3][n] doubles (FP32 values
// widened exactly), id the n particle ids (empty when the frame has none).
// Returns false with a message in err on any I/O or format error.
bool read_frame_file(const char* path, FrameHeader& h, std::vector<double>& pos,
                     std::vector<int64_t>& id, std::string& err);

// tmp[d][id[k]] = pos[d][k] for the n frame entries (pos, tmp: [3][n]), with
// seen[i] counting how often particle i was named; bad |= 1 for an id outside
// [0, n), |= 2 (second kernel) for a particle named other than once.
cudaError_t launch_scatter_by_id(const double* pos, const int64_t* id, int64_t n, double* tmp,
                                 int* seen, int* bad, cudaStream_t s);

}  // namespace chad
