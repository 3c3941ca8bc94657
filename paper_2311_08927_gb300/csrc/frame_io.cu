// Particle frames from an external CFD solver.  The paper's coupling reads
// the SPH particles of every CFD step from files (Sec. 2.3) and names that
// file traffic as a main cost (Sec. 4.3); here a frame is one binary file per
// step (positions, optional velocities and particle ids, FP32 or FP64), read
// on the host in one pass per array and scattered into the library's particle
// order on the GPU.  A CFD that sorts its particles every step (as SPH codes
// do for their neighbour search) writes them in any order with their ids.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>

#include "frames.h"

namespace chad {

bool read_frame_file(const char* path, FrameHeader& h, std::vector<double>& pos,
                     std::vector<int64_t>& id, std::string& err) {
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    err = std::string("cannot open frame file ") + path;
    return false;
  }
  auto fail = [&](const char* m) {
    std::fclose(f);
    err = m;
    return false;
  };
  if (std::fread(&h, sizeof(h), 1, f) != 1) return fail("frame file shorter than its header");
  if (std::memcmp(h.magic, "CHADFRM", 8) != 0) return fail("not a frame file (magic)");
  if (h.version != 1) return fail("unsupported frame version");
  if (h.dtype != 4 && h.dtype != 8) return fail("frame dtype must be 4 or 8 bytes");
  if (!(h.fields & kFramePos)) return fail("frame has no positions");
  if (h.fields & ~(kFramePos | kFrameVel | kFrameId)) return fail("unknown frame fields");
  if (h.n > (uint64_t(1) << 40)) return fail("frame particle count out of range");
  const size_t n = (size_t)h.n;
  pos.resize(3 * n);
  if (h.dtype == 8) {
    if (std::fread(pos.data(), sizeof(double), 3 * n, f) != 3 * n) return fail("frame truncated (positions)");
  } else {
    std::vector<float> buf(3 * n);
    if (std::fread(buf.data(), sizeof(float), 3 * n, f) != 3 * n) return fail("frame truncated (positions)");
    for (size_t i = 0; i < 3 * n; ++i) pos[i] = (double)buf[i];
  }
  if (h.fields & kFrameVel) {
    if (std::fseek(f, (long)(3 * n * h.dtype), SEEK_CUR) != 0) return fail("frame truncated (velocities)");
  }
  id.clear();
  if (h.fields & kFrameId) {
    std::vector<uint32_t> buf(n);
    if (std::fread(buf.data(), sizeof(uint32_t), n, f) != n) return fail("frame truncated (ids)");
    id.resize(n);
    for (size_t i = 0; i < n; ++i) id[i] = (int64_t)buf[i];
  }
  std::fclose(f);
  return true;
}

namespace {

__global__ void scatter_by_id_kernel(const double* pos, const int64_t* id, int64_t n, double* tmp,
                                     int* seen, int* bad) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int64_t i = id[k];
  if (i < 0 || i >= n) {
    atomicOr(bad, 1);
    return;
  }
  atomicAdd(&seen[i], 1);
  tmp[i] = pos[k];
  tmp[n + i] = pos[n + k];
  tmp[2 * n + i] = pos[2 * n + k];
}

__global__ void check_seen_kernel(const int* seen, int64_t n, int* bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && seen[i] != 1) atomicOr(bad, 2);
}

}  // namespace

cudaError_t launch_scatter_by_id(const double* pos, const int64_t* id, int64_t n, double* tmp,
                                 int* seen, int* bad, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(seen, 0, sizeof(int) * n, s);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((n + 255) / 256);
  scatter_by_id_kernel<<<grid, 256, 0, s>>>(pos, id, n, tmp, seen, bad);
  check_seen_kernel<<<grid, 256, 0, s>>>(seen, n, bad);
  return cudaGetLastError();
}

}  // namespace chad
