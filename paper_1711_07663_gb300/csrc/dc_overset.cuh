// dc_overset.cuh -- what follows the cut: the union of several cuts, the
// artificial-boundary faces, and the unblank step of a moving grid.
//
// Sec. 4.2 (final paragraphs): the hole cells of every cutting boundary are
// united into the final blanking; artificial-boundary faces are the faces with
// a hole cell on one side and a normal cell on the other.  Algorithm
// "Artificial Boundary unblank procedure" (Sec. 3): cuts at t and t + dt;
// wall cuts remove what either removes, overset cuts only what both remove;
// cells removed before and kept now are unblanked.  One cut removes its HOLE
// elements, and for a solid wall its FRINGE elements too (an overset boundary
// keeps the elements it passes through, which provide the overlap).
// Element-parallel and bandwidth-bound: one thread per element.
#pragma once

#include "dc_common.cuh"

namespace dc {

constexpr int OV_MAX_CUTS = 8;
enum : int { OV_WALL = 0, OV_OVERSET = 1 };

struct CutSet {
  const int8_t* flags[OV_MAX_CUTS];
  int kind[OV_MAX_CUTS];
  int n;
};

__device__ __forceinline__ bool ov_removed(int8_t f, int kind) {
  return f == DC_HOLE_ || (kind == OV_WALL && f == DC_FRINGE_);
}

// iblank (1 kept, 0 removed) of the union of the cuts
__global__ void __launch_bounds__(256) k_blank_union(CutSet cs, long long n, int8_t* __restrict__ iblank) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    bool rem = false;
    for (int k = 0; k < cs.n; ++k) rem |= ov_removed(cs.flags[k][e], cs.kind[k]);
    iblank[e] = rem ? 0 : 1;
  }
}

// per kept element, bit j when its neighbour across local face j is removed;
// count[0] += the number of such faces
__global__ void __launch_bounds__(256) k_ab_faces(long long n, const int8_t* __restrict__ iblank,
                                                  const long long* __restrict__ nbr, uint8_t* __restrict__ mask,
                                                  unsigned long long* __restrict__ count) {
  unsigned long long c = 0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    uint8_t m = 0;
    if (iblank[e]) {
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const long long o = nbr[6 * e + j];
        if (o >= 0 && o < n && !iblank[o]) m |= (uint8_t)(1u << j);
      }
    }
    mask[e] = m;
    c += __popc((unsigned)m);
  }
  for (int s = 16; s; s >>= 1) c += __shfl_xor_sync(0xffffffffu, c, s);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// the unblank step for one cut kind: iblank now, and the elements to unblank;
// count[0] += their number
__global__ void __launch_bounds__(256) k_unblank(int kind, long long n, const int8_t* __restrict__ iblank_prev,
                                                 const int8_t* __restrict__ ft, const int8_t* __restrict__ ftp,
                                                 int8_t* __restrict__ iblank, uint8_t* __restrict__ unb,
                                                 unsigned long long* __restrict__ count) {
  unsigned long long c = 0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const bool rt = ov_removed(ft[e], kind), rtp = ov_removed(ftp[e], kind);
    const bool now = kind == OV_WALL ? (rt || rtp) : (rt && rtp);
    const bool u = iblank_prev[e] == 0 && !now;
    iblank[e] = now ? 0 : 1;
    unb[e] = u ? 1 : 0;
    c += u;
  }
  for (int s = 16; s; s >>= 1) c += __shfl_xor_sync(0xffffffffu, c, s);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

}  // namespace dc
