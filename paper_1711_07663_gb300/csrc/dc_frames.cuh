// dc_frames.cuh -- the sweeps over every element node (the cold path of a
// grid): element node boxes rounded outward (k_elem_boxes, every resident
// grid and the allocation-free cut) and, for the donor search's grid, also the
// element frame (k_elem_frames: origin at the centre of the float box, node
// coordinates relative to it rounded to float, [e][x|y|z block][node]).
//
// The node array is the one place the whole grid is read ((p+1)^3 x 3 FP64 per
// element, 170 MB at 64^3 Q2), so it is read as contiguous tiles: a block
// takes `eb` consecutive elements at a time (eb * (p+1)^3 * 24 bytes, at most
// 48 KB), one thread copies each tile into shared memory with a bulk
// asynchronous copy (cp.async.bulk, completion counted on an mbarrier) ahead
// of its use (two buffers: the next copy is in flight while the block works on
// the current tile), and the block writes its
// boxes, origins and frame coordinates from shared memory in element order,
// so every global access of the sweep is a contiguous span.  Tiles whose
// global address or size is not a multiple of 16 bytes (a node array that is
// not 16-byte aligned, the grid's last tile) are loaded by the threads with
// plain coalesced loads instead.
//
// Every wait on the mbarrier is bounded: a wait that runs out sets *err, the
// block waits (bounded again) for its own copies, and returns.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <limits.h>
#include <stdint.h>

namespace dc {

constexpr int FR_THREADS = 256;
// a ring of FR_STAGES tile buffers of at most 48 KB: a block keeps
// FR_STAGES - 1 copies in flight while it reduces the tile it holds
constexpr int FR_STAGES = 2;
constexpr int FR_MAX_TILE_BYTES = 48 * 1024;
constexpr unsigned FR_WAIT_LIMIT = 1u << 22;  // try_wait polls before a wait gives up

// elements per tile: the largest power of two (<= 128) whose nodes fit the
// tile, but at least 8 (a group of FR_THREADS / eb <= 32 threads reduces one
// element's nodes within a warp)
__host__ __device__ inline int frames_tile_elems(int npe) {
  int eb = 128;
  while (eb > 8 && (long long)eb * npe * 24 > FR_MAX_TILE_BYTES) eb >>= 1;
  return eb;
}

// GB300 issues FP64 arithmetic at about 1/64 of its FP32 rate, so the box of
// the nodes is taken on integer keys of the FP64 bit patterns: for finite
// doubles the key order is the numeric order (negative values have their
// magnitude bits flipped), and the key map is its own inverse.
__device__ __forceinline__ long long fr_key(long long b) { return b ^ ((b >> 63) & 0x7fffffffffffffffLL); }

__device__ __forceinline__ unsigned fr_smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void fr_bar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(fr_smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one thread: expect `bytes` on the barrier and start the bulk copy
__device__ __forceinline__ void fr_bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fr_smem_addr(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          fr_smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(fr_smem_addr(bar))
      : "memory");
}

// bounded wait for phase `parity` of the barrier; false if it never came
__device__ __forceinline__ bool fr_bar_wait(uint64_t* bar, unsigned parity) {
  for (unsigned it = 0; it < FR_WAIT_LIMIT; ++it) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(fr_smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// grid: persistent blocks of FR_THREADS threads, dynamic shared memory
// FR_STAGES * eb * npe * 24 bytes (the tile buffers).  loc/org may be null (boxes
// only), ext_sum may be null.
__global__ void __launch_bounds__(FR_THREADS) k_elem_frames(const double* __restrict__ nodes, long long n_elem,
                                                            int npe, int eb, float* __restrict__ box,
                                                            float* __restrict__ loc, double* __restrict__ org,
                                                            int* __restrict__ bad, double* __restrict__ ext_sum,
                                                            int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar[FR_STAGES];
  __shared__ double s_org[128][3];
  __shared__ double s_ext[FR_THREADS / 32];
  __shared__ int s_bad;
  const int tid = threadIdx.x;
  const long long tile_doubles = (long long)eb * npe * 3;
  double* const buf0 = reinterpret_cast<double*>(smem);
  const long long n_tiles = (n_elem + eb - 1) / eb;
  const bool aligned = ((uintptr_t)nodes & 15) == 0;
  // a tile goes by bulk copy when its address and size are 16-byte multiples
  auto bulk_ok = [&](long long t) {
    const long long ne = (t + 1) * eb <= n_elem ? eb : n_elem - t * eb;
    return aligned && ((t * eb * npe * 24) & 15) == 0 && ((ne * npe * 24) & 15) == 0;
  };
  auto tile_elems = [&](long long t) { return (int)((t + 1) * eb <= n_elem ? eb : n_elem - t * eb); };
  if (tid == 0) {
    for (int b = 0; b < FR_STAGES; ++b) fr_bar_init(&bar[b]);
    s_bad = 0;
  }
  if (tid < FR_THREADS / 32) s_ext[tid] = 0.0;
  __syncthreads();
  long long t = blockIdx.x;
  unsigned phase = 0u;   // bit b: parity of buffer b's next phase
  unsigned issued = 0u;  // bit b: buffer b has a bulk copy outstanding (thread 0's record)
  bool failed = false;
  // the first FR_STAGES - 1 tiles of this block
  for (int j = 0; j < FR_STAGES - 1; ++j) {
    const long long tj = t + (long long)j * gridDim.x;
    if (tj < n_tiles && tid == 0 && bulk_ok(tj)) {
      fr_bulk_load(buf0 + j * tile_doubles, nodes + tj * tile_doubles, (unsigned)(tile_elems(tj) * npe * 24), &bar[j]);
      issued |= 1u << j;
    }
  }
  // per element: T_E = FR_THREADS / eb threads (eb <= 128 so T_E >= 2)
  const int te = FR_THREADS / eb;
  double ext_acc = 0.0;
  for (int k = 0; t < n_tiles; ++k, t += gridDim.x) {
    const int b = k % FR_STAGES;
    const long long tn = t + (long long)(FR_STAGES - 1) * gridDim.x;
    const int bn = (k + FR_STAGES - 1) % FR_STAGES;
    if (tn < n_tiles && tid == 0 && bulk_ok(tn)) {
      // buffer bn held the tile of the last round, released by its final barrier
      fr_bulk_load(buf0 + bn * tile_doubles, nodes + tn * tile_doubles, (unsigned)(tile_elems(tn) * npe * 24),
                   &bar[bn]);
      issued |= 1u << bn;
    }
    const int ne = tile_elems(t);
    double* tb = buf0 + b * tile_doubles;
    if (bulk_ok(t)) {
      if (fr_bar_wait(&bar[b], (phase >> b) & 1u)) {
        phase ^= 1u << b;
        issued &= ~(1u << b);
      } else {
        failed = true;  // phase and count stay: the clean-up waits for this copy
      }
    } else {
      const double* src = nodes + t * tile_doubles;
      for (long long j = tid; j < (long long)ne * npe * 3; j += FR_THREADS) tb[j] = src[j];
    }
    if (__syncthreads_or(failed)) {
      failed = true;
      break;
    }
    // boxes: thread group g (te threads) reduces element g's nodes, on the
    // integer keys (a coordinate of magnitude 1e300 or more, or not finite,
    // marks the grid bad)
    const int g = tid / te, r = tid - g * te;
    const long long big = __double_as_longlong(1e300);
    long long klo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, khi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
    bool nonfinite = false;
    if (g < ne) {
      const long long* x = reinterpret_cast<const long long*>(tb) + (long long)g * npe * 3;
      for (int nd = r; nd < npe; nd += te)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const long long b = x[3 * nd + a];
          nonfinite |= (b & 0x7fffffffffffffffLL) >= big;
          const long long k = fr_key(b);
          klo[a] = min(klo[a], k);
          khi[a] = max(khi[a], k);
        }
    }
    for (int s = 1; s < te; s <<= 1)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        klo[a] = min(klo[a], __shfl_xor_sync(0xffffffffu, klo[a], s));
        khi[a] = max(khi[a], __shfl_xor_sync(0xffffffffu, khi[a], s));
      }
    if (nonfinite) s_bad = 1;
    if (g < ne && r == 0) {
      const long long e = t * eb + g;
      double ext = 0.0;
      double lo[3], hi[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        lo[a] = __longlong_as_double(fr_key(klo[a]));
        hi[a] = __longlong_as_double(fr_key(khi[a]));
      }
      for (int a = 0; a < 3; ++a) {
        const float bl = __double2float_rd(lo[a]), bh = __double2float_ru(hi[a]);
        box[6 * e + a] = bl;
        box[6 * e + 3 + a] = bh;
        s_org[g][a] = 0.5 * ((double)bl + (double)bh);
        ext = fmax(ext, hi[a] - lo[a]);
      }
      if (ext < 1e300) ext_acc += ext;
    }
    __syncthreads();
    if (loc) {
      // the tile's frame coordinates are one contiguous span of the output
      const int per = 3 * npe;
      float* out = loc + t * eb * (long long)per;
      for (int j = tid; j < ne * per; j += FR_THREADS) {
        const int el = j / per, rr = j - el * per, a = rr / npe, nd = rr - a * npe;
        out[j] = (float)(tb[(long long)el * per + 3 * nd + a] - s_org[el][a]);
      }
      for (int j = tid; j < ne * 3; j += FR_THREADS) org[t * eb * 3 + j] = s_org[j / 3][j % 3];
    }
    __syncthreads();  // this buffer and s_org are free for the next tiles
  }
  if (failed) {
    // a copy never completed: note it, let this block's own copies land
    // (bounded), and leave
    if (tid == 0) {
      atomicOr(err, 1);
      for (int b = 0; b < FR_STAGES; ++b)
        if ((issued >> b) & 1u) fr_bar_wait(&bar[b], (phase >> b) & 1u);  // at most one copy per buffer
    }
    return;
  }
  if (ext_sum) {
    for (int s = 16; s; s >>= 1) ext_acc += __shfl_xor_sync(0xffffffffu, ext_acc, s);
    if ((tid & 31) == 0) s_ext[tid >> 5] = ext_acc;
    __syncthreads();
    if (tid == 0) {
      double sum = 0.0;
      for (int w = 0; w < FR_THREADS / 32; ++w) sum += s_ext[w];
      if (sum > 0.0) atomicAdd(ext_sum, sum);
    }
  }
  __syncthreads();
  if (tid == 0 && s_bad) atomicOr(bad, 1);
}

// Element node boxes only, read straight from global memory: a group of
// FB_GROUP = 4 threads per element, 8 elements per warp.  Thread r of a group
// reads the element's coordinates r, r + 4, r + 8, ... (every load of a warp
// covers 32 contiguous bytes of each of its 8 elements), twelve at a time, so
// that within each twelve its three values fall on the axes r mod 3, r + 1 and
// r + 2 mod 3 in that order: fixed accumulators, no indexing by axis.  The
// boxes are taken on order-preserving 64-bit integer keys of the FP64 bits
// (fr_key), so the sweep does no FP64 arithmetic but the final outward
// rounding; a coordinate of magnitude 1e300 or more, or not finite, is found
// on the reduced keys.
// No shared memory or barrier: the whole SM's warps keep loads in flight,
// which is what the sweep (a pure stream over the node array) needs.  The
// grid is one wave (fb_grid): the loop strides over the elements, so no SM
// idles through a partial second wave.
constexpr int FB_GROUP = 4;

// an order-preserving key of a finite double as two 32-bit words (high word
// signed, low word unsigned, compared in that order; the surface tiles' face
// boxes use it)
struct FbKey {
  int h;
  unsigned l;
};
__device__ __forceinline__ FbKey fb_key(long long b) {
  int h = (int)(b >> 32);
  unsigned l = (unsigned)b;
  const int neg = h >> 31;  // all ones for a negative value: flip its magnitude bits
  return FbKey{h ^ (neg & 0x7fffffff), l ^ (unsigned)neg};
}
__device__ __forceinline__ bool fb_less(FbKey a, FbKey b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }
__device__ __forceinline__ double fb_value(FbKey k) {
  const int neg = k.h >> 31;
  const int h = k.h ^ (neg & 0x7fffffff);
  const unsigned l = k.l ^ (unsigned)neg;
  return __longlong_as_double(((long long)h << 32) | (long long)l);
}

__global__ void __launch_bounds__(256) k_elem_boxes(const double* __restrict__ nodes, long long n_elem, int npe,
                                                    float* __restrict__ box, int* __restrict__ bad,
                                                    double* __restrict__ ext_sum) {
  const int lane = threadIdx.x & 31, r = lane & (FB_GROUP - 1);
  const int nval = 3 * npe;  // in-element indices are 32-bit (measured faster)
  // keys of +-1e300: a reduced box beyond them holds a huge or non-finite node
  const long long kbig64 = fr_key(__double_as_longlong(1e300)), knbig64 = fr_key(__double_as_longlong(-1e300));
  const long long stride = (long long)gridDim.x * (blockDim.x / FB_GROUP);
  float ext_acc = 0.f;  // this thread's share of the extent sum
  bool nonfinite = false;
  // the loop runs in step across each warp (its groups' shuffles)
  for (long long e0 = ((long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) / FB_GROUP; e0 < n_elem;
       e0 += stride) {
    const long long e = e0 + (lane >> 2);
    const bool valid = e < n_elem;
    long long lo0 = LLONG_MAX, lo1 = LLONG_MAX, lo2 = LLONG_MAX, hi0 = LLONG_MIN, hi1 = LLONG_MIN, hi2 = LLONG_MIN;
    if (valid) {
      const long long* x = reinterpret_cast<const long long*>(nodes) + e * nval;
#pragma unroll 4
      for (int c = 0; c < nval; c += 12) {
        const int i0 = c + r, i1 = i0 + 4, i2 = i0 + 8;
        // past the end a load of x[0] keeps the access in bounds; its value
        // is not used
        const long long b0 = __ldg(x + (i0 < nval ? i0 : 0));
        const long long b1 = __ldg(x + (i1 < nval ? i1 : 0));
        const long long b2 = __ldg(x + (i2 < nval ? i2 : 0));
        const bool v0 = i0 < nval, v1 = i1 < nval, v2 = i2 < nval;
        const long long q0 = fr_key(b0), q1 = fr_key(b1), q2 = fr_key(b2);
        if (v0) { lo0 = min(lo0, q0); hi0 = max(hi0, q0); }
        if (v1) { lo1 = min(lo1, q1); hi1 = max(hi1, q1); }
        if (v2) { lo2 = min(lo2, q2); hi2 = max(hi2, q2); }
      }
    }
    // accumulator j of thread r holds axis (r + j) mod 3: put them in axis order
    const int m = r % 3;
    long long lo[3], hi[3];
    lo[0] = m == 0 ? lo0 : (m == 1 ? lo2 : lo1);
    lo[1] = m == 0 ? lo1 : (m == 1 ? lo0 : lo2);
    lo[2] = m == 0 ? lo2 : (m == 1 ? lo1 : lo0);
    hi[0] = m == 0 ? hi0 : (m == 1 ? hi2 : hi1);
    hi[1] = m == 0 ? hi1 : (m == 1 ? hi0 : hi2);
    hi[2] = m == 0 ? hi2 : (m == 1 ? hi1 : hi0);
#pragma unroll
    for (int s = 1; s < FB_GROUP; s <<= 1)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], s));
        hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], s));
      }
    // thread r < 3 of the group rounds axis r outward (one FP64 conversion
    // pair per thread instead of three on one: this GPU's FP64 pipe is slow);
    // the element's extent, which only sizes the hole map, is taken in float
    float ext = 0.f;
    if (valid && r < 3) {
      const long long kl = r == 0 ? lo[0] : (r == 1 ? lo[1] : lo[2]);
      const long long kh = r == 0 ? hi[0] : (r == 1 ? hi[1] : hi[2]);
      nonfinite |= kh >= kbig64 || kl <= knbig64;
      // (the key map is its own inverse)
      const float bl = __double2float_rd(__longlong_as_double(fr_key(kl)));
      const float bh = __double2float_ru(__longlong_as_double(fr_key(kh)));
      box[6 * e + r] = bl;
      box[6 * e + 3 + r] = bh;
      ext = bh - bl;
    }
    ext = fmaxf(ext, __shfl_xor_sync(0xffffffffu, ext, 1));
    ext = fmaxf(ext, __shfl_xor_sync(0xffffffffu, ext, 2));
    if (valid && r == 0 && ext < 1e30f) ext_acc += ext;
  }
  if (__any_sync(0xffffffffu, nonfinite) && lane == 0) atomicOr(bad, 1);
  if (ext_sum) {
    for (int s = 16; s; s >>= 1) ext_acc += __shfl_xor_sync(0xffffffffu, ext_acc, s);
    if (lane == 0 && ext_acc > 0.f) atomicAdd(ext_sum, (double)ext_acc);
  }
}

// k_elem_boxes' grid: one wave of resident blocks of 256 threads (no more
// blocks than 64-element groups)
inline unsigned fb_grid(long long n_elem, int n_sm) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_elem_boxes, 256, 0) != cudaSuccess || occ < 1) occ = 1;
  return (unsigned)std::max<long long>(1, std::min<long long>((n_elem + 63) / 64, (long long)n_sm * occ));
}

// dynamic shared memory of k_elem_frames for elements of npe nodes
inline size_t frames_smem(int npe) { return (size_t)FR_STAGES * frames_tile_elems(npe) * npe * 24; }

}  // namespace dc
