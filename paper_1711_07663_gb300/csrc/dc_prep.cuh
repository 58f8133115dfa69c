// dc_prep.cuh -- surface ingest, Cartesian hole map, face bins and the element
// classification/compaction kernels of libdirectcut.
//
// Sec. 4.2 of the paper ("Parallel Direct Cut Algorithm"): a hole map is a
// Cartesian grid of cubes of size ds (60-80 along the longest side), painted
// from its border; cubes touching the surface are "2", cubes outside "0", cubes
// inside "1".  Elements entirely inside "1" cubes are holes, elements entirely
// inside "0" cubes (or outside the map) are field, the rest go on to the
// distance tests.  Here the map is built exactly (conservatively):
//   * a cube is NEAR when a face's node box, inflated by the fringe margin,
//     overlaps it (the node box contains the linearised face);
//   * the non-NEAR cubes are split into connected components (runs along x,
//     union-find over face-adjacent runs); components touching the border are
//     outside; every other component is labelled by the winding number of its
//     first cube's centre (the cube centre is at least ds/2 from the surface);
//   * element boxes are looked up cube by cube, so an element is decided only
//     when every cube it may touch agrees.
#pragma once

#include "dc_common.cuh"

namespace dc {

__constant__ unsigned char c_etri[MAX_P][MAX_NTE][3];   // element boundary triangles, per p
__constant__ unsigned char c_ftri[MAX_Q][MAX_NTF][3];   // cut-face triangles, per q

constexpr int CUBE_PITCH = 96;  // bytes per x-row of the hole map (>= MAX_DIM, 16-byte multiple)

// ------------------------------------------------------------------ a1 + a2
// Pose transform (rounded exactly as ((R0 x + R1 y) + R2 z) + t, no fusion),
// per-face node boxes, surface box and largest face extent.
__global__ void k_surface(Inst* __restrict__ I, const long long* __restrict__ foff, int n_inst,
                          long long nf_total) {
  const unsigned FULL = 0xffffffffu;
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  bool valid = g < nf_total;
  int ii = valid ? find_inst(foff, n_inst, g) : 0;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  bool bad = false;
  if (valid) {
    Inst& in = I[ii];
    long long f = g - foff[ii];
    int npf = (in.q + 1) * (in.q + 1);
    const double* src = in.faces_in + f * npf * 3;
    double* dst = in.surf + f * npf * 3;
    for (int k = 0; k < npf; ++k) {
      double x = src[3 * k], y = src[3 * k + 1], z = src[3 * k + 2];
      double o[3];
      if (in.has_pose) {
        for (int a = 0; a < 3; ++a) {
          const double* R = in.pose + 4 * a;
          o[a] = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(R[0], x), __dmul_rn(R[1], y)), __dmul_rn(R[2], z)), R[3]);
        }
      } else {
        o[0] = x; o[1] = y; o[2] = z;
      }
      for (int a = 0; a < 3; ++a) {
        dst[3 * k + a] = o[a];
        bad |= !(fabs(o[a]) < 1e300);
        lo[a] = fmin(lo[a], o[a]);
        hi[a] = fmax(hi[a], o[a]);
      }
    }
    for (int a = 0; a < 3; ++a) {
      in.fbox64[6 * f + a] = lo[a];
      in.fbox64[6 * f + 3 + a] = hi[a];
      in.fbox[6 * f + a] = __double2float_rd(lo[a]);
      in.fbox[6 * f + 3 + a] = __double2float_ru(hi[a]);
      atomicMax(&in.fext_bits[a], __float_as_uint(__double2float_ru(hi[a] - lo[a]) * 1.000001f));
    }
    if (bad) atomicOr(&in.err, (int)ERR_NONFINITE);
  }
  int i0 = __shfl_sync(FULL, ii, 0);
  bool same = __all_sync(FULL, !valid || ii == i0);
  if (same) {
    for (int a = 0; a < 3; ++a) {
      for (int s = 16; s; s >>= 1) {
        lo[a] = fmin(lo[a], __shfl_xor_sync(FULL, lo[a], s));
        hi[a] = fmax(hi[a], __shfl_xor_sync(FULL, hi[a], s));
      }
    }
    if ((threadIdx.x & 31) == 0 && lo[0] <= hi[0]) {
      Inst& in = I[i0];
      for (int a = 0; a < 3; ++a) {
        atomicMin(&in.sbox_key[a], dkey(lo[a]));
        atomicMax(&in.sbox_key[3 + a], dkey(hi[a]));
      }
    }
  } else if (valid) {
    Inst& in = I[ii];
    for (int a = 0; a < 3; ++a) {
      atomicMin(&in.sbox_key[a], dkey(lo[a]));
      atomicMax(&in.sbox_key[3 + a], dkey(hi[a]));
    }
  }
}

// hole-map and bin geometry from the surface box (one thread per instance)
__global__ void k_grid(Inst* __restrict__ I, int n_inst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_inst) return;
  Inst& in = I[i];
  double lo[3], hi[3], L = 0.0;
  for (int a = 0; a < 3; ++a) {
    lo[a] = dkey_decode(in.sbox_key[a]);
    hi[a] = dkey_decode(in.sbox_key[3 + a]);
    L = fmax(L, hi[a] - lo[a]);
  }
  if (!(L > 0.0) || !(L < 1e300)) {
    in.err |= ERR_DEGENERATE;
    L = 1.0;
  }
  int cells = in.holemap_cells;
  double ds = L / cells;
  in.ds = ds;
  int nb = 1;
  for (int a = 0; a < 3; ++a) {
    double span = fmax(hi[a] - lo[a], 0.0) / ds;
    int n = (int)ceil(fmin(span, (double)cells));
    n = clampi(n, 1, cells);
    in.dims[a] = n + 2;
    in.origin[a] = lo[a] - ds;
    in.bdims[a] = (in.dims[a] + in.bin_cubes - 1) / in.bin_cubes;
    nb *= in.bdims[a];
  }
  in.bs = ds * in.bin_cubes;
  for (int a = 0; a < 3; ++a) in.origin_f[a] = (float)in.origin[a];
  in.inv_ds_f = (float)(1.0 / ds);
  in.inv_bs_f = (float)(1.0 / in.bs);
  if (nb > in.nbins_cap) in.err |= ERR_DEGENERATE;  // sized on the host for the worst case
}

__global__ void k_clear(Inst* __restrict__ I) {
  Inst& in = I[blockIdx.y];
  long long ncube = (long long)in.dims[1] * in.dims[2] * CUBE_PITCH;
  int nb = in.bdims[0] * in.bdims[1] * in.bdims[2];
  if (nb > in.nbins_cap) nb = 0;
  uint4* c4 = reinterpret_cast<uint4*>(in.cube);
  long long n4 = ncube / 16;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n4; k += (long long)gridDim.x * blockDim.x)
    c4[k] = make_uint4(0, 0, 0, 0);
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += (long long)gridDim.x * blockDim.x)
    in.bin_cnt[k] = 0;
}

__device__ __forceinline__ int cube_floor(double x, int n) {
  // floor(x) clamped into [-1, n] (x may be huge or NaN for degenerate input)
  if (!(x > -1.0)) return -1;
  if (!(x < (double)n)) return n;
  return (int)floor(x);
}

// the same for float arguments
__device__ __forceinline__ int cube_floorf(float x, int n) {
  if (!(x > -1.0f)) return -1;
  if (!(x < (float)n)) return n;
  return (int)floorf(x);
}

// a3: NEAR tags of the hole map, and face -> bin (bin of the box's min corner)
__global__ void k_tag(Inst* __restrict__ I, const long long* __restrict__ foff, int n_inst, long long nf_total) {
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nf_total) return;
  int ii = find_inst(foff, n_inst, g);
  Inst& in = I[ii];
  if (in.err & ERR_DEGENERATE) return;
  long long f = g - foff[ii];
  // cube range of the face box inflated by the fringe margin 2 tol, in float:
  // the extra 1e-3 cube (plus 16 ulp of the coordinates) only ever adds cubes
  const float mu = (float)(2.0 * in.tol);
  int c0[3], c1[3], b[3];
  for (int a = 0; a < 3; ++a) {
    float lo = in.fbox[6 * f + a], hi = in.fbox[6 * f + 3 + a];  // rounded outward
    float o = in.origin_f[a];
    float slack = 1e-3f + 16.0f * 5.9604645e-8f * (fabsf(lo) + fabsf(hi) + fabsf(o)) * in.inv_ds_f;
    float x0 = (lo - mu - o) * in.inv_ds_f - slack, x1 = (hi + mu - o) * in.inv_ds_f + slack;
    c0[a] = max(cube_floor((double)x0, in.dims[a]), 0);
    c1[a] = min(cube_floor((double)x1, in.dims[a]), in.dims[a] - 1);
    b[a] = clampi(cube_floor((double)((lo - o) * in.inv_bs_f), in.bdims[a]), 0, in.bdims[a] - 1);
  }
  for (int z = c0[2]; z <= c1[2]; ++z)
    for (int y = c0[1]; y <= c1[1]; ++y) {
      uint8_t* row = in.cube + ((long long)z * in.dims[1] + y) * CUBE_PITCH;
      for (int x = c0[0]; x <= c1[0]; ++x) row[x] = CUBE_NEAR;
    }
  int bi = (b[2] * in.bdims[1] + b[1]) * in.bdims[0] + b[0];
  in.fbin[f] = bi;
  atomicAdd(&in.bin_cnt[bi], 1);
}

// exclusive scan of the bin counts (one CTA per instance); counts become cursors
__global__ void k_bin_scan(Inst* __restrict__ I) {
  __shared__ int sums[1024];
  Inst& in = I[blockIdx.x];
  int nb = in.bdims[0] * in.bdims[1] * in.bdims[2];
  if ((in.err & ERR_DEGENERATE) || nb > in.nbins_cap) return;
  int t = threadIdx.x, T = blockDim.x;
  int chunk = (nb + T - 1) / T;
  int b0 = min(t * chunk, nb), b1 = min(b0 + chunk, nb);
  int s = 0;
  for (int k = b0; k < b1; ++k) s += in.bin_cnt[k];
  sums[t] = s;
  __syncthreads();
  for (int off = 1; off < T; off <<= 1) {
    int v = (t >= off) ? sums[t - off] : 0;
    __syncthreads();
    sums[t] += v;
    __syncthreads();
  }
  int run = sums[t] - s;
  for (int k = b0; k < b1; ++k) {
    int c = in.bin_cnt[k];
    in.bin_off[k] = run;
    run += c;
    in.bin_cnt[k] = 0;
  }
  if (t == T - 1) in.bin_off[nb] = sums[t];
}

__global__ void k_bin_fill(Inst* __restrict__ I, const long long* __restrict__ foff, int n_inst, long long nf_total) {
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nf_total) return;
  int ii = find_inst(foff, n_inst, g);
  Inst& in = I[ii];
  if (in.err & ERR_DEGENERATE) return;
  long long f = g - foff[ii];
  int b = in.fbin[f];
  int pos = in.bin_off[b] + atomicAdd(&in.bin_cnt[b], 1);
  in.bin_faces[pos] = (int)f;
}

// ------------------------------------------------------------------ a3: components
// The non-NEAR cubes of each x-row form runs; runs of face-adjacent rows that
// overlap in x are connected.  Five small kernels over all rows of all
// instances: runs into fixed per-row slots, union-find in global memory
// (hooks by atomicCAS at L2, larger root onto smaller, so parents always point
// to smaller slots and finds terminate), flatten + mark the components that
// touch the map border (outside), number the enclosed ones, write the states.
constexpr unsigned RUN_OUT = 1u, RUN_UNKNOWN = 2u;  // run_flag bits; component id in bits 4..

__device__ __forceinline__ void row_mask(const uint8_t* row, int nx, unsigned long long& m0, unsigned long long& m1) {
  // bit x set when cube x of the row is not NEAR
  const uint4* r4 = reinterpret_cast<const uint4*>(row);
  m0 = 0ull;
  m1 = 0ull;
#pragma unroll
  for (int w = 0; w < CUBE_PITCH / 16; ++w) {
    uint4 v = r4[w];
    unsigned wd[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int by = 0; by < 4; ++by) {
        int x = w * 16 + j * 4 + by;
        unsigned char c = (wd[j] >> (8 * by)) & 0xffu;
        if (x < nx && c != CUBE_NEAR) {
          if (x < 64) m0 |= 1ull << x; else m1 |= 1ull << (x - 64);
        }
      }
  }
}

// first set bit at or after x of the 128-bit mask (m0 low word), or 128
__device__ __forceinline__ int next_set(unsigned long long m0, unsigned long long m1, int x) {
  if (x < 64) {
    unsigned long long t = m0 & (~0ull << x);
    if (t) return __ffsll((long long)t) - 1;
    return m1 ? 64 + __ffsll((long long)m1) - 1 : 128;
  }
  if (x >= 128) return 128;
  unsigned long long t = m1 & (~0ull << (x - 64));
  return t ? 64 + __ffsll((long long)t) - 1 : 128;
}

__device__ __forceinline__ int rows_of(const Inst& in) { return in.dims[1] * in.dims[2]; }

// 1. runs of each row into slots (grid.y = instance)
__global__ void k_runs(Inst* __restrict__ I) {
  Inst& in = I[blockIdx.y];
  if (in.err & ERR_DEGENERATE) return;
  const int nx = in.dims[0], nrows = rows_of(in);
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += gridDim.x * blockDim.x) {
    unsigned long long m0, m1;
    uint8_t* row = in.cube + (long long)r * CUBE_PITCH;
    row_mask(row, nx, m0, m1);
    int n = 0, x = 0;
    bool over = false;
    while (true) {
      int x0 = next_set(m0, m1, x);
      if (x0 >= nx) break;
      int x1 = min(next_set(~m0, ~m1, x0), nx) - 1;
      if (n == RUNS_PER_ROW) { over = true; break; }
      int sl = r * RUNS_PER_ROW + n;
      in.run_xx[sl] = (unsigned short)(x0 | (x1 << 8));
      ++n;
      x = x1 + 1;
    }
    if (over) {
      // too many runs: make the row NEAR (walls only split components, and
      // every enclosed component is labelled by its winding number)
      for (int k = 0; k < nx; ++k) row[k] = CUBE_NEAR;
      n = 0;
    }
    in.run_cnt[r] = n;
  }
}

__device__ __forceinline__ bool overlap(unsigned short a, unsigned short b) {
  return (int)(a & 0xff) <= (int)(b >> 8) && (int)(b & 0xff) <= (int)(a >> 8);
}

// union-find over shared-memory parents that always point to smaller slots
// (path halving; hooks by atomicCAS of the larger root onto the smaller)
__device__ int uf_find(volatile int* parent, int i) {
  int p = parent[i];
  while (p != i) {
    int gp = parent[p];
    if (gp != p) parent[i] = gp;
    i = p;
    p = parent[i];
  }
  return i;
}

// root walk without writes: compression must first read every root this
// way, then (after a barrier) store them, because a concurrent path-splitting
// write could otherwise replace a stored root by an intermediate ancestor
__device__ __forceinline__ int uf_root(const volatile int* parent, int i) {
  int p;
  while ((p = parent[i]) != i) i = p;
  return i;
}

__device__ void uf_union(volatile int* parent, int a, int b) {
  while (true) {
    a = uf_find(parent, a);
    b = uf_find(parent, b);
    if (a == b) return;
    if (a < b) { int t = a; a = b; b = t; }
    if (atomicCAS((int*)&parent[a], a, b) == a) return;
  }
}

// 2. components inside each z-slice, in shared memory (one CTA per slice and
//    instance).  Runs of rows y and y-1 that overlap are joined; every run
//    records its slice root (the smallest slot of its slice component) in
//    run_par, every slice root gets a compact id (run_flag of the root slot),
//    its border bit and slot.  Each distinct (root of slice z, run of slice
//    z-1) overlap is emitted once; the join resolves the lower run's root.
// Labels of the runs of one slice by log-depth merging: in round w, the row
// blocks [2kw, 2kw+w) and [2kw+w, 2kw+2w) are joined across their boundary
// rows (every boundary y >= 1 is joined in exactly one round, w = its lowest
// set bit), one thread per boundary; then every run is relinked to its root
// (read all roots, barrier, write), so the trees stay flat and no find walks
// a chain.  One row per thread: ny <= blockDim.  Ends with parents = roots =
// the smallest slot of each component.
__device__ void slice_label(volatile int* par, const unsigned short* xx, const unsigned char* cnt, int ny) {
  const int y = threadIdx.x;
  const int n = y < ny ? cnt[y] : 0;
  for (int w = 1; w < ny; w <<= 1) {
    // boundary rows of this round: y = (2k+1) w
    if (y < ny && y >= w && ((y / w) & 1) && (y % w) == 0) {
      const int m = cnt[y - 1];
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < m; ++j)
          if (overlap(xx[y * RUNS_PER_ROW + k], xx[(y - 1) * RUNS_PER_ROW + j]))
            uf_union(par, y * RUNS_PER_ROW + k, (y - 1) * RUNS_PER_ROW + j);
    }
    __syncthreads();
    int rr[RUNS_PER_ROW];
    for (int k = 0; k < n; ++k) rr[k] = uf_root(par, y * RUNS_PER_ROW + k);
    __syncthreads();
    for (int k = 0; k < n; ++k) par[y * RUNS_PER_ROW + k] = rr[k];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_slice_cc(Inst* __restrict__ I) {
  constexpr int SL = MAX_DIM * RUNS_PER_ROW;
  __shared__ int par[SL];
  __shared__ unsigned short xx[SL], xxd[SL];
  __shared__ unsigned char cnt[MAX_DIM], cntd[MAX_DIM];
  __shared__ unsigned bord[SL];
  constexpr int HB = 2 * ZEDGE_CAP;                 // hash buckets for the distinct joins
  __shared__ unsigned long long ekeys[HB];
  __shared__ int s_ne, s_full, s_nloc;
  Inst& in = I[blockIdx.y];
  if (in.err & ERR_DEGENERATE) return;
  const int nx = in.dims[0], ny = in.dims[1], nz = in.dims[2];
  const int z = blockIdx.x;
  if (z >= nz) return;
  const int r0 = z * ny, rd0 = (z - 1) * ny;
  if (threadIdx.x == 0) { s_ne = 0; s_full = 0; s_nloc = 0; }
  for (int y = threadIdx.x; y < ny; y += blockDim.x) {
    cnt[y] = (unsigned char)in.run_cnt[r0 + y];
    cntd[y] = z > 0 ? (unsigned char)in.run_cnt[rd0 + y] : 0;
  }
  // the set of joins starts empty: shared memory may still hold keys of an
  // earlier block (the same slice of another instance has the same slots)
  for (int t = threadIdx.x; t < HB; t += blockDim.x) ekeys[t] = ~0ull;
  for (int k = threadIdx.x; k < ny * RUNS_PER_ROW; k += blockDim.x) {
    par[k] = k;
    bord[k] = 0u;
    xx[k] = in.run_xx[r0 * RUNS_PER_ROW + k];
    xxd[k] = z > 0 ? in.run_xx[rd0 * RUNS_PER_ROW + k] : 0;
  }
  __syncthreads();
  static_assert(MAX_DIM <= 256, "one row per thread");
  slice_label(par, xx, cnt, ny);
  // border bits of the slice roots; root slots, ids
  for (int y = threadIdx.x; y < ny; y += blockDim.x) {
    const int n = cnt[y];
    for (int k = 0; k < n; ++k) {
      const int sl = y * RUNS_PER_ROW + k;
      unsigned short a = xx[sl];
      bool b = y == 0 || y == ny - 1 || z == 0 || z == nz - 1 || (a & 0xff) == 0 || (int)(a >> 8) == nx - 1;
      if (b && !(((volatile unsigned*)bord)[par[sl]] & 1u)) atomicOr(&bord[par[sl]], 1u);
      in.run_par[(r0 + y) * RUNS_PER_ROW + k] = r0 * RUNS_PER_ROW + par[sl];
    }
  }
  __syncthreads();
  // compact ids of this slice's roots: the range [z R, z R + R), R = ROOTS_PER_SLICE
  for (int y = threadIdx.x; y < ny; y += blockDim.x) {
    const int n = cnt[y];
    for (int k = 0; k < n; ++k) {
      const int sl = y * RUNS_PER_ROW + k;
      if (par[sl] != sl) continue;
      int loc = atomicAdd(&s_nloc, 1);
      if (loc >= ROOTS_PER_SLICE) continue;
      const int id = z * ROOTS_PER_SLICE + loc;
      const int gs = r0 * RUNS_PER_ROW + sl;
      in.run_flag[gs] = (unsigned)id;
      in.root_info[id] = bord[sl];
      in.root_slot[id] = gs;
    }
  }
  __syncthreads();
  for (int t = s_nloc + threadIdx.x; t < ROOTS_PER_SLICE; t += blockDim.x) in.root_slot[z * ROOTS_PER_SLICE + t] = -1;
  // distinct joins with slice z-1: key = (root slot here, root slot below)
  if (z > 0) {
    for (int y = threadIdx.x; y < ny; y += blockDim.x) {
      const int n = cnt[y], m = cntd[y];
      for (int k = 0; k < n; ++k) {
        const int sl = y * RUNS_PER_ROW + k;
        for (int j = 0; j < m; ++j) {
          const int sd = y * RUNS_PER_ROW + j;
          if (!overlap(xx[sl], xxd[sd])) continue;
          unsigned long long key = ((unsigned long long)(r0 * RUNS_PER_ROW + par[sl]) << 32) |
                                   (unsigned)(rd0 * RUNS_PER_ROW + sd);
          // shared hash set, open addressing, bounded probing
          unsigned h = (unsigned)((key * 0x9E3779B97F4A7C15ull) >> 40) & (HB - 1);
          bool done = false;
          for (int probe = 0; probe < HB && !done; ++probe) {
            unsigned long long old = atomicCAS(&ekeys[h], ~0ull, key);
            done = (old == ~0ull || old == key);
            h = (h + 1) & (HB - 1);
          }
          if (!done) s_full = 1;
        }
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < HB; t += blockDim.x) {
    unsigned long long k = ekeys[t];
    if (k == ~0ull) continue;
    int pos = atomicAdd(&s_ne, 1);
    if (pos < ZEDGE_CAP) {
      in.zedge[z * 2 * ZEDGE_CAP + 2 * pos] = (int)(k >> 32);
      in.zedge[z * 2 * ZEDGE_CAP + 2 * pos + 1] = (int)(k & 0xffffffffu);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_nloc > ROOTS_PER_SLICE) atomicOr(&in.err, (int)ERR_RUNS);
    if (s_full || s_ne > ZEDGE_CAP) {
      atomicOr(&in.err, (int)ERR_RUNS);  // the join degrades the map to NEAR: still exact
      in.zedge_cnt[z] = 0;
    } else {
      in.zedge_cnt[z] = s_ne;
    }
  }
}

// 3. join the slices (one CTA per instance, shared memory over the compact
//    slice roots): components with a border run are outside; the others are
//    numbered (at most MAX_COMP get a winding-number seed); each compact root
//    receives its final label.
__global__ void __launch_bounds__(1024) k_join_cc(Inst* __restrict__ I) {
  __shared__ int par[ROOT_CAP];
  __shared__ unsigned flag[ROOT_CAP];
  __shared__ int eoff[MAX_DIM + 1];
  __shared__ int s_ncomp;
  Inst& in = I[blockIdx.x];
  if (in.err & ERR_DEGENERATE) return;
  const int nz = in.dims[2];
  const int nroots = nz * ROOTS_PER_SLICE;
  if (in.err & ERR_RUNS) {
    // too many slice components for the tables: every undecided cube becomes
    // NEAR (exact: those elements take the exact test)
    const int nx = in.dims[0], nrows = in.dims[1] * nz;
    if (threadIdx.x == 0) { in.err |= ERR_RUNS; in.ncomp = 0; }
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
      in.run_cnt[r] = 0;
      uint8_t* row = in.cube + (long long)r * CUBE_PITCH;
      for (int x = 0; x < nx; ++x) row[x] = CUBE_NEAR;
    }
    return;
  }
  if (threadIdx.x == 0) s_ncomp = 0;
  for (int i = threadIdx.x; i < nroots; i += blockDim.x) {
    par[i] = i;
    // ids a slice did not use are marked outside so they are never numbered
    flag[i] = (in.root_slot[i] < 0 || in.root_info[i]) ? RUN_OUT : 0u;
  }
  // per-slice edge counts (parallel loads), then their prefix from shared memory
  for (int z = threadIdx.x; z < nz; z += blockDim.x) eoff[z + 1] = z ? in.zedge_cnt[z] : 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    eoff[0] = 0;
    for (int z = 1; z <= nz; ++z) eoff[z] += eoff[z - 1];
  }
  __syncthreads();
  // edges of all slices, flattened over the threads
  for (int e = threadIdx.x; e < eoff[nz]; e += blockDim.x) {
    int lo = 0, hi = nz - 1;
    while (lo < hi) { int mid = (lo + hi + 1) >> 1; if (eoff[mid] <= e) lo = mid; else hi = mid - 1; }
    const int z = lo, t = e - eoff[z];
    // a: root slot of the run above; b: slot of the run below, whose slice
    // root the lower slice recorded in run_par
    int a = (int)in.run_flag[in.zedge[z * 2 * ZEDGE_CAP + 2 * t]];
    int b = (int)in.run_flag[in.run_par[in.zedge[z * 2 * ZEDGE_CAP + 2 * t + 1]]];
    uf_union(par, a, b);
  }
  __syncthreads();
  {
    // two-phase compression (ROOT_CAP <= 4 * blockDim)
    static_assert(ROOT_CAP <= 4 * 1024, "four roots per thread");  // 48 x 82 = 3936
    int rr[4];
    for (int m = 0; m < 4; ++m) {
      int i = threadIdx.x + m * blockDim.x;
      rr[m] = i < nroots ? uf_root(par, i) : 0;
    }
    __syncthreads();
    for (int m = 0; m < 4; ++m) {
      int i = threadIdx.x + m * blockDim.x;
      if (i >= nroots) continue;
      par[i] = rr[m];
      if ((flag[i] & RUN_OUT) && !(((volatile unsigned*)flag)[rr[m]] & RUN_OUT)) atomicOr(&flag[rr[m]], RUN_OUT);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nroots; i += blockDim.x) {
    if (par[i] != i || (flag[i] & RUN_OUT)) continue;
    int c = atomicAdd(&s_ncomp, 1);
    if (c < MAX_COMP) {
      flag[i] |= (unsigned)c << 4;
      int gs = in.root_slot[i];
      in.comp_seed[c] = (gs / RUNS_PER_ROW) * CUBE_PITCH + (in.run_xx[gs] & 0xff);
    } else {
      flag[i] |= RUN_UNKNOWN;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nroots; i += blockDim.x) in.root_label[i] = flag[par[i]];
  if (threadIdx.x == 0) in.ncomp = s_ncomp;
}

// 5. cube states of each row from its runs (16-byte stores)
__global__ void k_run_states(Inst* __restrict__ I) {
  Inst& in = I[blockIdx.y];
  if (in.err & ERR_DEGENERATE) return;
  const int nrows = rows_of(in);
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += gridDim.x * blockDim.x) {
    const int n = in.run_cnt[r];
    if (!n) continue;  // all NEAR (or a row made NEAR in step 1)
    unsigned w[CUBE_PITCH / 4];
#pragma unroll
    for (int i = 0; i < CUBE_PITCH / 4; ++i) w[i] = 0x02020202u;
    for (int k = 0; k < n; ++k) {
      int sl = r * RUNS_PER_ROW + k;
      unsigned fl = in.root_label[in.run_flag[in.run_par[sl]]];
      unsigned v = (fl & RUN_OUT) ? CUBE_OUT : ((fl & RUN_UNKNOWN) ? CUBE_NEAR : (CUBE_COMP0 + (fl >> 4)));
      unsigned short xx = in.run_xx[sl];
      int x0 = xx & 0xff, x1 = xx >> 8;
#pragma unroll
      for (int i = 0; i < CUBE_PITCH / 4; ++i) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          int x = 4 * i + b;
          if (x >= x0 && x <= x1) w[i] = (w[i] & ~(0xffu << (8 * b))) | (v << (8 * b));
        }
      }
    }
    uint4* row4 = reinterpret_cast<uint4*>(in.cube + (long long)r * CUBE_PITCH);
#pragma unroll
    for (int i = 0; i < CUBE_PITCH / 16; ++i) row4[i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
  }
}

// winding number of each enclosed component's seed cube centre (FP32 solid
// angles: the centre is >= ds/2 from every surface point, so the sum is far
// from the 1/2 decision level)
__global__ void k_winding(Inst* __restrict__ I) {
  Inst& in = I[blockIdx.z];
  const int k = blockIdx.y;
  if (k >= min(in.ncomp, MAX_COMP) || (in.err & ERR_DEGENERATE)) return;
  const int q = in.q, ntf = 2 * q * q, npf = (q + 1) * (q + 1);
  long long ntri = in.n_faces * ntf;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float om = 0.0f;
  if (t < ntri) {
    int seed = in.comp_seed[k];
    int row = seed / CUBE_PITCH, x = seed % CUBE_PITCH;
    int y = row % in.dims[1], z = row / in.dims[1];
    double P[3] = {in.origin[0] + (x + 0.5) * in.ds, in.origin[1] + (y + 0.5) * in.ds, in.origin[2] + (z + 0.5) * in.ds};
    long long f = t / ntf;
    int tt = (int)(t - f * ntf);
    const double* fn = in.surf + f * npf * 3;
    float v[3][3];
    for (int c = 0; c < 3; ++c) {
      int nd = c_ftri[q - 1][tt][c];
      for (int a = 0; a < 3; ++a) v[c][a] = (float)(fn[3 * nd + a] - P[a]);
    }
    float la = sqrtf(v[0][0] * v[0][0] + v[0][1] * v[0][1] + v[0][2] * v[0][2]);
    float lb = sqrtf(v[1][0] * v[1][0] + v[1][1] * v[1][1] + v[1][2] * v[1][2]);
    float lc = sqrtf(v[2][0] * v[2][0] + v[2][1] * v[2][1] + v[2][2] * v[2][2]);
    float cx = v[1][1] * v[2][2] - v[1][2] * v[2][1];
    float cy = v[1][2] * v[2][0] - v[1][0] * v[2][2];
    float cz = v[1][0] * v[2][1] - v[1][1] * v[2][0];
    float det = v[0][0] * cx + v[0][1] * cy + v[0][2] * cz;
    float ab = v[0][0] * v[1][0] + v[0][1] * v[1][1] + v[0][2] * v[1][2];
    float ac = v[0][0] * v[2][0] + v[0][1] * v[2][1] + v[0][2] * v[2][2];
    float bc = v[1][0] * v[2][0] + v[1][1] * v[2][1] + v[1][2] * v[2][2];
    float den = la * lb * lc + ab * lc + ac * lb + bc * la;
    om = 2.0f * atan2f(det, den);
  }
  for (int s = 16; s; s >>= 1) om += __shfl_xor_sync(0xffffffffu, om, s);
  __shared__ float ws[32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) ws[w] = om;
  __syncthreads();
  if (w == 0) {
    float v = lane < (blockDim.x >> 5) ? ws[lane] : 0.0f;
    for (int s = 16; s; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    if (lane == 0) atomicAdd(&in.comp_w[k], v * (float)(0.25 / 3.14159265358979323846));
  }
}

// ------------------------------------------------------------------ a4: classify + compact
struct CandList {
  unsigned long long* cand;   // (instance << 40) | element
  unsigned long long cap;
  unsigned long long* count;  // [0] candidates, [1] work cursor of the exact kernel
};

__global__ void __launch_bounds__(256) k_classify(Inst* __restrict__ I, const long long* __restrict__ eoff, int n_inst,
                                                  long long ne_total, CandList cl,
                                                  unsigned long long* __restrict__ n_hole_map) {
  const unsigned FULL = 0xffffffffu;
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  bool valid = g < ne_total;
  bool cand = false, hole = false;
  int ii = 0;
  long long e = 0;
  if (valid) {
    ii = find_inst(eoff, n_inst, g);
    Inst& in = I[ii];
    e = g - eoff[ii];
    const float* bb = in.eaabb + 6 * e;
    float2 b01 = *reinterpret_cast<const float2*>(bb);
    float2 b23 = *reinterpret_cast<const float2*>(bb + 2);
    float2 b45 = *reinterpret_cast<const float2*>(bb + 4);
    float lo[3] = {b01.x, b01.y, b23.x}, hi[3] = {b23.y, b45.x, b45.y};
    int8_t flag = DC_FIELD_;
    if (in.err & (ERR_DEGENERATE | ERR_NONFINITE)) {
      // invalid surface: the call reports DC_EINVAL; leave the bins untouched
    } else {
      float inv = (float)(1.0 / in.ds);
      int c0[3], c1[3];
      bool outside = false, partial = false;
      for (int a = 0; a < 3; ++a) {
        float o = (float)in.origin[a];
        float x0 = (lo[a] - o) * inv - 1e-3f, x1 = (hi[a] - o) * inv + 1e-3f;
        int n = in.dims[a];
        int i0 = (x0 > -1.0f) ? (x0 < (float)n ? (int)floorf(x0) : n) : -1;
        int i1 = (x1 > -1.0f) ? (x1 < (float)n ? (int)floorf(x1) : n) : -1;
        if (i1 < 0 || i0 > n - 1) outside = true;
        if (i0 < 0 || i1 > n - 1) partial = true;
        c0[a] = max(i0, 0);
        c1[a] = min(i1, n - 1);
      }
      if (!outside) {
        bool any_in = false, any_out = partial, any_near = false;
        for (int z = c0[2]; z <= c1[2] && !any_near; ++z)
          for (int y = c0[1]; y <= c1[1] && !any_near; ++y) {
            const uint8_t* row = in.cube + ((long long)z * in.dims[1] + y) * CUBE_PITCH;
            for (int x = c0[0]; x <= c1[0]; ++x) {
              uint8_t s = row[x];
              if (s == CUBE_OUT) {
                any_out = true;
              } else if (s >= CUBE_COMP0 && s < CUBE_COMP0 + MAX_COMP) {
                float w = in.comp_w[s - CUBE_COMP0];
                if (w > 0.75f && w < 1.25f) any_in = true;
                else if (w > -0.25f && w < 0.25f) any_out = true;
                else { any_near = true; break; }
              } else {
                any_near = true;
                break;
              }
            }
          }
        if (any_near || (any_in && any_out)) cand = true;
        else flag = any_in ? DC_HOLE_ : DC_FIELD_;
      }
    }
    if (!cand) {
      hole = flag == DC_HOLE_;
      in.flags[e] = flag;
      if (in.dist) in.dist[e] = (flag == DC_HOLE_) ? -HUGE_VAL : HUGE_VAL;
    }
  }
  const unsigned hm = __ballot_sync(FULL, hole);
  if (hm && (threadIdx.x & 31) == 0) atomicAdd(n_hole_map, (unsigned long long)__popc(hm));
  unsigned m = __ballot_sync(FULL, cand);
  if (m) {
    int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&cl.count[0], (unsigned long long)__popc(m));
    base = __shfl_sync(FULL, base, 0);
    if (cand) {
      unsigned long long pos = base + __popc(m & ((1u << lane) - 1u));
      if (pos < cl.cap) cl.cand[pos] = ((unsigned long long)ii << 40) | (unsigned long long)e;
    }
  }
}

}  // namespace dc
