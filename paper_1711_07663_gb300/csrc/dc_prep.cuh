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

// a3: NEAR tags of the hole map, and face -> bin (bin of the box's min corner)
__global__ void k_tag(Inst* __restrict__ I, const long long* __restrict__ foff, int n_inst, long long nf_total) {
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nf_total) return;
  int ii = find_inst(foff, n_inst, g);
  Inst& in = I[ii];
  if (in.err & ERR_DEGENERATE) return;
  long long f = g - foff[ii];
  const double ds = in.ds;
  const double mu = 2.0 * in.tol + 1e-9 * ds;  // fringe margin, with room for rounding
  int c0[3], c1[3], b[3];
  for (int a = 0; a < 3; ++a) {
    double lo = in.fbox64[6 * f + a], hi = in.fbox64[6 * f + 3 + a];
    c0[a] = max(cube_floor((lo - mu - in.origin[a]) / ds - 1e-6, in.dims[a]), 0);
    c1[a] = min(cube_floor((hi + mu - in.origin[a]) / ds + 1e-6, in.dims[a]), in.dims[a] - 1);
    b[a] = clampi(cube_floor((lo - in.origin[a]) / in.bs, in.bdims[a]), 0, in.bdims[a] - 1);
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
// Run descriptor: x1 bits 0-6, x0 bits 7-13, row bits 14-26; flags in 27-31.
constexpr unsigned RUN_OUT = 1u << 31, RUN_UNKNOWN = 1u << 30;
__device__ __forceinline__ unsigned run_x1(unsigned d) { return d & 127u; }
__device__ __forceinline__ unsigned run_x0(unsigned d) { return (d >> 7) & 127u; }
__device__ __forceinline__ unsigned run_row(unsigned d) { return (d >> 14) & 8191u; }
__device__ __forceinline__ unsigned run_comp(unsigned d) { return (d >> 27) & 7u; }

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

__device__ __forceinline__ bool mbit(unsigned long long m0, unsigned long long m1, int x) {
  return x < 64 ? ((m0 >> x) & 1ull) : ((m1 >> (x - 64)) & 1ull);
}

__device__ int uf_find(volatile int* parent, int i) {
  // path halving; parents always point to smaller indices, so this terminates
  int p = parent[i];
  while (p != i) {
    int gp = parent[p];
    if (gp != p) parent[i] = gp;
    i = p;
    p = parent[i];
  }
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

// One CTA per instance.  Dynamic shared memory: row offsets, run descriptors
// and union-find parents for up to `cap` runs.
__global__ void __launch_bounds__(1024) k_holemap_cc(Inst* __restrict__ I, int cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_total, s_ncomp;
  Inst& in = I[blockIdx.x];
  if (in.err & ERR_DEGENERATE) return;
  const int nx = in.dims[0], ny = in.dims[1], nz = in.dims[2];
  const int nrows = ny * nz;
  int* row_off = reinterpret_cast<int*>(smem);
  unsigned* desc = reinterpret_cast<unsigned*>(row_off + MAX_DIM * MAX_DIM + 1);
  volatile int* parent = reinterpret_cast<volatile int*>(desc + cap);
  const int tid = threadIdx.x, T = blockDim.x;

  // 1. runs per row
  for (int r = tid; r < nrows; r += T) {
    unsigned long long m0, m1;
    row_mask(in.cube + (long long)r * CUBE_PITCH, nx, m0, m1);
    unsigned long long s0 = m0 & ~(m0 << 1);
    unsigned long long s1 = m1 & ~((m1 << 1) | (m0 >> 63));
    row_off[r] = __popcll(s0) + __popcll(s1);
  }
  __syncthreads();
  // 2. exclusive scan of row counts (chunked; T threads)
  {
    int chunk = (nrows + T - 1) / T;
    int r0 = min(tid * chunk, nrows), r1 = min(r0 + chunk, nrows);
    int s = 0;
    for (int r = r0; r < r1; ++r) s += row_off[r];
    // block scan of s via warp shuffles
    __shared__ int wsum[32];
    int lane = tid & 31, w = tid >> 5;
    int v = s;
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane == 31) wsum[w] = v;
    __syncthreads();
    if (w == 0) {
      int x = (lane < (T >> 5)) ? wsum[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
      }
      wsum[lane] = x;
    }
    __syncthreads();
    int excl = v - s + (w ? wsum[w - 1] : 0);
    __syncthreads();
    int run = excl;
    for (int r = r0; r < r1; ++r) {
      int c = row_off[r];
      row_off[r] = run;
      run += c;
    }
    if (tid == T - 1) { row_off[nrows] = run; s_total = run; s_ncomp = 0; }
  }
  __syncthreads();
  const int R = s_total;
  if (R > cap) {
    // Too many runs for the table: degrade every undecided cube to NEAR.
    // The classification stays exact (those elements take the exact test).
    if (tid == 0) { in.err |= ERR_RUNS; in.ncomp = 0; }
    for (int r = tid; r < nrows; r += T) {
      uint8_t* row = in.cube + (long long)r * CUBE_PITCH;
      for (int x = 0; x < nx; ++x) row[x] = CUBE_NEAR;
    }
    return;
  }
  // 3. run table
  for (int r = tid; r < nrows; r += T) {
    unsigned long long m0, m1;
    row_mask(in.cube + (long long)r * CUBE_PITCH, nx, m0, m1);
    int k = row_off[r];
    int x = 0;
    while (x < nx) {
      if (!mbit(m0, m1, x)) { ++x; continue; }
      int x0 = x;
      while (x < nx && mbit(m0, m1, x)) ++x;
      desc[k] = ((unsigned)r << 14) | ((unsigned)x0 << 7) | (unsigned)(x - 1);
      parent[k] = k;
      ++k;
    }
  }
  __syncthreads();
  // 4. union face-adjacent runs (rows y+1 and z+1)
  for (int i = tid; i < R; i += T) {
    unsigned d = desc[i];
    int r = run_row(d), x0 = run_x0(d), x1 = run_x1(d);
    int y = r % ny, z = r / ny;
    int nbr[2] = {(y + 1 < ny) ? r + 1 : -1, (z + 1 < nz) ? r + ny : -1};
    for (int t = 0; t < 2; ++t) {
      if (nbr[t] < 0) continue;
      for (int j = row_off[nbr[t]]; j < row_off[nbr[t] + 1]; ++j) {
        unsigned e = desc[j];
        if ((int)run_x0(e) <= x1 && (int)run_x1(e) >= x0) uf_union(parent, i, j);
      }
    }
  }
  __syncthreads();
  // 5. compress; components that touch the map border are outside
  for (int i = tid; i < R; i += T) {
    int root = uf_find(parent, i);
    parent[i] = root;
    unsigned d = desc[i];
    int r = run_row(d), y = r % ny, z = r / ny;
    bool border = run_x0(d) == 0 || (int)run_x1(d) == nx - 1 || y == 0 || y == ny - 1 || z == 0 || z == nz - 1;
    // test first: the border runs all share one root, and serialised atomics
    // on a single shared-memory word would dominate the kernel
    if (border && !(((volatile unsigned*)desc)[root] & RUN_OUT)) atomicOr(&desc[root], RUN_OUT);
  }
  __syncthreads();
  // 6. number the enclosed components
  for (int i = tid; i < R; i += T) {
    if (parent[i] == i && !(desc[i] & RUN_OUT)) {
      int k = atomicAdd(&s_ncomp, 1);
      if (k < MAX_COMP) {
        atomicOr(&desc[i], (unsigned)k << 27);
        unsigned d = desc[i];
        in.comp_seed[k] = (int)(run_row(d) * CUBE_PITCH + run_x0(d));
        in.comp_w[k] = 0.0f;
      } else {
        atomicOr(&desc[i], RUN_UNKNOWN);
      }
    }
  }
  __syncthreads();
  // 7. write the states
  for (int i = tid; i < R; i += T) {
    unsigned d = desc[i];
    unsigned rd = desc[parent[i]];
    uint8_t st = (rd & RUN_OUT) ? CUBE_OUT : ((rd & RUN_UNKNOWN) ? CUBE_NEAR : (uint8_t)(CUBE_COMP0 + run_comp(rd)));
    uint8_t* row = in.cube + (long long)run_row(d) * CUBE_PITCH;
    for (int x = run_x0(d); x <= (int)run_x1(d); ++x) row[x] = st;
  }
  if (tid == 0) in.ncomp = min(s_ncomp, MAX_COMP);
}

// winding number of each enclosed component's seed cube centre (FP32 solid
// angles: the centre is >= ds/2 from every surface point, so the sum is far
// from the 1/2 decision level)
__global__ void k_winding(Inst* __restrict__ I) {
  Inst& in = I[blockIdx.z];
  const int k = blockIdx.y;
  if (k >= in.ncomp || (in.err & ERR_DEGENERATE)) return;
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
                                                  long long ne_total, CandList cl) {
  const unsigned FULL = 0xffffffffu;
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  bool valid = g < ne_total;
  bool cand = false;
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
      in.flags[e] = flag;
      if (in.dist) in.dist[e] = (flag == DC_HOLE_) ? -HUGE_VAL : HUGE_VAL;
    }
  }
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
