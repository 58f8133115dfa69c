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
#include "dc_frames.cuh"

namespace dc {

__constant__ unsigned char c_etri[MAX_P][MAX_NTE][3];   // element boundary triangles, per p
__constant__ unsigned char c_ftri[MAX_Q][MAX_NTF][3];   // cut-face triangles, per q

constexpr int CUBE_PITCH = 96;  // bytes per x-row of the hole map (>= MAX_DIM, 16-byte multiple)

// ------------------------------------------------------------------ a1 + a2
constexpr int SURF_FPB = 16;  // faces per block of k_surface (a tile of the fused prep kernel)

// hole-map and bin geometry of one instance from its surface box.  Any cube
// size serves (every consumer rounds outward and reads the one stored value),
// so it is derived in FP32, where this GPU's FP64 pipe would take
// microseconds of one thread's time: ds is a float (exact in FP64), the cube
// counts cover the box with a padding cube on each side (an underestimate of
// one cube from rounding is within that padding).
__device__ void grid_from_box(Inst& in) {
  double lo[3], hi[3];
  float span[3], L = 0.f;
  for (int a = 0; a < 3; ++a) {
    lo[a] = dkey_decode(atomicOr(&in.sbox_key[a], 0ull));
    hi[a] = dkey_decode(atomicOr(&in.sbox_key[3 + a], 0ull));
    span[a] = __double2float_ru(hi[a] - lo[a]);
    L = fmaxf(L, span[a]);
  }
  if (!(L > 0.f) || !(L < 1e30f)) {
    atomicOr(&in.err, (int)ERR_DEGENERATE);
    L = 1.f;
  }
  // cubes on the longest side: as configured, or cubes_per_edge (1.8 unless
  // tuned) per element edge (a map much finer than the elements only
  // multiplies the cubes each element and face covers; a coarser one widens
  // the band of candidates)
  int cells = in.holemap_cells;
  if (cells <= 0) {
    const float a = in.h_elem > 0.f ? in.cubes_per_edge * L / in.h_elem : 64.f;
    cells = (int)fminf(fmaxf(a + 0.5f, 16.f), (float)MAX_CELLS);
  }
  const float ds_f = L / (float)cells;
  const float inv_ds = 1.0f / ds_f;
  const double ds = (double)ds_f;
  in.ds = ds;
  int nb = 1;
  for (int a = 0; a < 3; ++a) {
    const float cf = fminf(fmaxf(span[a], 0.f) * inv_ds, (float)cells);
    const int n = clampi((int)ceilf(cf), 1, cells);
    in.dims[a] = n + 2;
    in.origin[a] = lo[a] - ds;
    in.bdims[a] = (in.dims[a] + in.bin_cubes - 1) / in.bin_cubes;
    nb *= in.bdims[a];
  }
  in.bs = ds * in.bin_cubes;
  for (int a = 0; a < 3; ++a) in.origin_f[a] = (float)in.origin[a];
  in.inv_ds_f = inv_ds;
  in.inv_bs_f = 1.0f / (ds_f * (float)in.bin_cubes);
  if (nb > in.nbins_cap) atomicOr(&in.err, (int)ERR_DEGENERATE);  // sized on the host for the worst case
}

// Pose transform (rounded exactly as ((R0 x + R1 y) + R2 z) + t, no fusion),
// per-face node boxes, surface box and largest face extent.  Grid (blocks of
// SURF_FPB faces, instances): threads transform nodes, then one thread per
// (face, axis) takes the face's box from shared memory; the last block of an
// instance to finish derives its hole-map grid.
// SURF_FPB faces of instance `in` from face f0 (one block): pose, face boxes,
// and the block's share of the surface box and face extents.  With
// derive_grid, the last block of the instance to finish derives its hole-map
// grid (the fused prep kernel derives it after a grid barrier instead).
__device__ void surface_tile(Inst& in, long long f0, bool derive_grid) {
  __shared__ double s_x[SURF_FPB * MAX_NPF * 3];
  __shared__ unsigned long long s_key[6];
  __shared__ unsigned s_ext[3];
  __shared__ int s_last;
  const long long F = in.n_faces;
  const int nf = (int)min((long long)SURF_FPB, F - f0);
  const int npf = (in.q + 1) * (in.q + 1);
  const int nval = nf * npf * 3;
  if (threadIdx.x < 6) s_key[threadIdx.x] = threadIdx.x < 3 ? ~0ull : 0ull;
  if (threadIdx.x < 3) s_ext[threadIdx.x] = 0u;
  const double* src = in.faces_in + f0 * npf * 3;
  double* dst = in.surf + f0 * npf * 3;
  // |v| >= 1e300 or not finite, tested on the bit pattern (integer words, no
  // FP64 arithmetic: the FP64 pipe of this GPU is slow)
  const int bigh = (int)(__double_as_longlong(1e300) >> 32);
  const unsigned bigl = (unsigned)__double_as_longlong(1e300);
  auto huge = [&](double v) {
    const long long b = __double_as_longlong(v);
    const int mh = (int)(b >> 32) & 0x7fffffff;
    return mh > bigh || (mh == bigh && (unsigned)b >= bigl);
  };
  bool bad = false;
  if (in.has_pose) {
    for (int k = threadIdx.x; k < nf * npf; k += blockDim.x) {
      const double x = src[3 * k], y = src[3 * k + 1], z = src[3 * k + 2];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double* R = in.pose + 4 * a;
        const double v = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(R[0], x), __dmul_rn(R[1], y)), __dmul_rn(R[2], z)), R[3]);
        s_x[3 * k + a] = v;
        dst[3 * k + a] = v;
        bad |= huge(v);
      }
    }
  } else {
    for (int k = threadIdx.x; k < nval; k += blockDim.x) {
      const double v = src[k];
      s_x[k] = v;
      dst[k] = v;
      bad |= huge(v);
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&in.err, (int)ERR_NONFINITE);
  // face boxes: thread (face, axis), on the order-preserving integer keys of
  // the coordinates (all finite here, or the cut is rejected)
  if (threadIdx.x < nf * 3) {
    const int lf = threadIdx.x / 3, a = threadIdx.x - lf * 3;
    FbKey klo{INT_MAX, 0xffffffffu}, khi{INT_MIN, 0u};
    for (int k = 0; k < npf; ++k) {
      const FbKey q = fb_key(__double_as_longlong(s_x[(lf * npf + k) * 3 + a]));
      if (fb_less(q, klo)) klo = q;
      if (fb_less(khi, q)) khi = q;
    }
    const double lo = fb_value(klo), hi = fb_value(khi);
    const long long f = f0 + lf;
    in.fbox[6 * f + a] = __double2float_rd(lo);
    in.fbox[6 * f + 3 + a] = __double2float_ru(hi);
    atomicMin(&s_key[a], dkey(lo));
    atomicMax(&s_key[3 + a], dkey(hi));
    atomicMax(&s_ext[a], __float_as_uint(__double2float_ru(hi - lo) * 1.000001f));
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    atomicMin(&in.sbox_key[threadIdx.x], s_key[threadIdx.x]);
    atomicMax(&in.sbox_key[3 + threadIdx.x], s_key[3 + threadIdx.x]);
    atomicMax(&in.fext_bits[threadIdx.x], s_ext[threadIdx.x]);
  }
  if (derive_grid) {
    // the last block of this instance derives the grid
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned nblk = (unsigned)((F + SURF_FPB - 1) / SURF_FPB);
      s_last = atomicAdd(&in.surf_done, 1u) == nblk - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
      __threadfence();
      grid_from_box(in);
    }
  }
  __syncthreads();  // the shared arrays may be reused by the next tile
}

// Pose transform (rounded exactly as ((R0 x + R1 y) + R2 z) + t, no fusion),
// per-face node boxes, surface box and largest face extent.  Grid (blocks of
// SURF_FPB faces, instances): threads transform nodes, then one thread per
// (face, axis) takes the face's box from shared memory; the last block of an
// instance to finish derives its hole-map grid.
__global__ void __launch_bounds__(256) k_surface(Inst* __restrict__ I) {
  pdl_enter();
  Inst& in = I[blockIdx.y];
  const long long f0 = (long long)blockIdx.x * SURF_FPB;
  if (f0 >= in.n_faces) return;
  surface_tile(in, f0, true);
}

// zero the hole map, the bin counts and the row counters of one instance;
// thread `t` of `nt` takes every nt-th word
__device__ void clear_inst(Inst& in, long long t, long long nt) {
  long long ncube = (long long)in.dims[1] * in.dims[2] * CUBE_PITCH;
  int nb = in.bdims[0] * in.bdims[1] * in.bdims[2];
  if (nb > in.nbins_cap) nb = 0;
  uint4* c4 = reinterpret_cast<uint4*>(in.cube);
  long long n4 = ncube / 16;
  for (long long k = t; k < n4; k += nt) c4[k] = make_uint4(0, 0, 0, 0);
  for (long long k = t; k < nb; k += nt) in.bin_cnt[k] = 0;
  const int nrows = in.dims[1] * in.dims[2];
  for (long long k = t; k < nrows; k += nt) in.row_cnt[k] = 0;
}

// the same over the map's, bins' and rows' full capacity (the grid not yet known)
__device__ void clear_inst_cap(Inst& in, long long t, long long nt) {
  uint4* c4 = reinterpret_cast<uint4*>(in.cube);
  const long long n4 = (long long)MAX_DIM * MAX_DIM * CUBE_PITCH / 16;
  for (long long k = t; k < n4; k += nt) c4[k] = make_uint4(0, 0, 0, 0);
  for (long long k = t; k < in.nbins_cap; k += nt) in.bin_cnt[k] = 0;
  for (long long k = t; k < (long long)MAX_DIM * MAX_DIM; k += nt) in.row_cnt[k] = 0;
}

__global__ void k_clear(Inst* __restrict__ I) {
  pdl_enter();
  clear_inst(I[blockIdx.y], (long long)blockIdx.x * blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
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

// a3: NEAR tags of the hole map, and face -> bin (bin of the box's min
// corner).  TAG_R threads share a face: thread r tags the face's cube rows r,
// r + TAG_R, ... (a face box spans a few rows of a few cubes each), and thread
// 0 also files the face in its bin.  g numbers (face, r) pairs over all
// instances.
constexpr int TAG_R = 8;
__device__ void tag_face(Inst* __restrict__ I, const long long* __restrict__ foff, int n_inst, long long nf_total,
                         long long g) {
  const long long gf = g / TAG_R;
  const int r = (int)(g - gf * TAG_R);
  if (gf >= nf_total) return;
  int ii = find_inst(foff, n_inst, gf);
  Inst& in = I[ii];
  if (in.err & ERR_DEGENERATE) return;
  long long f = gf - foff[ii];
  // cube range of the face box inflated by the fringe margin 2 tol, in float:
  // the extra 1e-3 cube (plus 16 ulp of the coordinates) only ever adds cubes
  const float mu = (float)(2.0 * in.tol);
  int c0[3], c1[3], b[3];
  for (int a = 0; a < 3; ++a) {
    float lo = in.fbox[6 * f + a], hi = in.fbox[6 * f + 3 + a];  // rounded outward
    float o = in.origin_f[a];
    float slack = 1e-3f + 16.0f * 5.9604645e-8f * (fabsf(lo) + fabsf(hi) + fabsf(o)) * in.inv_ds_f;
    float x0 = (lo - mu - o) * in.inv_ds_f - slack, x1 = (hi + mu - o) * in.inv_ds_f + slack;
    c0[a] = max(cube_floorf(x0, in.dims[a]), 0);
    c1[a] = min(cube_floorf(x1, in.dims[a]), in.dims[a] - 1);
    b[a] = clampi(cube_floorf((lo - o) * in.inv_bs_f, in.bdims[a]), 0, in.bdims[a] - 1);
  }
  const int ny = c1[1] - c0[1] + 1, nz = c1[2] - c0[2] + 1;
  if (ny > 0 && nz > 0 && c1[0] >= c0[0])
    for (int k = r; k < ny * nz; k += TAG_R) {
      const int z = c0[2] + k / ny, y = c0[1] + k % ny;
      uint8_t* row = in.cube + ((long long)z * in.dims[1] + y) * CUBE_PITCH;
      for (int x = c0[0]; x <= c1[0]; ++x) row[x] = CUBE_NEAR;
    }
  if (r == 0) {
    int bi = (b[2] * in.bdims[1] + b[1]) * in.bdims[0] + b[0];
    in.fbin[f] = bi;
    atomicAdd(&in.bin_cnt[bi], 1);
  }
}

// grid: nf_total * TAG_R threads
__global__ void k_tag(Inst* __restrict__ I, const long long* __restrict__ foff, int n_inst, long long nf_total) {
  pdl_enter();
  tag_face(I, foff, n_inst, nf_total, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// exclusive scan of the bin counts (one block per instance; 256 threads in
// the fused prep kernel, 1024 in k_bin_scan), in passes of BIN_PER_T x 32
// bins per warp: lane l of warp w holds bins base + 32 j + l (j < BIN_PER_T,
// so every load and store of a warp is one contiguous span), the warp scans
// each row of 32 with shuffles, the block scans the warp totals, and a carry
// runs over the passes; counts become cursors (zero) as their offsets are
// written
constexpr int BIN_PER_T = 16;
__device__ void bin_scan_inst(Inst& in) {
  __shared__ int wsum[32];
  const int nb = in.bdims[0] * in.bdims[1] * in.bdims[2];
  if ((in.err & ERR_DEGENERATE) || nb > in.nbins_cap) return;
  const unsigned FULL = 0xffffffffu;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
  const int per_warp = 32 * BIN_PER_T;
  int carry = 0;
  for (int base = 0; base < nb; base += nw * per_warp) {
    const int wb = base + wid * per_warp;
    int v[BIN_PER_T];
#pragma unroll
    for (int j = 0; j < BIN_PER_T; ++j) {
      const int idx = wb + 32 * j + lane;
      v[j] = idx < nb ? in.bin_cnt[idx] : 0;
    }
    int wrun = 0;  // the warp's running total before row j
#pragma unroll
    for (int j = 0; j < BIN_PER_T; ++j) {
      int x = v[j];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(FULL, x, d);
        if (lane >= d) x += y;
      }
      const int row_total = __shfl_sync(FULL, x, 31);
      v[j] = wrun + x - v[j];  // exclusive offset within the warp's span
      wrun += row_total;
    }
    if (lane == 0) wsum[wid] = wrun;
    __syncthreads();
    if (wid == 0) {
      int y = lane < nw ? wsum[lane] : 0;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int z = __shfl_up_sync(FULL, y, d);
        if (lane >= d) y += z;
      }
      wsum[lane] = y;  // inclusive over warps
    }
    __syncthreads();
    const int off = carry + (wid > 0 ? wsum[wid - 1] : 0);
#pragma unroll
    for (int j = 0; j < BIN_PER_T; ++j) {
      const int idx = wb + 32 * j + lane;
      if (idx < nb) {
        in.bin_off[idx] = off + v[j];
        in.bin_cnt[idx] = 0;
      }
    }
    carry += wsum[nw - 1];
    __syncthreads();  // wsum is rewritten by the next pass (or instance)
  }
  if (t == 0) in.bin_off[nb] = carry;
}

__global__ void __launch_bounds__(1024) k_bin_scan(Inst* __restrict__ I) {
  pdl_enter();
  bin_scan_inst(I[blockIdx.x]);
}

__device__ __forceinline__ void bin_fill(Inst* __restrict__ I, const long long* __restrict__ foff, int n_inst,
                                         long long nf_total, long long g) {
  if (g >= nf_total) return;
  int ii = find_inst(foff, n_inst, g);
  Inst& in = I[ii];
  if (in.err & ERR_DEGENERATE) return;
  long long f = g - foff[ii];
  int b = in.fbin[f];
  int pos = in.bin_off[b] + atomicAdd(&in.bin_cnt[b], 1);
  in.bin_faces[pos] = (int)f;
  // the box beside the id: a search over a bin reads both at once
#pragma unroll
  for (int a = 0; a < 6; ++a) in.bin_fbox[6 * (long long)pos + a] = in.fbox[6 * f + a];
}

// ------------------------------------------------------------------ a3: inside / outside
// Every cube that no inflated face box touches lies wholly on one side of the
// closed surface.  Its side is read off the winding number at the centre line
// of its x-row (y, z fixed at the row's cube centres): starting at 0 in the
// padding cube, the winding number changes by -1 at each surface triangle the
// line leaves the body through (normal x component > 0) and +1 at each it
// enters through, and those crossings lie in NEAR cubes.  The paper fills the
// non-NEAR cubes from the map's border instead; for a closed surface the two
// agree wherever the fill reaches, and the winding number also settles
// cavities the fill cannot reach.
//
// Whether the line at p = (y_c, z_c) meets triangle ABC is decided by the
// exact signs of the edge functions E(U->V; p) = (V_y - U_y)(p_z - U_z) -
// (V_z - U_z)(p_y - U_y) of the FP64 vertices: a float evaluation with an
// error bound first, then an FP64 one with the static bound of Shewchuk's
// orientation test, then the exact value as a floating-point expansion
// (error-free sums and FMA products).  An exact zero is resolved by simulation
// of simplicity, moving p to (p_y + e, p_z + e^2) for an infinitesimal e, so
// that every crossing of the watertight triangulated surface is counted
// exactly once.

// Knuth's two-sum and the FMA two-product: s + e equals the exact result
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  const double bv = __dsub_rn(s, a), av = __dsub_rn(s, bv);
  e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
}
__device__ __forceinline__ void two_prod(double a, double b, double& p, double& e) {
  p = __dmul_rn(a, b);
  e = __fma_rn(a, b, -p);
}

// Exact sign of (Qy - Py)(pz - Pz) - (Qz - Pz)(py - Py) (products of exact
// two-term differences, summed into a nonoverlapping expansion; exact unless
// a product underflows), then the simulation-of-simplicity terms for a zero.
__device__ __noinline__ int edge_sign_exact(const double* P, const double* Q, double py, double pz) {
  double a[2], b[2], c[2], d[2];
  two_sum(Q[1], -P[1], a[1], a[0]);
  two_sum(pz, -P[2], b[1], b[0]);
  two_sum(Q[2], -P[2], c[1], c[0]);
  two_sum(py, -P[1], d[1], d[0]);
  double h[17];
  int m = 0;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j)
      for (int k = 0; k < 2; ++k) {
        double t[2];
        if (k == 0) two_prod(a[i], b[j], t[0], t[1]);
        else { two_prod(c[i], d[j], t[0], t[1]); t[0] = -t[0]; t[1] = -t[1]; }
        for (int r = 0; r < 2; ++r) {
          // grow the expansion h by t[r]
          double qv = t[r];
          int w = 0;
          for (int u = 0; u < m; ++u) {
            double sum, err;
            two_sum(qv, h[u], sum, err);
            if (err != 0.0) h[w++] = err;
            qv = sum;
          }
          if (qv != 0.0 || w == 0) h[w++] = qv;
          m = w;
        }
      }
  for (int u = m - 1; u >= 0; --u)
    if (h[u] != 0.0) return h[u] > 0.0 ? 1 : -1;
  // exactly zero: the sign at (py + e, pz + e^2)
  if (Q[2] != P[2]) return Q[2] < P[2] ? 1 : -1;
  if (Q[1] != P[1]) return Q[1] > P[1] ? 1 : -1;
  return 0;  // the edge projects to a point
}

// exact sign of E(U->V; p): the FP64 static filter, else the expansion; both
// from the lexicographically smaller end, so that the two orientations of an
// edge give opposite signs
__device__ __forceinline__ int edge_sign(const double* U, const double* V, double py, double pz) {
  const bool uv = U[1] < V[1] || (U[1] == V[1] && (U[2] < V[2] || (U[2] == V[2] && U[0] < V[0])));
  const double* P = uv ? U : V;
  const double* Q = uv ? V : U;
  const double t1 = __dmul_rn(__dsub_rn(Q[1], P[1]), __dsub_rn(pz, P[2]));
  const double t2 = __dmul_rn(__dsub_rn(Q[2], P[2]), __dsub_rn(py, P[1]));
  const double bound = 4.0 * 1.1102230246251565e-16 * (fabs(t1) + fabs(t2));
  const double e = __dsub_rn(t1, t2);
  int sg = e > bound ? 1 : (e < -bound ? -1 : edge_sign_exact(P, Q, py, pz));
  return uv ? sg : -sg;
}

constexpr int ROW_UNDECIDED = 1 << 20;  // added to a row's crossing count when its list is full

// one thread per surface triangle: its crossings with the row centre lines
__device__ __forceinline__ void row_cross(Inst& in, long long g) {
  if (in.err & (ERR_DEGENERATE | ERR_NONFINITE)) return;
  const int q = in.q, npf = (q + 1) * (q + 1), ntf = 2 * q * q;
  const long long f = g / ntf;
  if (f >= in.n_faces) return;
  const int t = (int)(g - f * ntf);
  const double* fn = in.surf + f * npf * 3;
  const double* A = fn + 3 * c_ftri[q - 1][t][0];
  const double* B = fn + 3 * c_ftri[q - 1][t][1];
  const double* C = fn + 3 * c_ftri[q - 1][t][2];
  const double ds = in.ds, oy = in.origin[1], oz = in.origin[2];
  // float coordinates relative to A (each within u of its FP64 value)
  const float by = (float)(B[1] - A[1]), bz = (float)(B[2] - A[2]), bx = (float)(B[0] - A[0]);
  const float cy = (float)(C[1] - A[1]), cz = (float)(C[2] - A[2]), cx = (float)(C[0] - A[0]);
  const float ay0 = (float)(A[1] - oy), az0 = (float)(A[2] - oz), ax0 = (float)(A[0] - in.origin[0]);
  const float inv = in.inv_ds_f;
  // rows whose centre may lie over the triangle's box: the float box and the
  // scaling are within 4u (map extent) < 1e-4 cube of exact
  const float ylo = ay0 + fminf(0.f, fminf(by, cy)), yhi = ay0 + fmaxf(0.f, fmaxf(by, cy));
  const float zlo = az0 + fminf(0.f, fminf(bz, cz)), zhi = az0 + fmaxf(0.f, fmaxf(bz, cz));
  const int y0 = max((int)ceilf(ylo * inv - 0.5f - 1e-4f), 0), y1 = min((int)floorf(yhi * inv - 0.5f + 1e-4f), in.dims[1] - 1);
  const int z0 = max((int)ceilf(zlo * inv - 0.5f - 1e-4f), 0), z1 = min((int)floorf(zhi * inv - 0.5f + 1e-4f), in.dims[2] - 1);
  const float u = 5.9604644775390625e-8f;
  for (int kz = z0; kz <= z1; ++kz) {
    const double pz = oz + ((double)kz + 0.5) * ds;
    const float qz = (float)(pz - A[2]);
    for (int ky = y0; ky <= y1; ++ky) {
      const double py = oy + ((double)ky + 0.5) * ds;
      const float qy = (float)(py - A[1]);
      // float edge functions relative to A; each input is within u M of the
      // exact difference, so |E_float - E| <= 64 u M^2
      const float eab = by * qz - bz * qy;
      const float ebc = (cy - by) * (qz - bz) - (cz - bz) * (qy - by);
      const float eca = cz * qy - cy * qz;
      const float M = fmaxf(fmaxf(fmaxf(fabsf(by), fabsf(bz)), fmaxf(fabsf(cy), fabsf(cz))), fmaxf(fabsf(qy), fabsf(qz)));
      const float bnd = 64.0f * u * M * M;
      int sab = eab > bnd ? 1 : (eab < -bnd ? -1 : 2);
      int sbc = ebc > bnd ? 1 : (ebc < -bnd ? -1 : 2);
      int sca = eca > bnd ? 1 : (eca < -bnd ? -1 : 2);
      if ((sab == 1 || sbc == 1 || sca == 1) && (sab == -1 || sbc == -1 || sca == -1)) continue;  // outside
      if (sab == 2) sab = edge_sign(A, B, py, pz);
      if (sbc == 2) sbc = edge_sign(B, C, py, pz);
      if (sca == 2) sca = edge_sign(C, A, py, pz);
      if (sab == 0 || sab != sbc || sbc != sca) continue;
      // crossing: x from the barycentric weights (clamped: a point of the
      // triangle, so inside its face box and a NEAR cube)
      const float s = (float)sab;
      const float wa = fmaxf(s * ebc, 0.f), wb = fmaxf(s * eca, 0.f), wc = fmaxf(s * eab, 0.f);
      const float wsum = wa + wb + wc;
      const float xr = wsum > 0.f ? (wb * bx + wc * cx) / wsum : 0.f;
      const int xc = clampi((int)floorf((ax0 + xr) * inv), 0, in.dims[0] - 1);
      int* cnt = in.row_cnt + (kz * in.dims[1] + ky);
      const int pos_k = atomicAdd(cnt, 1);
      // all edge functions positive: the normal has x component > 0 and the
      // line leaves the body here (-1); negative: it enters (+1)
      if (pos_k < ROW_XCAP) in.row_x[(kz * in.dims[1] + ky) * ROW_XCAP + pos_k] = (xc << 1) | (sab > 0 ? 0 : 1);
      else if (pos_k == ROW_XCAP) atomicAdd(cnt, ROW_UNDECIDED);
    }
  }
}

// face -> bin fill (blocks [0, fill_blocks), one thread per face over all
// instances) and row crossings (the other blocks, one thread per triangle of
// instance blockIdx.y): both read only what the earlier kernels wrote
__global__ void __launch_bounds__(256) k_fill_cross(Inst* __restrict__ I, const long long* __restrict__ foff,
                                                    int n_inst, long long nf_total, int fill_blocks) {
  pdl_enter();
  if ((int)blockIdx.x < fill_blocks) {
    if (blockIdx.y == 0) bin_fill(I, foff, n_inst, nf_total, (long long)blockIdx.x * blockDim.x + threadIdx.x);
    return;
  }
  row_cross(I[blockIdx.y], (long long)(blockIdx.x - fill_blocks) * blockDim.x + threadIdx.x);
}

// one warp per row: winding number of each cube that is not NEAR
__device__ void row_label(Inst& in, int r, int lane) {
  if (in.err & (ERR_DEGENERATE | ERR_NONFINITE)) return;
  const int nrows = in.dims[1] * in.dims[2];
  if (r >= nrows) return;
  const int cnt = in.row_cnt[r];
  const bool undecided = cnt > ROW_XCAP;
  if (undecided && lane == 0) atomicAdd(&in.rows_undecided, 1);
  const int x0 = 4 * lane;
  if (x0 >= in.dims[0]) return;
  unsigned* word = reinterpret_cast<unsigned*>(in.cube + (long long)r * CUBE_PITCH + x0);
  unsigned v = *word;
  const int* xs = in.row_x + (long long)r * ROW_XCAP;
  int w[4] = {0, 0, 0, 0};
  if (!undecided)
    for (int i = 0; i < cnt; ++i) {
      const int e = xs[i], xc = e >> 1, d = (e & 1) ? 1 : -1;
#pragma unroll
      for (int k = 0; k < 4; ++k) w[k] += xc < x0 + k ? d : 0;
    }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (x0 + k >= in.dims[0]) break;
    const unsigned b = (v >> (8 * k)) & 0xffu;
    if (b == CUBE_NEAR) continue;
    const unsigned st = undecided ? CUBE_NEAR : (w[k] == 0 ? CUBE_OUT : (w[k] == 1 ? CUBE_IN : CUBE_NEAR));
    v = (v & ~(0xffu << (8 * k))) | (st << (8 * k));
  }
  *word = v;
}

__global__ void __launch_bounds__(256) k_row_label(Inst* __restrict__ I) {
  pdl_enter();
  row_label(I[blockIdx.y], blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), threadIdx.x & 31);
}

// ------------------------------------------------------------------ a4: classify + compact
struct CandList {
  unsigned long long* cand;   // (instance << 40) | element
  unsigned long long cap;
  unsigned long long* count;  // [0] candidates, [1] work cursor of the exact kernel
};

// hole-map label of a point: 1 inside, 2 outside, 0 undecided (near a cube
// face, or in a NEAR cube).  Float arithmetic; `m` (in cube units) covers its
// rounding.
__device__ __forceinline__ int point_label(const Inst& in, float x, float y, float z, float m) {
  float c[3] = {(x - in.origin_f[0]) * in.inv_ds_f, (y - in.origin_f[1]) * in.inv_ds_f,
                (z - in.origin_f[2]) * in.inv_ds_f};
  int ix[3];
  for (int a = 0; a < 3; ++a) {
    if (c[a] < -m || c[a] > (float)in.dims[a] + m) return 2;  // outside the map: outside the surface box
    float fl = floorf(c[a]);
    if (c[a] - fl < m || fl + 1.0f - c[a] < m) return 0;      // too close to a cube face
    ix[a] = (int)fl;
    if (ix[a] < 0 || ix[a] >= in.dims[a]) return 0;
  }
  uint8_t s = in.cube[((long long)ix[2] * in.dims[1] + ix[1]) * CUBE_PITCH + ix[0]];
  if (s == CUBE_OUT) return 2;
  if (s == CUBE_IN) return 1;
  return 0;
}


// element g (every lane of a warp calls it; g past the end is a no-op lane):
// box against the hole map -> hole / field written, or listed as a candidate
__device__ void classify_elem(Inst* __restrict__ I, const long long* __restrict__ eoff, int n_inst,
                              long long ne_total, const CandList& cl, unsigned long long* __restrict__ cnt,
                              long long g) {
  const unsigned FULL = 0xffffffffu;
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
      const float inv = in.inv_ds_f;
      int c0[3], c1[3];
      bool outside = false, partial = false;
      for (int a = 0; a < 3; ++a) {
        const float o = in.origin_f[a];
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
              } else if (s == CUBE_IN) {
                any_in = true;
              } else {
                any_near = true;
                break;
              }
            }
          }
        if (any_near || (any_in && any_out)) {
          cand = true;
          // the exact stage reads every candidate's FP64 nodes next: start
          // bringing them into L2 now (a hint; 128-byte lines)
          const int npe = (in.p + 1) * (in.p + 1) * (in.p + 1);
          const char* nb = reinterpret_cast<const char*>(in.nodes + e * npe * 3);
          const char* ne = nb + npe * 24;
          for (const char* a = reinterpret_cast<const char*>(reinterpret_cast<uintptr_t>(nb) & ~uintptr_t(127)); a < ne;
               a += 128)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
        } else {
          flag = any_in ? DC_HOLE_ : DC_FIELD_;
        }
      }
    }
    if (!cand) {
      hole = flag == DC_HOLE_;
      in.flags[e] = flag;
      if (in.dist) in.dist[e] = (flag == DC_HOLE_) ? -HUGE_VAL : HUGE_VAL;
      if (in.dist32) in.dist32[e] = (flag == DC_HOLE_) ? -INFINITY : INFINITY;
    }
  }
  const unsigned hm = __ballot_sync(FULL, hole);
  if (hm && (threadIdx.x & 31) == 0) atomicAdd(&cnt[12], (unsigned long long)__popc(hm));
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

__global__ void __launch_bounds__(256) k_classify(Inst* __restrict__ I, const long long* __restrict__ eoff, int n_inst,
                                                  long long ne_total, CandList cl,
                                                  unsigned long long* __restrict__ cnt) {
  pdl_enter();
  classify_elem(I, eoff, n_inst, ne_total, cl, cnt, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// ------------------------------------------------------------------ the fused prep
// Grid barrier of the fused prep kernel.  The kernel is launched cooperatively,
// so every block is resident: each block's first thread makes the block's
// writes visible (fence), arrives, and waits with acquire loads until every
// block of the grid has arrived at this barrier (the count is never reset
// within a launch: barrier k waits for k * gridDim.x arrivals).  The wait is
// bounded: a wait that runs out sets *timed_out, which every later barrier
// sees, and the kernel leaves.
constexpr unsigned PREP_WAIT_LIMIT = 1u << 22;

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ bool prep_barrier(unsigned* count, unsigned k, unsigned* timed_out) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = ld_acquire_gpu(timed_out) == 0u;
    if (ok) {
      __threadfence();
      atomicAdd(count, 1u);
      const unsigned target = k * gridDim.x;
      for (unsigned it = 0; ld_acquire_gpu(count) < target; ++it) {
        if (it >= PREP_WAIT_LIMIT || ld_acquire_gpu(timed_out) != 0u) {
          atomicExch(timed_out, 1u);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// The surface ingest, hole map, face bins and element classification of a
// cut (a1-a4) in one cooperative launch: four steps (five for a batch), each
// a grid-stride loop over independent pieces of work, separated by grid
// barriers, which leaves the launch and drain of small kernels out of the
// chain.  sync[0]
// counts barrier arrivals, sync[1] records a barrier that ran out (the cut
// then reports an internal error).
// classify = 0: the classification is left to a separate k_classify launch
// (a batch of millions of elements, which a grid of one launch per SM's
// worth of threads would step through serially).
__global__ void __launch_bounds__(256) k_prep(Inst* __restrict__ I, const long long* __restrict__ off, int n_inst,
                                              long long nf_total, long long ne_total, CandList cl,
                                              unsigned long long* __restrict__ cnt, unsigned* __restrict__ sync,
                                              int classify) {
  pdl_enter();
  const long long* foff = off;
  const long long* eoff = off + n_inst + 1;
  const long long* toff = off + 2 * (n_inst + 1);   // surface tiles
  const long long* troff = off + 3 * (n_inst + 1);  // surface triangles
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthr = (long long)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  const long long gwarp = tid >> 5, nwarp = nthr >> 5;
  unsigned k = 0;
  // a1 + a2: pose and face boxes, SURF_FPB faces per block and step, the
  // tiles of every instance spread over the whole grid; the block that
  // finishes an instance's last tile derives its hole-map grid (a tile
  // counter per instance).  A single instance's map, bin counts and row
  // counts are cleared here to their full capacity (under a megabyte), which
  // needs no grid
  if (n_inst == 1) {
    clear_inst_cap(I[0], tid, nthr);
    // the classification reads every element box last: start bringing them
    // into L2 now (a hint, for grids whose boxes take a fraction of L2)
    const long long bytes = I[0].n_elem * 24;
    if (bytes <= (32ll << 20)) {
      const char* eb = reinterpret_cast<const char*>(I[0].eaabb);
      for (long long o = tid * 128; o < bytes; o += nthr * 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(eb + o));
    }
  }
  for (long long t = blockIdx.x; t < toff[n_inst]; t += gridDim.x) {
    const int ii = find_inst(toff, n_inst, t);
    surface_tile(I[ii], (t - toff[ii]) * SURF_FPB, true);
  }
  if (!prep_barrier(sync, ++k, sync + 1)) return;
  if (n_inst > 1) {
    // a batch clears what its grids use
    for (int ii = 0; ii < n_inst; ++ii) clear_inst(I[ii], tid, nthr);
    if (!prep_barrier(sync, ++k, sync + 1)) return;
  }
  // a3: NEAR cubes tagged and bins counted; the row centre lines' crossings
  // (which read only the posed surface and the grid) alongside
  // (one index space, so that the two kinds of work run on different threads)
  {
    const long long ntag = nf_total * TAG_R, nall = ntag + troff[n_inst];
    for (long long g = tid; g < nall; g += nthr) {
      if (g < ntag) {
        tag_face(I, foff, n_inst, nf_total, g);
      } else {
        const long long gt = g - ntag;
        const int ii = find_inst(troff, n_inst, gt);
        row_cross(I[ii], gt - troff[ii]);
      }
    }
  }
  if (!prep_barrier(sync, ++k, sync + 1)) return;
  // the bin counts scanned (a block per instance) while the other blocks
  // label the rows (crossings and NEAR tags are complete)
  {
    const int n_scan = min(n_inst, (int)(gridDim.x / 2));
    if ((int)blockIdx.x < n_scan) {
      for (int ii = blockIdx.x; ii < n_inst; ii += n_scan) bin_scan_inst(I[ii]);
    } else {
      const long long wpb = blockDim.x >> 5;
      const long long lw = gwarp - (long long)n_scan * wpb, nlw = nwarp - (long long)n_scan * wpb;
      for (int ii = 0; ii < n_inst; ++ii) {
        Inst& in = I[ii];
        const long long nrows = (long long)in.dims[1] * in.dims[2];
        for (long long r = lw; r < nrows; r += nlw) row_label(in, (int)r, lane);
      }
    }
  }
  if (!prep_barrier(sync, ++k, sync + 1)) return;
  // a4: faces into their bins, and every element against the map (warps
  // step together for the compaction), on separate threads
  // (the classification's index space starts after the fill's threads,
  // rounded to whole blocks so that warps stay aligned)
  const long long nfill = (nf_total + 255) / 256 * 256;
  for (long long g = tid; g < nf_total; g += nthr) bin_fill(I, foff, n_inst, nf_total, g);
  if (!classify) return;
  const long long first = nfill < nthr / 2 ? nfill : 0;
  for (long long base = tid - lane - first; base < ne_total; base += nthr)
    if (base >= 0) classify_elem(I, eoff, n_inst, ne_total, cl, cnt, base + lane);
}

}  // namespace dc
