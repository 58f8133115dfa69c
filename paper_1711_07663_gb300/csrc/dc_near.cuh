// dc_near.cuh -- the flags-only exact stage as flat kernels.
//
// When only flags are requested, an element needs the triangle search for one
// question only: does some triangle pair of the element and the surface come
// within tol (Sec. 4.2: "intersecting" elements)?  If not, its side is the
// hole-map label of any of its nodes (a labelled node lies in a cube that no
// face box touches).  Only pairs whose boxes come within tol can answer yes,
// so no branch and bound is needed and the work is flat:
//   k_near1       warp per candidate: node labels; nodes with both labels make
//                 the element fringe (its closed boundary crosses the surface);
//                 faces whose boxes come within tol of the element box become
//                 (element, face) tasks.  An element without tasks takes its
//                 label's side.
//   k_near_pairs  warp per task: the face's nodes in the element frame (float,
//                 kept for k_near_eval), triangle boxes of face and element in
//                 that frame; the pairs whose boxes come within tol (less the
//                 rounding bound) are listed.
//   k_near_eval   thread per pair: FP32 triangle-triangle test, with a
//                 certified crossing test and an FP64 re-solve of the pairs
//                 whose FP32 lower bound does not clear tol; a pair within tol
//                 marks its element fringe.
//   k_near3       thread per candidate: fringe, or its label's side.
// Elements that need distances, carry no label and are not fringe, or find a
// list full are decided by the full search (k_exact) afterwards.  The element
// frame (origin at the centre of the element's float box, node coordinates
// rounded to float) is the one the full search uses, computed once per
// resident grid; FP64 arithmetic, slow on this GPU, is left to the rare
// re-solves and to the per-task conversion of face nodes into the frame.
#pragma once

#include "dc_exact.cuh"

namespace dc {

// per-candidate status word
constexpr unsigned NS_PENDING = 1u, NS_IN = 2u, NS_FRINGE = 4u, NS_NOLABEL = 8u, NS_OVERFLOW = 16u;

struct NearBufs {
  unsigned* status;              // [candidate capacity]
  unsigned long long* task;      // (candidate position << 32) | face
  unsigned long long task_cap;
  unsigned long long* pair;      // (task << 16) | (element triangle << 8) | face triangle
  unsigned long long pair_cap;
  float* tface;                  // [task][3][(q+1)^2]: the task's face nodes in the element frame
  int tstride;                   // floats per task in tface
  unsigned long long* f64;       // pairs left to the FP64 test (pair index)
  unsigned long long f64_cap;
  unsigned long long* cnt;       // [0] tasks, [2] pairs, [5] pairs given the full FP32 test,
                                 // [6] FP64 list (counts may exceed the capacity)
};

__device__ __forceinline__ void push_full(CandList full, unsigned long long ent) {
  unsigned long long pos = atomicAdd(&full.count[0], 1ull);
  if (pos < full.cap) full.cand[pos] = ent;
}

__device__ __forceinline__ unsigned long long ucount(const unsigned long long* c, unsigned long long cap) {
  unsigned long long n = *c;
  return n < cap ? n : cap;
}


__global__ void __launch_bounds__(256) k_near1(Inst* __restrict__ I, CandList cl, CandList full, NearBufs nb,
                                               unsigned long long* __restrict__ gcnt) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
  const unsigned long long ncand = ucount(cl.count, cl.cap);
  unsigned long long n_fringe = 0, n_hole = 0, n_field = 0;
  for (unsigned long long w = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < ncand;
       w += nwarps) {
    const unsigned long long ent = cl.cand[w];
    const Inst& in = I[(int)(ent >> 40)];
    const long long e = (long long)(ent & ((1ull << 40) - 1ull));
    if (in.want_dist) {
      if (lane == 0) { nb.status[w] = 0u; push_full(full, ent); }
      continue;
    }
    const int p = in.p, npe = (p + 1) * (p + 1) * (p + 1);
    const float* gb = in.eaabb + 6 * e;
    float gbox[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) gbox[a] = gb[a];
    // node labels: node = frame origin + float local coordinate, as in the
    // full search (margin in cube units for the float rounding)
    const float* el = in.eloc + e * 3 * npe;
    float lx[4], ly[4], lz[4];
    float smax = 0.f;
    int nloc = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int nd = lane + 32 * r;
      lx[r] = ly[r] = lz[r] = 0.f;
      if (nd < npe) {
        lx[r] = el[nd];
        ly[r] = el[npe + nd];
        lz[r] = el[2 * npe + nd];
        smax = fmaxf(smax, fmaxf(fabsf(lx[r]), fmaxf(fabsf(ly[r]), fabsf(lz[r]))));
        nloc = r + 1;
      }
    }
    smax = warp_max(smax);
    int lab_or = 0;
    {
      const float ox = (float)in.eorg[3 * e], oy = (float)in.eorg[3 * e + 1], oz = (float)in.eorg[3 * e + 2];
      const float gm = fmaxf(fmaxf(fabsf(ox), fabsf(oy)), fabsf(oz)) + smax;
      const float m = 1e-5f + 16.0f * 5.9604645e-8f * gm * in.inv_ds_f;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (k < nloc) lab_or |= point_label(in, ox + lx[k], oy + ly[k], oz + lz[k], m);
    }
    const bool any_in = __any_sync(FULL, lab_or & 1), any_out = __any_sync(FULL, lab_or & 2);
    if (any_in && any_out) {
      if (lane == 0) { in.flags[e] = DC_FRINGE_; nb.status[w] = 0u; }
      n_fringe += (lane == 0);
      continue;
    }
    // faces whose boxes come within tol of the element box (each face sits in
    // the one bin of its box's low corner, hence the fext widening)
    const float fext[3] = {__uint_as_float(in.fext_bits[0]), __uint_as_float(in.fext_bits[1]),
                           __uint_as_float(in.fext_bits[2])};
    float gmax = 0.f;
#pragma unroll
    for (int a = 0; a < 6; ++a) gmax = fmaxf(gmax, fabsf(gbox[a]));
    const float tolf = in.tol_f;
    int b0[3], b1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float rf = tolf * 1.0001f;
      float glo = gbox[a] - rf - fext[a], ghi = gbox[3 + a] + rf;
      float oo = in.origin_f[a];
      float slack = 1e-3f + 16.0f * 5.9604645e-8f * (fabsf(glo) + fabsf(ghi) + fabsf(oo)) * in.inv_bs_f;
      b0[a] = clampi(cube_floorf((glo - oo) * in.inv_bs_f - slack, in.bdims[a]), 0, in.bdims[a] - 1);
      b1[a] = clampi(cube_floorf((ghi - oo) * in.inv_bs_f + slack, in.bdims[a]), 0, in.bdims[a] - 1);
    }
    const int nbx = b1[0] - b0[0] + 1, nby = b1[1] - b0[1] + 1, nbins = nbx * nby * (b1[2] - b0[2] + 1);
    int ntask = 0;
    bool overflow = false;
    for (int cb = 0; cb < nbins; cb += 32) {
      // up to 32 bins at once: lane j reads bin cb + j, a warp scan numbers
      // their faces, and the lanes walk the faces in steps of 32
      const int j = cb + lane;
      int f0 = 0, cnt = 0;
      if (j < nbins) {
        const int bx = b0[0] + j % nbx, by = b0[1] + (j / nbx) % nby, bz = b0[2] + j / (nbx * nby);
        const int bi = (bz * in.bdims[1] + by) * in.bdims[0] + bx;
        f0 = in.bin_off[bi];
        cnt = in.bin_off[bi + 1] - f0;
      }
      int incl = cnt;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int v = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += v;
      }
      const int excl = incl - cnt, total = __shfl_sync(FULL, incl, 31);
      for (int base = 0; base < total; base += 32) {
        const int k = base + lane, kk = min(k, total - 1);
        // the last lane whose first index is <= kk holds face kk
        int src = 0;
#pragma unroll
        for (int step = 16; step; step >>= 1) {
          const int c = src + step;
          if (__shfl_sync(FULL, excl, c) <= kk) src = c;
        }
        const int fsrc = __shfl_sync(FULL, f0, src), esrc = __shfl_sync(FULL, excl, src);
        bool keep = false;
        int f = 0;
        if (k < total) {
          f = in.bin_faces[fsrc + (kk - esrc)];
          const float* fb = in.fbox + 6 * (long long)f;
          float bb[6] = {fb[0], fb[1], fb[2], fb[3], fb[4], fb[5]};
          float fm = 0.f;
#pragma unroll
          for (int a = 0; a < 6; ++a) fm = fmaxf(fm, fabsf(bb[a]));
          float lb = box_dist<float>(gbox[0], gbox[1], gbox[2], gbox[3], gbox[4], gbox[5], bb[0], bb[1], bb[2],
                                     bb[3], bb[4], bb[5]);
          lb -= 8.0f * 5.9604645e-8f * fmaxf(gmax, fm);  // rounding of the float box distance
          keep = lb <= tolf;
        }
        const unsigned m = __ballot_sync(FULL, keep);
        if (m) {
          unsigned long long pos0 = 0;
          if (lane == 0) pos0 = atomicAdd(&nb.cnt[0], (unsigned long long)__popc(m));
          pos0 = __shfl_sync(FULL, pos0, 0);
          const unsigned long long pos = pos0 + __popc(m & ((1u << lane) - 1u));
          // every slot below the capacity is written, so readers of the
          // first min(count, capacity) entries see only valid tasks
          if (keep) {
            if (pos < nb.task_cap) nb.task[pos] = (w << 32) | (unsigned)f;
            else overflow = true;
          }
          ntask += __popc(m);
        }
      }
    }
    overflow = __any_sync(FULL, overflow);
    if (lane == 0) {
      const bool labelled = any_in || any_out;
      if (overflow || (ntask == 0 && !labelled)) {
        // the full search decides it (the tasks already listed are skipped:
        // the status is not pending)
        nb.status[w] = 0u;
        push_full(full, ent);
      } else if (ntask == 0) {
        in.flags[e] = any_in ? DC_HOLE_ : DC_FIELD_;
        nb.status[w] = 0u;
        n_hole += any_in;
        n_field += !any_in;
      } else {
        nb.status[w] = NS_PENDING | (any_in ? NS_IN : 0u) | (labelled ? 0u : NS_NOLABEL);
      }
    }
  }
  if (lane == 0 && (n_fringe | n_hole | n_field)) {
    atomicAdd(&gcnt[3], n_fringe);
    atomicAdd(&gcnt[4], n_hole);
    atomicAdd(&gcnt[5], n_field);
  }
}

constexpr int NEAR_PBUF = 128;  // per-warp staging of listed pairs

__device__ __forceinline__ void flush_pairs(NearBufs nb, CandList cl, unsigned long long* buf, int& nbuf, int lane) {
  const unsigned FULL = 0xffffffffu;
  __syncwarp();
  unsigned long long pos0 = 0;
  if (lane == 0) pos0 = atomicAdd(&nb.cnt[2], (unsigned long long)nbuf);
  pos0 = __shfl_sync(FULL, pos0, 0);
  for (int i = lane; i < nbuf; i += 32) {
    const unsigned long long v = buf[i];
    if (pos0 + i < nb.pair_cap) {
      nb.pair[pos0 + i] = v;
    } else {
      // no room: its element goes to the full search
      const unsigned long long w = nb.task[v >> 16] >> 32;
      atomicOr(&nb.status[w], NS_OVERFLOW);
    }
  }
  nbuf = 0;
  __syncwarp();
  (void)cl;
}

__global__ void __launch_bounds__(256) k_near_pairs(Inst* __restrict__ I, CandList cl, NearBufs nb,
                                                    unsigned long long* __restrict__ gcnt) {
  const unsigned FULL = 0xffffffffu;
  __shared__ unsigned char s_et[MAX_P][MAX_NTE][3], s_ft[MAX_Q][MAX_NTF][3];
  __shared__ float s_en[8][3 * MAX_NPE];          // element nodes, frame coordinates (x, y, z blocks)
  __shared__ float s_fn[8][3 * MAX_NPF];          // face nodes, same frame
  __shared__ float s_fb[8][6][MAX_NTF];           // face triangle boxes
  __shared__ float s_eb[8][6][32];                // boxes of the near element triangles of a chunk
  __shared__ int s_ci[8][32];                     // and their triangle numbers
  __shared__ unsigned long long s_pb[8][NEAR_PBUF];
  for (int i = threadIdx.x; i < (int)sizeof(s_et); i += blockDim.x) (&s_et[0][0][0])[i] = (&c_etri[0][0][0])[i];
  for (int i = threadIdx.x; i < (int)sizeof(s_ft); i += blockDim.x) (&s_ft[0][0][0])[i] = (&c_ftri[0][0][0])[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float* en = s_en[wid];
  float* fnl = s_fn[wid];
  float(*fb)[MAX_NTF] = s_fb[wid];
  float(*eb)[32] = s_eb[wid];
  int* cidx = s_ci[wid];
  unsigned long long* pb = s_pb[wid];
  int nbuf = 0;
  const unsigned long long ntask = ucount(nb.cnt, nb.task_cap), ncand = ucount(cl.count, cl.cap);
  const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
  unsigned long long n_task = 0;
  for (unsigned long long t = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + wid; t < ntask; t += nwarps) {
    const unsigned long long tk = nb.task[t];
    const unsigned long long w = tk >> 32;
    const int f = (int)(tk & 0xffffffffu);
    if (w >= ncand) continue;
    const unsigned st = ((volatile unsigned*)nb.status)[w];
    if (!(st & NS_PENDING) || (st & (NS_FRINGE | NS_OVERFLOW))) continue;
    const unsigned long long ent = cl.cand[w];
    const Inst& in = I[(int)(ent >> 40)];
    const long long e = (long long)(ent & ((1ull << 40) - 1ull));
    if (f < 0 || f >= in.n_faces) continue;
    const int p = in.p, q = in.q;
    const int npe = (p + 1) * (p + 1) * (p + 1), nte = 12 * p * p, npf = (q + 1) * (q + 1), ntf = 2 * q * q;
    const float tolf = in.tol_f;
    __syncwarp();
    // the face's nodes in the element frame (the one FP64 step of a task),
    // kept for the pair kernel; the element's from the resident frame
    const double* fn = in.surf + (long long)f * npf * 3;
    float* tf = nb.tface + t * (unsigned long long)nb.tstride;
    float smax = 0.f;
    for (int k = lane; k < 3 * npf; k += 32) {
      const int nd = k / 3, a = k - nd * 3;
      const float v = (float)(fn[k] - in.eorg[3 * e + a]);
      fnl[a * npf + nd] = v;
      tf[a * npf + nd] = v;
      smax = fmaxf(smax, fabsf(v));
    }
    const float* el = in.eloc + e * 3 * npe;
    for (int k = lane; k < 3 * npe; k += 32) {
      const float v = el[k];
      en[k] = v;
      smax = fmaxf(smax, fabsf(v));
    }
    smax = warp_max(smax);
    // pairs whose boxes are farther than tol plus the rounding bound of the
    // float copies cannot come within tol
    const float sigma = (float)C_SIGMA * Eps<float>::u * smax;
    __syncwarp();
    float flo[3] = {INFINITY, INFINITY, INFINITY}, fhi[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (lane < ntf) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int nd = s_ft[q - 1][lane][c];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const float v = fnl[a * npf + nd];
          flo[a] = fminf(flo[a], v);
          fhi[a] = fmaxf(fhi[a], v);
        }
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) { fb[a][lane] = flo[a]; fb[3 + a][lane] = fhi[a]; }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) { flo[a] = warp_min(flo[a]); fhi[a] = warp_max(fhi[a]); }
    __syncwarp();
    // pairs: lane = (group k, face triangle ts), groups of 32 / ntf lanes;
    // the lane's face-triangle box stays in registers
    const int G = ntf <= 32 ? 32 / ntf : 1;
    const int lk = lane / ntf, lts = lane - lk * ntf;
    const bool lvalid = lk < G;
    float my[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) my[a] = fb[a][lvalid ? lts : 0];
    for (int base = 0; base < nte; base += 32) {
      // element triangles of this chunk near the face box, compacted
      const int te = base + lane;
      bool near = false;
      float tlo[3] = {INFINITY, INFINITY, INFINITY}, thi[3] = {-INFINITY, -INFINITY, -INFINITY};
      if (te < nte) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int nd = s_et[p - 1][te][c];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const float v = en[a * npe + nd];
            tlo[a] = fminf(tlo[a], v);
            thi[a] = fmaxf(thi[a], v);
          }
        }
        near = box_dist<float>(tlo[0], tlo[1], tlo[2], thi[0], thi[1], thi[2], flo[0], flo[1], flo[2], fhi[0], fhi[1],
                               fhi[2]) - sigma <= tolf;
      }
      const unsigned em = __ballot_sync(FULL, near);
      if (near) {
        const int r = __popc(em & ((1u << lane) - 1u));
#pragma unroll
        for (int a = 0; a < 3; ++a) { eb[a][r] = tlo[a]; eb[3 + a][r] = thi[a]; }
        cidx[r] = te;
      }
      const int nnear = __popc(em);
      __syncwarp();
      for (int g0 = 0; g0 < nnear; g0 += G) {
        const int kk = g0 + lk;
        const bool valid = lvalid && kk < nnear;
        bool keep = false;
        int tk = 0;
        if (valid) {
          tk = cidx[kk];
          keep = box_dist<float>(eb[0][kk], eb[1][kk], eb[2][kk], eb[3][kk], eb[4][kk], eb[5][kk], my[0], my[1], my[2],
                                 my[3], my[4], my[5]) - sigma <= tolf;
        }
        const unsigned m = __ballot_sync(FULL, keep);
        if (m) {
          if (nbuf + __popc(m) > NEAR_PBUF) flush_pairs(nb, cl, pb, nbuf, lane);
          if (keep) pb[nbuf + __popc(m & ((1u << lane) - 1u))] = (t << 16) | ((unsigned)tk << 8) | (unsigned)lts;
          nbuf += __popc(m);
        }
      }
      __syncwarp();
    }
    n_task++;
  }
  if (nbuf) flush_pairs(nb, cl, pb, nbuf, lane);
  if (lane == 0 && n_task) atomicAdd(&gcnt[0], n_task);
}

template <class T>
__device__ __forceinline__ V3<T> pick3(const V3<T>* v, int j) {
  return j == 0 ? v[0] : (j == 1 ? v[1] : v[2]);
}

// Plane separation, in FP32 on the float copies A, B of the exact triangles
// (every coordinate within u S of the exact one, S >= every |coordinate|):
// true when the exact triangles are certainly farther apart than tol.
//
// If all three signed volumes s_j = n . (b_j - a_0) (n = the normal of A)
// exceed t |n| in one sign, B lies beyond A's plane by more than t, so
// d(A, B) > t.  Rounding: the float copies move each triangle by at most
// sqrt(3) u S; the computed n differs from the exact normal of the copies by
// at most 56 u S^2 in length, each s_j by at most 194 u S^3 + 14 u |n| S;
// with |n| > 512 u S^2 the margin K = 64 u S + 8 u tol + 512 u S^3 / |n|
// covers all of it (about twice what the sum needs).  The same holds with the
// roles of A and B swapped.
__device__ __forceinline__ bool near_separated(const V3<float>* A, const V3<float>* B, float S, float tolf) {
  const float u = Eps<float>::u;
  const V3<float> na = cross(A[1] - A[0], A[2] - A[0]), nb = cross(B[1] - B[0], B[2] - B[0]);
  const float la = sqrtf(dot(na, na)), lb = sqrtf(dot(nb, nb));
  const float S2 = S * S, S3 = S2 * S;
  const float ta = (tolf + 64.0f * u * S + 8.0f * u * tolf + 512.0f * u * S3 / la) * la;
  const float tb = (tolf + 64.0f * u * S + 8.0f * u * tolf + 512.0f * u * S3 / lb) * lb;
  const float s0 = dot(na, B[0] - A[0]), s1 = dot(na, B[1] - A[0]), s2 = dot(na, B[2] - A[0]);
  const float r0 = dot(nb, A[0] - B[0]), r1 = dot(nb, A[1] - B[0]), r2 = dot(nb, A[2] - B[0]);
  const bool sa = la > 512.0f * u * S2 &&
                  (fminf(s0, fminf(s1, s2)) > ta || fmaxf(s0, fmaxf(s1, s2)) < -ta);
  const bool sb = lb > 512.0f * u * S2 &&
                  (fminf(r0, fminf(r1, r2)) > tb || fmaxf(r0, fmaxf(r1, r2)) < -tb);
  return sa || sb;
}

// One listed pair, loaded: the float copies and the bound S, its candidate
// position w and the task's face f.  False if the pair is void (a capacity
// guard) or its element is already fringe.
struct NearPair {
  V3<float> A[3], B[3];
  float S;
  unsigned long long w;
  int f, te, ts;
  const Inst* in;
  long long e;
};

__device__ __forceinline__ bool load_pair(const Inst* __restrict__ I, const CandList& cl, const NearBufs& nb,
                                          const unsigned char (*s_et)[MAX_NTE][3],
                                          const unsigned char (*s_ft)[MAX_NTF][3], unsigned long long i,
                                          unsigned long long ntask, unsigned long long ncand, NearPair& P) {
  const unsigned long long pr = nb.pair[i];
  const unsigned long long t = pr >> 16;
  P.te = (int)((pr >> 8) & 255u);
  P.ts = (int)(pr & 255u);
  if (t >= ntask) return false;
  const unsigned long long tk = nb.task[t];
  P.w = tk >> 32;
  P.f = (int)(tk & 0xffffffffu);
  if (P.w >= ncand) return false;
  if (((volatile unsigned*)nb.status)[P.w] & NS_FRINGE) return false;
  const unsigned long long ent = cl.cand[P.w];
  P.in = &I[(int)(ent >> 40)];
  P.e = (long long)(ent & ((1ull << 40) - 1ull));
  const int p = P.in->p, q = P.in->q;
  if (P.te >= 12 * p * p || P.ts >= 2 * q * q || P.f < 0 || P.f >= P.in->n_faces) return false;
  const int npe = (p + 1) * (p + 1) * (p + 1), npf = (q + 1) * (q + 1);
  const float* el = P.in->eloc + P.e * 3 * npe;
  const float* tf = nb.tface + t * (unsigned long long)nb.tstride;
  float S = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int ni = s_et[p - 1][P.te][c], nj = s_ft[q - 1][P.ts][c];
    P.A[c] = mkv(el[ni], el[npe + ni], el[2 * npe + ni]);
    P.B[c] = mkv(tf[nj], tf[npf + nj], tf[2 * npf + nj]);
    S = fmaxf(S, fmaxf(fmaxf(fabsf(P.A[c].x), fabsf(P.A[c].y)), fabsf(P.A[c].z)));
    S = fmaxf(S, fmaxf(fmaxf(fabsf(P.B[c].x), fabsf(P.B[c].y)), fabsf(P.B[c].z)));
  }
  P.S = S;
  return true;
}

// Closest points of two segments (the formulas of seg_seg2), with every
// branch replaced by a select so that the lanes of a warp stay together.
__device__ __forceinline__ float seg_seg2_flat(V3<float> p, V3<float> d1, V3<float> q, V3<float> d2, V3<float>& cp,
                                               V3<float>& cq) {
  const V3<float> r = p - q;
  const float a = dot(d1, d1), e = dot(d2, d2), f = dot(d2, r), c = dot(d1, r), b = dot(d1, d2);
  const bool a0 = !(a > 0.f), e0 = !(e > 0.f);
  const float den = a * e - b * b;
  const float sg = den > 0.f ? clamp01((b * f - c * e) / (den > 0.f ? den : 1.f)) : 0.f;
  const float ee = e0 ? 1.f : e, aa = a0 ? 1.f : a;
  const float tg = (b * sg + f) / ee;
  const float slo = clamp01(-c / aa), shi = clamp01((b - c) / aa);
  float s = tg < 0.f ? slo : (tg > 1.f ? shi : sg);
  float t = tg < 0.f ? 0.f : (tg > 1.f ? 1.f : tg);
  // degenerate segments
  const float tf = clamp01(f / ee);
  s = a0 ? 0.f : (e0 ? slo : s);
  t = a0 ? (e0 ? 0.f : tf) : (e0 ? 0.f : t);
  cp = p + s * d1;
  cq = q + t * d2;
  const V3<float> w = cp - cq;
  return dot(w, w);
}

// The crossing tests of the triangle-triangle test, branch-free: the first
// edge found (in the test's order) is certified for the exact triangles.
// True if the pair certainly crosses (its element is fringe).
__device__ __noinline__ bool near_cross(const NearPair& P) {
  const float rho = 2.0f * Eps<float>::u * P.S;
  const V3<float>* a = P.A;
  const V3<float>* b = P.B;
  const V3<float> na = cross(a[1] - a[0], a[2] - a[0]), nb = cross(b[1] - b[0], b[2] - b[0]);
  float sb[3], sa[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) { sb[j] = dot(na, b[j] - a[0]); sa[j] = dot(nb, a[j] - b[0]); }
  const bool sepB = (sb[0] > 0.f && sb[1] > 0.f && sb[2] > 0.f) || (sb[0] < 0.f && sb[1] < 0.f && sb[2] < 0.f);
  const bool sepA = (sa[0] > 0.f && sa[1] > 0.f && sa[2] > 0.f) || (sa[0] < 0.f && sa[1] < 0.f && sa[2] < 0.f);
  const bool nosep = !sepA && !sepB;
  int xc = -1;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int k = (j + 1) % 3;
    {
      const float s0 = sb[j], s1 = sb[k];
      const bool c = nosep && ((s0 <= 0.f && s1 >= 0.f) || (s0 >= 0.f && s1 <= 0.f)) && s0 != s1;
      const V3<float> X = b[j] + (s0 / (c ? s0 - s1 : 1.f)) * (b[k] - b[j]);
      if (xc < 0 && c && in_tri(X, a[0], a[1], a[2], na)) xc = j;
    }
    {
      const float s0 = sa[j], s1 = sa[k];
      const bool c = nosep && ((s0 <= 0.f && s1 >= 0.f) || (s0 >= 0.f && s1 <= 0.f)) && s0 != s1;
      const V3<float> X = a[j] + (s0 / (c ? s0 - s1 : 1.f)) * (a[k] - a[j]);
      if (xc < 0 && c && in_tri(X, b[0], b[1], b[2], nb)) xc = 3 + j;
    }
  }
  if (__any_sync(__activemask(), xc >= 0)) {
    // one uniform call: lanes without a crossing certify a dummy and ignore it
    const int j = xc < 0 ? 0 : xc % 3;
    const V3<float>* se = (xc < 3) ? b : a;
    const V3<float>* tt = (xc < 3) ? a : b;
    const bool cert = certified_cross<float>(pick3(se, j), pick3(se, (j + 1) % 3), tt[0], tt[1], tt[2], rho);
    return xc >= 0 && cert;
  }
  return false;
}

// The FP32 bounds of the triangle-triangle test, branch-free: the best
// vertex-over-interior or edge-edge pair gives U and the gap L along its
// direction.  0: farther than tol, 2: undecided in FP32 (left to FP64).
__device__ __noinline__ int near_bounds(const NearPair& P) {
  const float sigma = (float)C_SIGMA * Eps<float>::u * P.S;
  const V3<float>* a = P.A;
  const V3<float>* b = P.B;
  const V3<float> na = cross(a[1] - a[0], a[2] - a[0]), nb = cross(b[1] - b[0], b[2] - b[0]);
  float sb[3], sa[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) { sb[j] = dot(na, b[j] - a[0]); sa[j] = dot(nb, a[j] - b[0]); }
  float best = INFINITY;
  V3<float> ca = a[0], cb = b[0];
  const float na2 = dot(na, na), nb2 = dot(nb, nb);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    {
      const V3<float> X = b[j] - (sb[j] / (na2 > 0.f ? na2 : 1.f)) * na;
      const V3<float> w = b[j] - X;
      const float d2 = dot(w, w);
      const bool ok = na2 > 0.f && in_tri(X, a[0], a[1], a[2], na) && d2 < best;
      best = ok ? d2 : best;
      ca = ok ? X : ca;
      cb = ok ? b[j] : cb;
    }
    {
      const V3<float> X = a[j] - (sa[j] / (nb2 > 0.f ? nb2 : 1.f)) * nb;
      const V3<float> w = a[j] - X;
      const float d2 = dot(w, w);
      const bool ok = nb2 > 0.f && in_tri(X, b[0], b[1], b[2], nb) && d2 < best;
      best = ok ? d2 : best;
      ca = ok ? a[j] : ca;
      cb = ok ? X : cb;
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      V3<float> cp, cq;
      const float d2 = seg_seg2_flat(a[i], a[(i + 1) % 3] - a[i], b[j], b[(j + 1) % 3] - b[j], cp, cq);
      const bool ok = d2 < best;
      best = ok ? d2 : best;
      ca = ok ? cp : ca;
      cb = ok ? cq : cb;
    }
  const V3<float> w = cb - ca;
  const float U = sqrtf(dot(w, w));
  float L = 0.f;
  if (U > 0.f) {
    const V3<float> wh = (1.0f / U) * w;
    const float bmin = fminf(dot(wh, b[0]), fminf(dot(wh, b[1]), dot(wh, b[2])));
    const float amax = fmaxf(dot(wh, a[0]), fmaxf(dot(wh, a[1]), dot(wh, a[2])));
    L = fmaxf(bmin - amax, 0.f);
  }
  return L - sigma > P.in->tol_f ? 0 : 2;
}

constexpr int NEAR_Q = 64;  // per-warp queue of undecided pairs

// Pass 1 over the listed pairs: certified crossings mark their elements
// fringe, so that pass 2 skips every other pair of those elements.
__global__ void __launch_bounds__(256) k_near_cross(Inst* __restrict__ I, CandList cl, NearBufs nb) {
  __shared__ unsigned char s_et[MAX_P][MAX_NTE][3], s_ft[MAX_Q][MAX_NTF][3];
  for (int i = threadIdx.x; i < (int)sizeof(s_et); i += blockDim.x) (&s_et[0][0][0])[i] = (&c_etri[0][0][0])[i];
  for (int i = threadIdx.x; i < (int)sizeof(s_ft); i += blockDim.x) (&s_ft[0][0][0])[i] = (&c_ftri[0][0][0])[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const unsigned long long npairs = ucount(nb.cnt + 2, nb.pair_cap), ntask = ucount(nb.cnt, nb.task_cap),
                           ncand = ucount(cl.count, cl.cap);
  const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
  for (unsigned long long base = ((unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32ull;
       base < npairs; base += nwarps * 32ull) {
    const unsigned long long i = base + lane;
    NearPair P;
    const bool ok = i < npairs && load_pair(I, cl, nb, s_et, s_ft, i, ntask, ncand, P);
    if (ok && near_cross(P)) atomicOr(&nb.status[P.w], NS_FRINGE);
    __syncwarp();
  }
}

__global__ void __launch_bounds__(256, 2) k_near_eval(Inst* __restrict__ I, CandList cl, NearBufs nb,
                                                      unsigned long long* __restrict__ gcnt) {
  const unsigned FULL = 0xffffffffu;
  __shared__ unsigned char s_et[MAX_P][MAX_NTE][3], s_ft[MAX_Q][MAX_NTF][3];
  __shared__ unsigned long long s_q[8][NEAR_Q];
  for (int i = threadIdx.x; i < (int)sizeof(s_et); i += blockDim.x) (&s_et[0][0][0])[i] = (&c_etri[0][0][0])[i];
  for (int i = threadIdx.x; i < (int)sizeof(s_ft); i += blockDim.x) (&s_ft[0][0][0])[i] = (&c_ftri[0][0][0])[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long* q = s_q[wid];
  const unsigned long long npairs = ucount(nb.cnt + 2, nb.pair_cap), ntask = ucount(nb.cnt, nb.task_cap),
                           ncand = ucount(cl.count, cl.cap);
  const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
  unsigned n_bulk = 0, n_full = 0;
  int nq = 0;
  // the undecided pairs, 32 lanes at a time
  auto drain = [&](int n) {
    int res = 0;
    unsigned long long w = 0;
    if (lane < n) {
      NearPair P;
      if (load_pair(I, cl, nb, s_et, s_ft, q[lane], ntask, ncand, P)) {
        res = near_bounds(P);
        w = P.w;
        n_full++;
      }
    }
    const unsigned m64 = __ballot_sync(FULL, res == 2);
    if (m64) {
      unsigned long long pos0 = 0;
      if (lane == 0) pos0 = atomicAdd(&nb.cnt[6], (unsigned long long)__popc(m64));
      pos0 = __shfl_sync(FULL, pos0, 0);
      const unsigned long long pos = pos0 + __popc(m64 & ((1u << lane) - 1u));
      if (res == 2) {
        if (pos < nb.f64_cap) nb.f64[pos] = q[lane];
        else atomicOr(&nb.status[w], NS_OVERFLOW);
      }
    }
    __syncwarp();
    const int rem = nq - n;
    const unsigned long long v = lane < rem ? q[n + lane] : 0ull;
    __syncwarp();
    if (lane < rem) q[lane] = v;
    nq = rem;
    __syncwarp();
  };
  for (unsigned long long base = ((unsigned long long)blockIdx.x * (blockDim.x >> 5) + wid) * 32ull; base < npairs;
       base += nwarps * 32ull) {
    const unsigned long long i = base + lane;
    bool undecided = false;
    if (i < npairs) {
      NearPair P;
      if (load_pair(I, cl, nb, s_et, s_ft, i, ntask, ncand, P)) {
        n_bulk++;
        undecided = !near_separated(P.A, P.B, P.S, P.in->tol_f);
      }
    }
    const unsigned m = __ballot_sync(FULL, undecided);
    if (undecided) q[nq + __popc(m & ((1u << lane) - 1u))] = i;
    nq += __popc(m);
    __syncwarp();
    if (nq >= 32) drain(32);
  }
  while (nq > 0) drain(min(nq, 32));
  n_bulk = __reduce_add_sync(FULL, n_bulk);
  n_full = __reduce_add_sync(FULL, n_full);
  if (lane == 0 && n_bulk) {
    atomicAdd(&gcnt[1], (unsigned long long)n_bulk);
    atomicAdd(&nb.cnt[5], (unsigned long long)n_full);
  }
}

// FP64 distance of one triangle pair, the 21 parts of the triangle-triangle
// test spread over the lanes (lanes 0-5: an edge of one triangle through the
// other; 6-11: a vertex over the other's interior; 12-20: edge pairs), then a
// warp minimum: the same values the one-thread test computes, at a fraction
// of its latency (FP64 issues slowly on this GPU).  a, b: the FP64 vertices in
// the element frame.  Returns the distance (0 for a crossing).
__device__ double tritri64_warp(const V3<double>* a, const V3<double>* b, int lane) {
  const V3<double> na = cross(a[1] - a[0], a[2] - a[0]), nb = cross(b[1] - b[0], b[2] - b[0]);
  double sb[3], sa[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) { sb[j] = dot(na, b[j] - a[0]); sa[j] = dot(nb, a[j] - b[0]); }
  const bool sepB = (sb[0] > 0.0 && sb[1] > 0.0 && sb[2] > 0.0) || (sb[0] < 0.0 && sb[1] < 0.0 && sb[2] < 0.0);
  const bool sepA = (sa[0] > 0.0 && sa[1] > 0.0 && sa[2] > 0.0) || (sa[0] < 0.0 && sa[1] < 0.0 && sa[2] < 0.0);
  const double na2 = dot(na, na), nb2 = dot(nb, nb);
  double d2 = INFINITY;
  bool cross_hit = false;
  if (lane < 6) {
    if (!sepA && !sepB) {
      const int j = lane % 3, k = (j + 1) % 3;
      const bool ofB = lane < 3;  // edge of B through A, else edge of A through B
      const double s0 = ofB ? sb[j] : sa[j], s1 = ofB ? sb[k] : sa[k];
      if (((s0 <= 0.0 && s1 >= 0.0) || (s0 >= 0.0 && s1 <= 0.0)) && s0 != s1) {
        const V3<double> P0 = ofB ? pick3(b, j) : pick3(a, j), P1 = ofB ? pick3(b, k) : pick3(a, k);
        const V3<double> X = P0 + (s0 / (s0 - s1)) * (P1 - P0);
        cross_hit = ofB ? in_tri(X, a[0], a[1], a[2], na) : in_tri(X, b[0], b[1], b[2], nb);
      }
    }
  } else if (lane < 12) {
    const int j = (lane - 6) % 3;
    if (lane < 9) {
      if (na2 > 0.0) {
        const V3<double> bj = pick3(b, j);
        const V3<double> X = bj - (sb[j] / na2) * na;
        if (in_tri(X, a[0], a[1], a[2], na)) { const V3<double> w = bj - X; d2 = dot(w, w); }
      }
    } else if (nb2 > 0.0) {
      const V3<double> aj = pick3(a, j);
      const V3<double> X = aj - (sa[j] / nb2) * nb;
      if (in_tri(X, b[0], b[1], b[2], nb)) { const V3<double> w = aj - X; d2 = dot(w, w); }
    }
  } else if (lane < 21) {
    const int i = (lane - 12) / 3, j = (lane - 12) % 3;
    const V3<double> ai = pick3(a, i), bj = pick3(b, j);
    V3<double> cp, cq;
    d2 = seg_seg2(ai, pick3(a, (i + 1) % 3) - ai, bj, pick3(b, (j + 1) % 3) - bj, cp, cq);
  }
  if (__any_sync(0xffffffffu, cross_hit)) return 0.0;
  return sqrt(warp_min(d2));
}

// The pairs the FP32 test left undecided, once every certified crossing is
// known: warp per pair, skipped when its element is already fringe.
__global__ void __launch_bounds__(256) k_near_fp64(Inst* __restrict__ I, CandList cl, NearBufs nb,
                                                   unsigned long long* __restrict__ gcnt) {
  const int lane = threadIdx.x & 31;
  const unsigned long long n = ucount(nb.cnt + 6, nb.f64_cap), ntask = ucount(nb.cnt, nb.task_cap),
                           ncand = ucount(cl.count, cl.cap);
  const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
  unsigned long long n_re = 0;
  for (unsigned long long k = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < n;
       k += nwarps) {
    const unsigned long long pr = nb.pair[nb.f64[k]];
    const unsigned long long t = pr >> 16;
    const int te = (int)((pr >> 8) & 255u), ts = (int)(pr & 255u);
    if (t >= ntask) continue;
    const unsigned long long tk = nb.task[t];
    const unsigned long long w = tk >> 32;
    const int f = (int)(tk & 0xffffffffu);
    if (w >= ncand || (((volatile unsigned*)nb.status)[w] & NS_FRINGE)) continue;
    const unsigned long long ent = cl.cand[w];
    const Inst& in = I[(int)(ent >> 40)];
    const long long e = (long long)(ent & ((1ull << 40) - 1ull));
    const int p = in.p, q = in.q;
    if (te >= 12 * p * p || ts >= 2 * q * q || f < 0 || f >= in.n_faces) continue;
    const int npe = (p + 1) * (p + 1) * (p + 1), npf = (q + 1) * (q + 1);
    const double* en = in.nodes + e * npe * 3;
    const double* fn = in.surf + (long long)f * npf * 3;
    const double o[3] = {in.eorg[3 * e], in.eorg[3 * e + 1], in.eorg[3 * e + 2]};
    V3<double> a[3], b[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int ni = c_etri[p - 1][te][c], nj = c_ftri[q - 1][ts][c];
      a[c] = mkv(en[3 * ni] - o[0], en[3 * ni + 1] - o[1], en[3 * ni + 2] - o[2]);
      b[c] = mkv(fn[3 * nj] - o[0], fn[3 * nj + 1] - o[1], fn[3 * nj + 2] - o[2]);
    }
    const double d = tritri64_warp(a, b, lane);
    n_re++;
    if (lane == 0 && d <= in.tol) atomicOr(&nb.status[w], NS_FRINGE);
  }
  if (lane == 0 && n_re) atomicAdd(&gcnt[2], n_re);
}

__global__ void __launch_bounds__(256) k_near3(Inst* __restrict__ I, CandList cl, CandList full, NearBufs nb,
                                               unsigned long long* __restrict__ gcnt) {
  const unsigned long long ncand = ucount(cl.count, cl.cap);
  unsigned n_fringe = 0, n_hole = 0, n_field = 0;
  for (unsigned long long w = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; w < ncand;
       w += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned st = nb.status[w];
    if (!(st & NS_PENDING)) continue;
    const unsigned long long ent = cl.cand[w];
    const Inst& in = I[(int)(ent >> 40)];
    const long long e = (long long)(ent & ((1ull << 40) - 1ull));
    if (st & NS_FRINGE) {
      in.flags[e] = DC_FRINGE_;
      n_fringe++;
    } else if (st & (NS_NOLABEL | NS_OVERFLOW)) {
      push_full(full, ent);
    } else {
      in.flags[e] = (st & NS_IN) ? DC_HOLE_ : DC_FIELD_;
      n_hole += (st & NS_IN) != 0;
      n_field += (st & NS_IN) == 0;
    }
  }
  n_fringe = __reduce_add_sync(0xffffffffu, n_fringe);
  n_hole = __reduce_add_sync(0xffffffffu, n_hole);
  n_field = __reduce_add_sync(0xffffffffu, n_field);
  if ((threadIdx.x & 31) == 0 && (n_fringe | n_hole | n_field)) {
    atomicAdd(&gcnt[3], (unsigned long long)n_fringe);
    atomicAdd(&gcnt[4], (unsigned long long)n_hole);
    atomicAdd(&gcnt[5], (unsigned long long)n_field);
  }
}

}  // namespace dc
