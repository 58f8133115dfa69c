// dc_near.cuh -- the flags-only exact stage.
//
// When only flags are requested, an element needs the triangle search for one
// question only: does some triangle pair of the element and the surface come
// within tol (Sec. 4.2: "intersecting" elements)?  If not, its side is the
// hole-map label of any of its nodes (a labelled node lies in a cube that no
// face box touches).  Only pairs whose boxes come within tol can answer yes,
// so no branch and bound is needed:
//   k_near_main    warp per candidate: node labels (nodes with both labels:
//                  fringe); the faces whose boxes come within tol of the
//                  element box, gathered into a list first and then taken 8
//                  at a time, each converted once into the element frame;
//                  the triangle pairs whose boxes come within tol (less the
//                  rounding bound), 32 at a time: plane separation settles most,
//                  a certified FP32 crossing makes the element fringe and ends
//                  its search; the rest wait in a per-warp list until the
//                  element's faces are done, then (element still not fringe)
//                  take the FP32 bound test and, where that cannot clear tol,
//                  the FP64 test (warp-parallel).  The element is fringe, or
//                  takes its label's side.
// Elements that need distances, or carry no label and are not fringe, are
// listed for the full per-element search, which k_exact runs right after this
// kernel (FP32 with FP64 re-solves, FP64 for the elements whose re-solve list
// overflows); keeping that search and its shared scratch out of this kernel
// leaves it a smaller code footprint and more of the SM's storage as L1.  The
// element frame (origin at the centre of the element's float box, node
// coordinates rounded to float) is the one the full search uses, formed for
// each candidate from its FP64 nodes (candidates are a few percent of the grid:
// forming frames for every element when the grid is created would cost the
// sweep over the nodes more FP64 work than every cut's candidates together);
// the rest of the FP64 arithmetic, slow on this GPU, is the face conversions
// and the rare re-solves.
#pragma once

#include "dc_exact.cuh"

namespace dc {

struct NearBufs {
  unsigned long long* cnt;       // [0] faces tested, [3] full searches, [5] pairs given the full FP32 test
};

__device__ __forceinline__ unsigned long long ucount(const unsigned long long* c, unsigned long long cap) {
  unsigned long long n = *c;
  return n < cap ? n : cap;
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

// Certified crossings without divisions.  A signed volume of four of the
// float points, evaluated as in orient_cert, moves by at most
// B = 8 rho L^2 + 16 rho^2 L + 32 u L^3 when the points move to the exact
// (FP64) ones within rho = 2 u S, for L at least the longest edge vector plus
// 2 rho (orient_cert's bound).  Every point lies in [-S, S]^3, so
// L = 2 sqrt(3) S (1 + 1e-4) + 2 rho serves for all of them: one bound per
// pair instead of one square root per volume, never below orient_cert's.
// An edge PQ of one triangle crosses the other when P and Q lie beyond B on
// opposite sides of its plane and the three volumes of PQ with its edges
// exceed B in one sign; then the exact triangles intersect.  True if some
// edge of either triangle certainly crosses the other (the element is
// fringe).
__device__ __forceinline__ bool edge_cert(V3<float> P, V3<float> Q, const V3<float>* t, float B) {
  const V3<float> d = Q - P, e0 = t[0] - P, e1 = t[1] - P, e2 = t[2] - P;
  const float o0 = dot(cross(d, e0), e1), o1 = dot(cross(d, e1), e2), o2 = dot(cross(d, e2), e0);
  return (o0 > B && o1 > B && o2 > B) || (o0 < -B && o1 < -B && o2 < -B);
}
__device__ __forceinline__ bool near_cross(const V3<float>* a, const V3<float>* b, float S) {
  const float u = Eps<float>::u;
  const float rho = 2.0f * u * S;
  const float L = 3.4646f * S + 2.0f * rho;
  // (1.01: the rounding of the bound's own evaluation)
  const float B = 1.01f * (8.0f * rho * L * L + 16.0f * rho * rho * L + 32.0f * u * L * L * L);
  const V3<float> na = cross(a[1] - a[0], a[2] - a[0]), nb = cross(b[1] - b[0], b[2] - b[0]);
  float sb[3], sa[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) { sb[j] = dot(na, b[j] - a[0]); sa[j] = dot(nb, a[j] - b[0]); }
  bool hit = false;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int k = (j + 1) % 3;
    if (!hit && ((sb[j] > B && sb[k] < -B) || (sb[j] < -B && sb[k] > B))) hit = edge_cert(b[j], b[k], a, B);
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int k = (j + 1) % 3;
    if (!hit && ((sa[j] > B && sa[k] < -B) || (sa[j] < -B && sa[k] > B))) hit = edge_cert(a[j], a[k], b, B);
  }
  return hit;
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

// shared memory of one warp of k_near_main
constexpr int NEAR_UCAP = 32;  // undecided pairs a warp holds for its element

// a warp's counts of one launch, in its shared region (lane 0 keeps them)
enum { NW_FS, NW_FRINGE, NW_HOLE, NW_FIELD, NW_FACES, NW_PAIRS, NW_FULL, NW_RE, NW_N };


// The undecided pairs a warp holds for its element (nul <= 32, lane k takes
// pair k): the FP32 bounds of the compact triangle test, then the FP64 test
// (warp-parallel) for each pair those cannot clear.  True if a pair comes
// within tol.
__device__ __noinline__ bool near_settle(const Inst& in, long long e, const double* eo, const float* en,
                                         const int2* ul, int nul, const unsigned char (*s_et)[MAX_NTE][3],
                                         const unsigned char (*s_ft)[MAX_NTF][3], int lane,
                                         unsigned* wc) {
  const unsigned FULL = 0xffffffffu;
  const int p = in.p, q = in.q, npe = (p + 1) * (p + 1) * (p + 1), npf = (q + 1) * (q + 1);
  const float tolf = in.tol_f;
  bool open = false;
  int f = 0, te = 0, ts = 0;
  if (lane < nul) {
    const int2 v = ul[lane];
    f = v.x;
    te = v.y & 0xffff;
    ts = v.y >> 16;
    const double* fsp = in.surf + (long long)f * npf * 3;
    V3<float> A[3], B[3];
    float S = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int ni = s_et[p - 1][te][c], nj = s_ft[q - 1][ts][c];
      A[c] = mkv(en[ni], en[npe + ni], en[2 * npe + ni]);
      B[c] = mkv((float)(fsp[3 * nj] - eo[0]), (float)(fsp[3 * nj + 1] - eo[1]), (float)(fsp[3 * nj + 2] - eo[2]));
      S = fmaxf(S, fmaxf(fmaxf(fabsf(A[c].x), fabsf(A[c].y)), fabsf(A[c].z)));
      S = fmaxf(S, fmaxf(fmaxf(fabsf(B[c].x), fabsf(B[c].y)), fabsf(B[c].z)));
    }
    float U, L;
    V3<float> ca, cb;
    int xc;
    tritri<float, false>(A, B, U, L, ca, cb, xc);
    open = L - (float)C_SIGMA * Eps<float>::u * S <= tolf;
  }
  if (lane == 0) wc[NW_FULL] += (unsigned)nul;
  unsigned m64 = __ballot_sync(FULL, open);
  while (m64) {
    const int src = __ffs(m64) - 1;
    m64 &= m64 - 1;
    const int fs = __shfl_sync(FULL, f, src), tes = __shfl_sync(FULL, te, src), tss = __shfl_sync(FULL, ts, src);
    const double* en64 = in.nodes + e * npe * 3;
    const double* fn64 = in.surf + (long long)fs * npf * 3;
    V3<double> a[3], b[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int ni = s_et[p - 1][tes][c], nj = s_ft[q - 1][tss][c];
      a[c] = mkv(en64[3 * ni] - eo[0], en64[3 * ni + 1] - eo[1], en64[3 * ni + 2] - eo[2]);
      b[c] = mkv(fn64[3 * nj] - eo[0], fn64[3 * nj + 1] - eo[1], fn64[3 * nj + 2] - eo[2]);
    }
    const double d = tritri64_warp(a, b, lane);
    if (lane == 0) wc[NW_RE] += 1u;
    if (d <= in.tol) return true;
  }
  return false;
}

// faces of one candidate tested together (their nodes are loaded at once)
constexpr int NEAR_FB = 8;

// faces gathered for one candidate before its batches run (more wait for the
// next gathering round)
constexpr int NEAR_FLCAP = 64;

struct NearLayout {
  int en, eb, fl, ffb, fn, fb, ci, pq, ul, wc, total;
};
__host__ __device__ constexpr NearLayout near_layout(int pmax, int qmax) {
  const int npe = (pmax + 1) * (pmax + 1) * (pmax + 1), nte = 12 * pmax * pmax;
  const int npf = (qmax + 1) * (qmax + 1), ntf = 2 * qmax * qmax;
  NearLayout L{};
  int o = 0;
  L.en = o; o = align16(o + 3 * npe * 4);              // element nodes, frame coordinates (x, y, z blocks)
  L.eb = o; o = align16(o + 6 * nte * 4);              // element triangle boxes [6][nte]
  L.fl = o; o = align16(o + NEAR_FLCAP * 4);          // gathered faces (a batch is a run of NEAR_FB of them)
  L.ffb = o; o = align16(o + NEAR_FB * 8 * 4);         // their boxes in the frame (lo, hi)
  L.fn = o; o = align16(o + NEAR_FB * 3 * npf * 4);    // their nodes in the frame [face][x|y|z][node]
  L.fb = o; o = align16(o + NEAR_FB * 6 * ntf * 4);    // their triangle boxes [face][6][ntf]
  L.ci = o; o = align16(o + 32 * 4);                   // near (face, element triangle) of a chunk
  L.pq = o; o = align16(o + 64 * 4);                   // queued pairs (face << 16 | te << 8 | ts)
  L.ul = o; o = align16(o + NEAR_UCAP * 8);            // undecided pairs (face id, te | ts << 16)
  L.wc = o; o = align16(o + NW_N * 4);                 // the warp's counts
  L.total = o;
  return L;
}

// bytes of shared scratch per warp of k_near_main (the full per-element search
// runs in the exact kernels, with their own layout, so none is kept for it:
// the smaller reservation leaves the SM's combined L1 / shared storage to L1)
__host__ __device__ constexpr int near_region(int pmax, int qmax) { return near_layout(pmax, qmax).total; }

// at most 16 warps per block (4, 8 or 16 are launched; 128 registers per
// thread either way)
constexpr int NEAR_MAX_WARPS = 16;

// P, Q > 0: every instance has element order P and face order Q (counts and
// offsets known at compile time); P = Q = 0: any orders up to pmax, qmax.
template <int P, int Q>
__global__ void __launch_bounds__(NEAR_MAX_WARPS * 32, 1)
    k_near_main(Inst* __restrict__ I, CandList cl, CandList full, NearBufs nb, int pmax, int qmax, int cpw,
                unsigned long long* __restrict__ gcnt) {
  constexpr bool FIXED = P > 0 && Q > 0;
  const unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned char s_et[MAX_P][MAX_NTE][3], s_ft[MAX_Q][MAX_NTF][3];
  for (int i = threadIdx.x; i < (int)sizeof(s_et); i += blockDim.x) (&s_et[0][0][0])[i] = (&c_etri[0][0][0])[i];
  for (int i = threadIdx.x; i < (int)sizeof(s_ft); i += blockDim.x) (&s_ft[0][0][0])[i] = (&c_ftri[0][0][0])[i];
  pdl_enter();
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const NearLayout Lo = FIXED ? near_layout(P, Q) : near_layout(pmax, qmax);
  unsigned char* ws = smem + (size_t)wid * Lo.total;
  unsigned* const wc = reinterpret_cast<unsigned*>(ws + Lo.wc);
  if ((threadIdx.x & 31) < NW_N) wc[threadIdx.x & 31] = 0u;
  __syncwarp();
  // a candidate that needs the full per-element search (distances requested,
  // or no node labelled and not fringe) goes to the exact kernels' list;
  // k_exact runs right after this kernel
  auto full_one = [&](unsigned long long ent) {
    if (lane == 0) {
      wc[NW_FS] += 1u;
      const unsigned long long pos = atomicAdd(&full.count[0], 1ull);
      if (pos < full.cap) full.cand[pos] = ent;
    }
    __syncwarp();
  };
  float* en = reinterpret_cast<float*>(ws + Lo.en);
  float* eb = reinterpret_cast<float*>(ws + Lo.eb);
  int* const fl = reinterpret_cast<int*>(ws + Lo.fl);
  int* fid = fl;  // the faces of the current batch
  float* ffb = reinterpret_cast<float*>(ws + Lo.ffb);
  float* fnl = reinterpret_cast<float*>(ws + Lo.fn);
  float* fb = reinterpret_cast<float*>(ws + Lo.fb);
  int* ci = reinterpret_cast<int*>(ws + Lo.ci);
  int* pq = reinterpret_cast<int*>(ws + Lo.pq);
  int2* ul = reinterpret_cast<int2*>(ws + Lo.ul);
  const unsigned long long ncand = ucount(cl.count, cl.cap);
  // per-warp counts of one launch (32 bits suffice)
  unsigned long long w = 0, wend = 0;
  while (true) {
    // candidates are taken from a shared cursor, cpw at a time: their costs
    // differ widely
    if (w >= wend) {
      unsigned long long w0 = 0;
      if (lane == 0) w0 = atomicAdd(&cl.count[1], (unsigned long long)cpw);
      w0 = __shfl_sync(FULL, w0, 0);
      if (w0 >= ncand) break;
      w = w0;
      wend = w0 + (unsigned long long)cpw < ncand ? w0 + (unsigned long long)cpw : ncand;
    }
    const unsigned long long ent = cl.cand[w++];
    const Inst& in = I[(int)(ent >> 40)];
    const long long e = (long long)(ent & ((1ull << 40) - 1ull));
    if (in.want_dist) {
      full_one(ent);
      continue;
    }
    const int p = FIXED ? P : in.p, q = FIXED ? Q : in.q;
    const int npe = (p + 1) * (p + 1) * (p + 1), nte = 12 * p * p, npf = (q + 1) * (q + 1), ntf = 2 * q * q;
    const float* gb = in.eaabb + 6 * e;
    float gbox[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) gbox[a] = gb[a];
    // the element frame: origin at the centre of the float box, node
    // coordinates relative to it rounded to float (the full search's frame)
    const double eo[3] = {0.5 * ((double)gbox[0] + (double)gbox[3]), 0.5 * ((double)gbox[1] + (double)gbox[4]),
                          0.5 * ((double)gbox[2] + (double)gbox[5])};
    // element nodes in the frame, and their hole-map labels (node = frame
    // origin + float local coordinate, as in the full search)
    const double* xn = in.nodes + e * npe * 3;
    float smax = 0.f;
    int lab_or = 0;
    {
      const float ox = (float)eo[0], oy = (float)eo[1], oz = (float)eo[2];
      float lx[4], ly[4], lz[4];
      int nloc = 0;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int nd = lane + 32 * r;
        lx[r] = ly[r] = lz[r] = 0.f;
        if (nd < npe) {
          lx[r] = (float)(xn[3 * nd] - eo[0]);
          ly[r] = (float)(xn[3 * nd + 1] - eo[1]);
          lz[r] = (float)(xn[3 * nd + 2] - eo[2]);
          en[nd] = lx[r];
          en[npe + nd] = ly[r];
          en[2 * npe + nd] = lz[r];
          smax = fmaxf(smax, fmaxf(fabsf(lx[r]), fmaxf(fabsf(ly[r]), fabsf(lz[r]))));
          nloc = r + 1;
        }
      }
      smax = warp_max(smax);
      const float gm = fmaxf(fmaxf(fabsf(ox), fabsf(oy)), fabsf(oz)) + smax;
      const float m = 1e-5f + 16.0f * 5.9604645e-8f * gm * in.inv_ds_f;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (k < nloc) lab_or |= point_label(in, ox + lx[k], oy + ly[k], oz + lz[k], m);
    }
    const bool any_in = __any_sync(FULL, lab_or & 1), any_out = __any_sync(FULL, lab_or & 2);
    if (any_in && any_out) {
      // nodes on both sides: the closed element boundary crosses the surface
      if (lane == 0) in.flags[e] = DC_FRINGE_;
      if (lane == 0) wc[NW_FRINGE] += 1u;
      continue;
    }
    const float Se = smax, tolf = in.tol_f;
    bool have_eb = false;
    // element triangle boxes, once per element (when its first face is found)
    auto make_eb = [&]() {
      __syncwarp();
      for (int te = lane; te < nte; te += 32) {
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int nd = s_et[p - 1][te][c];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const float v = en[a * npe + nd];
            lo[a] = fminf(lo[a], v);
            hi[a] = fmaxf(hi[a], v);
          }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) { eb[a * nte + te] = lo[a]; eb[(3 + a) * nte + te] = hi[a]; }
      }
      __syncwarp();
    };
    // faces whose boxes come within tol of the element box (each face sits in
    // the one bin of its box's low corner, hence the fext widening)
    const float fext[3] = {__uint_as_float(in.fext_bits[0]), __uint_as_float(in.fext_bits[1]),
                           __uint_as_float(in.fext_bits[2])};
    float gmax = 0.f;
#pragma unroll
    for (int a = 0; a < 6; ++a) gmax = fmaxf(gmax, fabsf(gbox[a]));
    int b0[3], b1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float rf = tolf * 1.0001f;
      const float glo = gbox[a] - rf - fext[a], ghi = gbox[3 + a] + rf;
      const float oo = in.origin_f[a];
      const float slack = 1e-3f + 16.0f * 5.9604645e-8f * (fabsf(glo) + fabsf(ghi) + fabsf(oo)) * in.inv_bs_f;
      b0[a] = clampi(cube_floorf((glo - oo) * in.inv_bs_f - slack, in.bdims[a]), 0, in.bdims[a] - 1);
      b1[a] = clampi(cube_floorf((ghi - oo) * in.inv_bs_f + slack, in.bdims[a]), 0, in.bdims[a] - 1);
    }
    const int nbx = b1[0] - b0[0] + 1, nby = b1[1] - b0[1] + 1, nbins = nbx * nby * (b1[2] - b0[2] + 1);
    // lanes of the pair step: (group k, face triangle ts), 32 / ntf groups
    const int G = ntf <= 32 ? 32 / ntf : 1;
    const int lk = lane / ntf, lts = lane - lk * ntf;
    const bool lvalid = lk < G;
    bool fringe = false;
    int nul = 0;  // undecided pairs held in ul
    int nbf = 0;  // faces gathered into the batch
    int nq = 0;   // queued pairs
    // the held pairs: FP32 bounds (the compact form of the triangle test),
    // then FP64 (warp-parallel) for what they cannot clear
    auto settle = [&]() {
      __syncwarp();
      if (near_settle(in, e, eo, en, ul, nul, s_et, s_ft, lane, wc)) fringe = true;
      nul = 0;
      __syncwarp();
    };
    // the queued pairs, 32 lanes at a time: separation, then crossings; the
    // rest are listed undecided
    auto drain = [&](int n) {
      bool need = false, crossed = false;
      int fi = 0, te = 0, ts = 0;
      V3<float> A[3], B[3];
      float S = 0.f;
      if (lane < n) {
        const int code = pq[lane];
        fi = code >> 16;
        te = (code >> 8) & 255;
        ts = code & 255;
        const float* fx = fnl + fi * 3 * npf;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int ni = s_et[p - 1][te][c], nj = s_ft[q - 1][ts][c];
          A[c] = mkv(en[ni], en[npe + ni], en[2 * npe + ni]);
          B[c] = mkv(fx[nj], fx[npf + nj], fx[2 * npf + nj]);
          S = fmaxf(S, fmaxf(fmaxf(fabsf(A[c].x), fabsf(A[c].y)), fabsf(A[c].z)));
          S = fmaxf(S, fmaxf(fmaxf(fabsf(B[c].x), fabsf(B[c].y)), fabsf(B[c].z)));
        }
        need = !near_separated(A, B, S, tolf);
      }
      if (lane == 0) wc[NW_PAIRS] += (unsigned)n;
      if (need) crossed = near_cross(A, B, S);
      if (__any_sync(FULL, crossed)) {
        fringe = true;
      } else {
        const unsigned um = __ballot_sync(FULL, need);
        if (um) {
          if (nul + __popc(um) > 32) settle();
          if (!fringe) {
            if (need) ul[nul + __popc(um & ((1u << lane) - 1u))] = make_int2(fid[fi], te | (ts << 16));
            nul += __popc(um);
          }
        }
      }
      __syncwarp();
      const int rem = nq - n;
      const int v = lane < rem ? pq[n + lane] : 0;
      __syncwarp();
      if (lane < rem) pq[lane] = v;
      nq = rem;
      __syncwarp();
    };
    // the faces of the batch together: nodes into the frame (every node load
    // of the batch in flight at once), frame boxes and rounding bounds,
    // triangle boxes, then the (face, element triangle) pairs whose boxes come
    // within tol and their triangle pairs
    auto run_batch = [&]() {
      if (!have_eb) { make_eb(); have_eb = true; }
      if (lane == 0) wc[NW_FACES] += (unsigned)nbf;
      const int per = 3 * npf;
      // nodes of every face of the batch into the frame; the loads of all of
      // them are issued before any is used
      float smx = 0.f;
#pragma unroll
      for (int fi = 0; fi < NEAR_FB; ++fi) {
        if (fi < nbf) {
          const double* src = in.surf + (long long)fid[fi] * per;
          for (int r = lane; r < per; r += 32) {
            const int nd = r / 3, a = r - nd * 3;
            const float v = (float)(src[r] - eo[a]);
            fnl[fi * per + a * npf + nd] = v;
            smx = fmaxf(smx, fabsf(v));
          }
        }
      }
      // one rounding bound for the batch: the largest coordinate of the
      // element and of any of its faces (a bound for each face, as a
      // face's own largest coordinate is never above it)
      const float sigma = (float)C_SIGMA * Eps<float>::u * fmaxf(Se, warp_max(smx));
      if (lane < nbf) {
        // the face box in the frame, from its outward float box: the two
        // subtractions and the float origin are within 4u of their operands,
        // which the slack covers (it only widens the box)
        const float* fbx = in.fbox + 6 * (long long)fid[lane];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const float o = (float)eo[a], l = fbx[a], h = fbx[3 + a];
          const float sl = 4.0f * 5.9604645e-8f * (fabsf(l) + fabsf(h) + 2.0f * fabsf(o));
          ffb[lane * 8 + a] = (l - o) - sl;
          ffb[lane * 8 + 3 + a] = (h - o) + sl;
        }
      }
      __syncwarp();
      for (int k = lane; k < nbf * ntf; k += 32) {
        const int fi = k / ntf, ts = k - fi * ntf;
        const float* fx = fnl + fi * per;
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int nd = s_ft[q - 1][ts][c];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const float v = fx[a * npf + nd];
            lo[a] = fminf(lo[a], v);
            hi[a] = fmaxf(hi[a], v);
          }
        }
        float* fbo = fb + fi * 6 * ntf;
#pragma unroll
        for (int a = 0; a < 3; ++a) { fbo[a * ntf + ts] = lo[a]; fbo[(3 + a) * ntf + ts] = hi[a]; }
      }
      __syncwarp();
      for (int base = 0; base < nbf * nte && !fringe; base += 32) {
        // (face, element triangle) of this chunk whose boxes come within tol, compacted
        const int k = base + lane;
        bool near = false;
        int code = 0;
        if (k < nbf * nte) {
          const int fi = k / nte, te = k - fi * nte;
          const float* fr = ffb + fi * 8;
          near = box_dist<float>(eb[te], eb[nte + te], eb[2 * nte + te], eb[3 * nte + te], eb[4 * nte + te],
                                 eb[5 * nte + te], fr[0], fr[1], fr[2], fr[3], fr[4], fr[5]) - sigma <= tolf;
          code = (fi << 16) | te;
        }
        const unsigned em = __ballot_sync(FULL, near);
        if (near) ci[__popc(em & ((1u << lane) - 1u))] = code;
        const int nnear = __popc(em);
        __syncwarp();
        for (int g0 = 0; g0 < nnear && !fringe; g0 += G) {
          const int kk2 = g0 + lk;
          bool keep2 = false;
          int c2 = 0;
          if (lvalid && kk2 < nnear) {
            c2 = ci[kk2];
            const int fi = c2 >> 16, tk = c2 & 0xffff;
            const float* fbo = fb + fi * 6 * ntf;
            keep2 = box_dist<float>(eb[tk], eb[nte + tk], eb[2 * nte + tk], eb[3 * nte + tk], eb[4 * nte + tk],
                                    eb[5 * nte + tk], fbo[lts], fbo[ntf + lts], fbo[2 * ntf + lts],
                                    fbo[3 * ntf + lts], fbo[4 * ntf + lts], fbo[5 * ntf + lts]) - sigma <= tolf;
          }
          const unsigned m2 = __ballot_sync(FULL, keep2);
          if (keep2)
            pq[nq + __popc(m2 & ((1u << lane) - 1u))] = ((c2 >> 16) << 16) | ((c2 & 0xffff) << 8) | lts;
          nq += __popc(m2);
          __syncwarp();
          if (nq >= 32) drain(32);
        }
        __syncwarp();
      }
      if (!fringe && nq > 0) drain(nq);
      nq = 0;
      nbf = 0;
      __syncwarp();
    };
    // gather the faces of up to 32 bins at a time into the face list (lane j
    // reads bin cb + j, a warp scan numbers their faces, the lanes walk the
    // faces in steps of 32), then run the list's batches; a list that fills
    // up is tested before gathering resumes where it stopped
    int cb = 0, kbase = 0;
    while (cb < nbins && !fringe) {
      int nfl = 0;
      while (cb < nbins) {
        const int j = cb + lane;
        int bf0 = 0, bcnt = 0;
        if (j < nbins) {
          const int bx = b0[0] + j % nbx, by = b0[1] + (j / nbx) % nby, bz = b0[2] + j / (nbx * nby);
          const int bi = (bz * in.bdims[1] + by) * in.bdims[0] + bx;
          bf0 = in.bin_off[bi];
          bcnt = in.bin_off[bi + 1] - bf0;
        }
        int incl = bcnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int v = __shfl_up_sync(FULL, incl, d);
          if (lane >= d) incl += v;
        }
        const int excl = incl - bcnt, total = __shfl_sync(FULL, incl, 31);
        for (; kbase < total && nfl <= NEAR_FLCAP - 32; kbase += 32) {
          const int k = kbase + lane, kk = min(k, total - 1);
          int src = 0;
#pragma unroll
          for (int step = 16; step; step >>= 1) {
            const int c = src + step;
            if (__shfl_sync(FULL, excl, c) <= kk) src = c;
          }
          const int fsrc = __shfl_sync(FULL, bf0, src), esrc = __shfl_sync(FULL, excl, src);
          bool keep = false;
          int f = 0;
          if (k < total) {
            const int pos = fsrc + (kk - esrc);
            f = in.bin_faces[pos];
            const float* fbx = in.bin_fbox + 6 * (long long)pos;
            float bb[6] = {fbx[0], fbx[1], fbx[2], fbx[3], fbx[4], fbx[5]};
            float fm = 0.f;
#pragma unroll
            for (int a = 0; a < 6; ++a) fm = fmaxf(fm, fabsf(bb[a]));
            float lb = box_dist<float>(gbox[0], gbox[1], gbox[2], gbox[3], gbox[4], gbox[5], bb[0], bb[1], bb[2],
                                       bb[3], bb[4], bb[5]);
            lb -= 8.0f * 5.9604645e-8f * fmaxf(gmax, fm);  // rounding of the float box distance
            keep = lb <= tolf;
          }
          // the kept faces join the list in lane order
          const unsigned km = __ballot_sync(FULL, keep);
          if (keep) fl[nfl + __popc(km & ((1u << lane) - 1u))] = f;
          nfl += __popc(km);
        }
        if (kbase < total) break;  // the list is full: test it, then resume here
        cb += 32;
        kbase = 0;
      }
      __syncwarp();
      for (int s0 = 0; s0 < nfl && !fringe; s0 += NEAR_FB) {
        fid = fl + s0;
        nbf = min(NEAR_FB, nfl - s0);
        run_batch();
      }
    }
    if (!fringe && nul > 0) settle();
    if (lane == 0) {
      if (fringe) {
        in.flags[e] = DC_FRINGE_;
        wc[NW_FRINGE] += 1u;
      } else if (any_in || any_out) {
        in.flags[e] = any_in ? DC_HOLE_ : DC_FIELD_;
        wc[NW_HOLE] += any_in;
        wc[NW_FIELD] += !any_in;
      }
    }
    // no label and not fringe: the side needs the full search
    if (!fringe && !any_in && !any_out) full_one(ent);
    __syncwarp();
  }
  if (lane == 0) {
    const unsigned n_fringe = wc[NW_FRINGE], n_hole = wc[NW_HOLE], n_field = wc[NW_FIELD], n_faces = wc[NW_FACES];
    if (wc[NW_FS]) atomicAdd(&nb.cnt[3], (unsigned long long)wc[NW_FS]);
    if (n_fringe | n_hole | n_field) {
      atomicAdd(&gcnt[3], (unsigned long long)n_fringe);
      atomicAdd(&gcnt[4], (unsigned long long)n_hole);
      atomicAdd(&gcnt[5], (unsigned long long)n_field);
    }
    if (n_faces) {
      atomicAdd(&nb.cnt[0], (unsigned long long)n_faces);
      atomicAdd(&gcnt[0], (unsigned long long)n_faces);
      atomicAdd(&gcnt[1], (unsigned long long)wc[NW_PAIRS]);
      atomicAdd(&nb.cnt[5], (unsigned long long)wc[NW_FULL]);
      atomicAdd(&gcnt[2], (unsigned long long)wc[NW_RE]);
    }
  }
}

}  // namespace dc
