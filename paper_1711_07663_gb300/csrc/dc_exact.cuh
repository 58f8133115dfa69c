// dc_exact.cuh -- exact element-surface distance and side decision (a6-a9).
//
// Sec. 4.2 of the paper: for each element that the filters leave, faces are
// ranked by an approximate distance (box distance + 0.01 x centroid distance,
// Alg. cp0 / bboxdix), then the linearised element and face triangles are
// compared with a triangle-triangle distance (the modified Moller test of
// Alg. cp1 / cp2, tol = 1e-7); the nearest face's outward normal, averaged
// over faces at the same distance, gives the side.
//
// What differs from the paper's kernels, and why (the result is the exact
// minimum instead of a truncated search):
//   * no fixed N_F^1 = 16 / N_F^2 = 4 truncation and no nearest-corner halving:
//     faces are visited in the paper's ranking order but pruned only by a
//     certified bound (box distance > best distance so far), so no face that
//     can hold the minimum is ever dropped;
//   * the bulk of the triangle pairs is evaluated in FP32 in a frame centred on
//     the element, returning an upper bound U (distance between two computed
//     points of the triangles) and a lower bound L (gap between the triangles'
//     projections on the direction joining those points); with the rounding
//     bound sigma = C eps S (S the largest local coordinate), U + sigma and
//     L - sigma bracket the exact distance, so every pair that can reach the
//     minimum (or tie with it) is re-solved in FP64, and only those;
//   * a pair found crossing in FP32 is confirmed in FP64 at once, which settles
//     a fringe element without further search.
// One warp owns one candidate element at a time (persistent kernel, dynamic
// work counter), lanes split the triangle pairs, warp ballots compact the pairs
// that survive box pruning.
#pragma once

#include "dc_prep.cuh"

namespace dc {

template <class T> struct V3 { T x, y, z; };
template <class T> __host__ __device__ __forceinline__ V3<T> mkv(T x, T y, T z) { V3<T> r; r.x = x; r.y = y; r.z = z; return r; }
template <class T> __host__ __device__ __forceinline__ V3<T> operator-(V3<T> a, V3<T> b) { return mkv(a.x - b.x, a.y - b.y, a.z - b.z); }
template <class T> __host__ __device__ __forceinline__ V3<T> operator+(V3<T> a, V3<T> b) { return mkv(a.x + b.x, a.y + b.y, a.z + b.z); }
template <class T> __host__ __device__ __forceinline__ V3<T> operator*(T s, V3<T> a) { return mkv(s * a.x, s * a.y, s * a.z); }
template <class T> __host__ __device__ __forceinline__ T dot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> __host__ __device__ __forceinline__ V3<T> cross(V3<T> a, V3<T> b) {
  return mkv(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
template <class T> __host__ __device__ __forceinline__ T clamp01(T v) { return v < T(0) ? T(0) : (v > T(1) ? T(1) : v); }

template <class T> struct Eps;
template <> struct Eps<float> { static constexpr float u = 5.9604644775390625e-8f; };   // 2^-24
template <> struct Eps<double> { static constexpr double u = 1.1102230246251565e-16; }; // 2^-53
// Rounding bound of the FP32 triangle-pair routine in an element frame: with
// S the largest |local coordinate|, the rounded inputs move every point by at
// most sqrt(3) u S, the two returned points lie within a few u S of points of
// the triangles, and the distance and projection arithmetic adds a few u S
// more, so U + C_SIGMA u S and L - C_SIGMA u S bracket the exact distance.
constexpr double C_SIGMA = 64.0;

// Closest points of segments p + s d1 and q + t d2 (s, t in [0,1]): minimise
// the convex quadratic along s for the infinite lines, clamp, take the best t
// for that s, and if t had to be clamped re-take the best s for the clamped t.
template <class T>
__host__ __device__ __forceinline__ T seg_seg2(V3<T> p, V3<T> d1, V3<T> q, V3<T> d2, V3<T>& cp, V3<T>& cq) {
  V3<T> r = p - q;
  T a = dot(d1, d1), e = dot(d2, d2), f = dot(d2, r);
  T c = dot(d1, r), b = dot(d1, d2);
  T s, t;
  if (!(a > T(0)) && !(e > T(0))) {
    s = T(0); t = T(0);
  } else if (!(a > T(0))) {
    s = T(0); t = clamp01(f / e);
  } else if (!(e > T(0))) {
    t = T(0); s = clamp01(-c / a);
  } else {
    T den = a * e - b * b;
    s = den > T(0) ? clamp01((b * f - c * e) / den) : T(0);
    t = (b * s + f) / e;
    if (t < T(0)) { t = T(0); s = clamp01(-c / a); }
    else if (t > T(1)) { t = T(1); s = clamp01((b - c) / a); }
  }
  cp = p + s * d1;
  cq = q + t * d2;
  V3<T> w = cp - cq;
  return dot(w, w);
}

// Is X (on the plane of triangle v0 v1 v2 with normal n) inside the triangle?
template <class T>
__host__ __device__ __forceinline__ bool in_tri(V3<T> X, V3<T> v0, V3<T> v1, V3<T> v2, V3<T> n) {
  return dot(cross(v1 - v0, X - v0), n) >= T(0) && dot(cross(v2 - v1, X - v1), n) >= T(0) &&
         dot(cross(v0 - v2, X - v2), n) >= T(0);
}

// Triangle-triangle distance.  U: distance between the returned points ca (on
// triangle a) and cb (on b), 0 when an edge of one crosses the other; L: lower
// bound, the gap between the projections of both triangles on (cb - ca).
// xcode: -1, or which edge crossed: 0..2 edge j of b (b[j] -> b[j+1]) through
// a, 3..5 edge j of a through b.  UNROLL unrolls the vertex loops (vertices in
// registers, for kernels with registers to spare); the arithmetic is the same.
template <class T, bool UNROLL = false>
__host__ __device__ void tritri(const V3<T> a[3], const V3<T> b[3], T& U, T& L, V3<T>& ca, V3<T>& cb, int& xcode) {
  xcode = -1;
  V3<T> na = cross(a[1] - a[0], a[2] - a[0]);
  V3<T> nb = cross(b[1] - b[0], b[2] - b[0]);
  T sb[3], sa[3];
#pragma unroll (UNROLL ? 3 : 1)
  for (int j = 0; j < 3; ++j) { sb[j] = dot(na, b[j] - a[0]); sa[j] = dot(nb, a[j] - b[0]); }
  bool sepB = (sb[0] > T(0) && sb[1] > T(0) && sb[2] > T(0)) || (sb[0] < T(0) && sb[1] < T(0) && sb[2] < T(0));
  bool sepA = (sa[0] > T(0) && sa[1] > T(0) && sa[2] > T(0)) || (sa[0] < T(0) && sa[1] < T(0) && sa[2] < T(0));
  if (!sepA && !sepB) {
    // an edge of one triangle that reaches both sides of the other's plane,
    // crossing it inside the other triangle
    for (int j = 0; j < 3; ++j) {
      T s0 = sb[j], s1 = sb[(j + 1) % 3];
      if (((s0 <= T(0) && s1 >= T(0)) || (s0 >= T(0) && s1 <= T(0))) && s0 != s1) {
        V3<T> X = b[j] + (s0 / (s0 - s1)) * (b[(j + 1) % 3] - b[j]);
        if (in_tri(X, a[0], a[1], a[2], na)) { U = T(0); L = T(0); ca = X; cb = X; xcode = j; return; }
      }
      s0 = sa[j]; s1 = sa[(j + 1) % 3];
      if (((s0 <= T(0) && s1 >= T(0)) || (s0 >= T(0) && s1 <= T(0))) && s0 != s1) {
        V3<T> X = a[j] + (s0 / (s0 - s1)) * (a[(j + 1) % 3] - a[j]);
        if (in_tri(X, b[0], b[1], b[2], nb)) { U = T(0); L = T(0); ca = X; cb = X; xcode = 3 + j; return; }
      }
    }
  }
  T best = T(INFINITY);
  T na2 = dot(na, na), nb2 = dot(nb, nb);
  // vertex of one triangle over the interior of the other
  if (na2 > T(0)) {
#pragma unroll (UNROLL ? 3 : 1)
    for (int j = 0; j < 3; ++j) {
      V3<T> X = b[j] - (sb[j] / na2) * na;
      if (in_tri(X, a[0], a[1], a[2], na)) {
        V3<T> w = b[j] - X;
        T d2 = dot(w, w);
        if (d2 < best) { best = d2; ca = X; cb = b[j]; }
      }
    }
  }
  if (nb2 > T(0)) {
#pragma unroll (UNROLL ? 3 : 1)
    for (int j = 0; j < 3; ++j) {
      V3<T> X = a[j] - (sa[j] / nb2) * nb;
      if (in_tri(X, b[0], b[1], b[2], nb)) {
        V3<T> w = a[j] - X;
        T d2 = dot(w, w);
        if (d2 < best) { best = d2; ca = a[j]; cb = X; }
      }
    }
  }
  // edge pairs
#pragma unroll (UNROLL ? 3 : 1)
  for (int i = 0; i < 3; ++i) {
    V3<T> d1 = a[(i + 1) % 3] - a[i];
#pragma unroll (UNROLL ? 3 : 1)
    for (int j = 0; j < 3; ++j) {
      V3<T> cp, cq;
      T d2 = seg_seg2(a[i], d1, b[j], b[(j + 1) % 3] - b[j], cp, cq);
      if (d2 < best) { best = d2; ca = cp; cb = cq; }
    }
  }
  V3<T> w = cb - ca;
  U = sqrt(dot(w, w));
  if (U > T(0)) {
    V3<T> wh = (T(1) / U) * w;
    T bmin = dot(wh, b[0]), amax = dot(wh, a[0]);
    bmin = fmin(bmin, dot(wh, b[1])); bmin = fmin(bmin, dot(wh, b[2]));
    amax = fmax(amax, dot(wh, a[1])); amax = fmax(amax, dot(wh, a[2]));
    L = fmax(bmin - amax, T(0));
  } else {
    L = T(0);
  }
}

// Signed volume (x6) of tetrahedron (a, b, c, d) and a bound on how far it can
// move when every point is displaced by at most rho, plus the rounding of its
// evaluation: its gradient with respect to each point is a cross product of
// two edge vectors (|.| <= Lm^2, and <= 3 Lm^2 for a), so the first-order
// change is <= 6 rho Lm^2; the second-order term is <= 12 rho^2 Lm; three
// subtractions, a cross and a dot round to within 16 u Lm^3.
template <class T>
__device__ __forceinline__ T orient_cert(V3<T> a, V3<T> b, V3<T> c, V3<T> d, T rho, T& bound) {
  V3<T> e1 = b - a, e2 = c - a, e3 = d - a;
  T l2 = fmax(dot(e1, e1), fmax(dot(e2, e2), dot(e3, e3)));
  T Lm = sqrt(l2) * T(1.0001) + T(2) * rho;
  bound = T(8) * rho * Lm * Lm + T(16) * rho * rho * Lm + T(32) * Eps<T>::u * Lm * Lm * Lm;
  return dot(cross(e1, e2), e3);
}

// Certified crossing: segment PQ meets triangle (t0,t1,t2) for every placement
// of the five points within rho of the given ones (the rounded local copies of
// the FP64 input): P and Q strictly on opposite sides of the plane and the line
// PQ strictly inside the three edges, each signed volume exceeding its bound.
// Then the FP64 triangles intersect and their distance is exactly 0.
// (certified_cross_inl: the same test inlined, for callers whose live
// registers would otherwise be saved and restored around the call)
template <class T>
__device__ __forceinline__ bool certified_cross_inl(V3<T> P, V3<T> Q, V3<T> t0, V3<T> t1, V3<T> t2, T rho) {
  T b1, b2, c1, c2, c3;
  T o1 = orient_cert(t0, t1, t2, P, rho, b1);
  T o2 = orient_cert(t0, t1, t2, Q, rho, b2);
  if (!((o1 > b1 && o2 < -b2) || (o1 < -b1 && o2 > b2))) return false;
  T s1 = orient_cert(P, Q, t0, t1, rho, c1);
  T s2 = orient_cert(P, Q, t1, t2, rho, c2);
  T s3 = orient_cert(P, Q, t2, t0, rho, c3);
  return (s1 > c1 && s2 > c2 && s3 > c3) || (s1 < -c1 && s2 < -c2 && s3 < -c3);
}
template <class T>
__device__ __noinline__ bool certified_cross(V3<T> P, V3<T> Q, V3<T> t0, V3<T> t1, V3<T> t2, T rho) {
  return certified_cross_inl<T>(P, Q, t0, t1, t2, rho);
}

// ------------------------------------------------------------------ per-warp scratch
constexpr int FMAX = 128;   // gathered-face list
constexpr int QCAP = 64;    // pair queue (two batches)
constexpr int RCAP = 64;    // FP64 re-solve list

struct ExLayout {
  int en, ebox, fn, fbx, flist, queue, rlist, rres, total;
};
__host__ __device__ constexpr int align16(int x) { return (x + 15) & ~15; }
__host__ __device__ inline ExLayout ex_layout(int pmax, int qmax, int tsize) {
  int npe = (pmax + 1) * (pmax + 1) * (pmax + 1), nte = 12 * pmax * pmax;
  int npf = (qmax + 1) * (qmax + 1), ntf = 2 * qmax * qmax;
  ExLayout L;
  int o = 0;
  L.en = o; o = align16(o + 3 * npe * tsize);
  L.ebox = o; o = align16(o + 6 * nte * tsize);
  L.fn = o; o = align16(o + 3 * npf * tsize);
  L.fbx = o; o = align16(o + 6 * ntf * tsize);
  L.flist = o; o = align16(o + FMAX * 12);
  L.queue = o; o = align16(o + QCAP * 4);
  L.rlist = o; o = align16(o + RCAP * 12);
  L.rres = o; o = align16(o + RCAP * 7 * 8);
  L.total = o;
  return L;
}

struct ExCounters {
  unsigned long long faces, bulk, recheck, fringe, hole, field, fallback;
};

// Per-warp context, in shared memory: what one element's search reads
// (written by lane 0 when the warp takes the element).
template <class T>
struct WarpCtx {
  const Inst* in;
  long long e;
  int p, npe, nte, q, npf, ntf;
  double o[3];         // frame origin (centre of the element box), global coords
  float gbox[6];       // element box, global, float (rounded outward)
  T* ex; T* ey; T* ez;               // element nodes, local
  T* eb;                             // element triangle boxes [6][nte]
  T* fx; T* fy; T* fz;               // current face nodes, local
  T* fb;                             // face triangle boxes [6][ntf]
  int* fl_id; float* fl_key; float* fl_lb;  // gathered-face list
  int* queue;
  int* rl_face; unsigned* rl_tt; float* rl_lc;  // re-solve list: face, (te << 16 | ts), lower bound
  double* rres;                      // [RCAP][7]: d, ce xyz, cs xyz
  T Se;                              // largest |local coordinate| of the element
};

// Warp-uniform search state, in registers (every lane holds the same values)
template <class T>
struct WarpState {
  int lane;
  T Ucert;                           // certified upper bound on d(E) (search threshold)
  int nfl, nq, nrl;
  bool near_mode;                    // only decide d(E) <= tol (the side is known)
  bool labeled;                      // the hole map gave the side: ties are not needed
  bool overflow, fringe_done;
  unsigned fmask;                    // element faces whose triangles take part (bit f; 0x3f: all)
  double d_fringe;
  double dmin64;                     // FP64 minimum over re-solve entries already flushed
  T U32;                             // smallest bulk-precision pair distance (no margin)
};

template <class T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
  for (int s = 16; s; s >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, s));
  return v;
}
template <class T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int s = 16; s; s >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, s));
  return v;
}

template <class T>
__device__ __forceinline__ T box_dist(T alx, T aly, T alz, T ahx, T ahy, T ahz, T blx, T bly, T blz, T bhx, T bhy, T bhz) {
  T dx = fmax(fmax(blx - ahx, alx - bhx), T(0));
  T dy = fmax(fmax(bly - ahy, aly - bhy), T(0));
  T dz = fmax(fmax(blz - ahz, alz - bhz), T(0));
  return sqrt(dx * dx + dy * dy + dz * dz);
}

// FP64 triangle pair (element triangle te, surface triangle ts of face f) in
// the element frame
__device__ __noinline__ void pair64(const Inst& in, long long e, int p, int q, int te, long long f, int ts,
                                    const double* o, double* out) {
  const int npe = (p + 1) * (p + 1) * (p + 1), npf = (q + 1) * (q + 1);
  const double* en = in.nodes + e * npe * 3;
  const double* fn = in.surf + f * npf * 3;
  V3<double> a[3], b[3];
  for (int c = 0; c < 3; ++c) {
    int ni = c_etri[p - 1][te][c], nj = c_ftri[q - 1][ts][c];
    a[c] = mkv(en[3 * ni] - o[0], en[3 * ni + 1] - o[1], en[3 * ni + 2] - o[2]);
    b[c] = mkv(fn[3 * nj] - o[0], fn[3 * nj + 1] - o[1], fn[3 * nj + 2] - o[2]);
  }
  double U, L;
  V3<double> ca, cb;
  int xc;
  tritri<double>(a, b, U, L, ca, cb, xc);
  out[0] = U; out[1] = ca.x; out[2] = ca.y; out[3] = ca.z; out[4] = cb.x; out[5] = cb.y; out[6] = cb.z;
}

// FP64 re-solve of the listed pairs into a running minimum (lanes in
// parallel); used when the list fills and the side is already known
template <class T>
__device__ __noinline__ void flush_list(WarpCtx<T>& W, WarpState<T>& S, ExCounters& cnt) {
  const int lane = S.lane;
  double dmin = S.dmin64;
  for (int base = 0; base < S.nrl; base += 32) {
    int i = base + lane;
    if (i < S.nrl && W.rl_lc[i] <= (float)S.Ucert) {
      unsigned tt = W.rl_tt[i];
      double r[7];
      pair64(*W.in, W.e, W.p, W.q, (int)(tt >> 16), W.rl_face[i], (int)(tt & 0xffffu), W.o, r);
      dmin = fmin(dmin, r[0]);
    }
  }
  cnt.recheck += (unsigned long long)S.nrl;
  S.dmin64 = warp_min(dmin);
  S.nrl = 0;
  __syncwarp();
}

// evaluate the queued pairs of face f (n <= 32), lanes in parallel
template <class T>
__device__ __noinline__ void eval_batch(WarpCtx<T>& W, WarpState<T>& S, int n, int f, T sigma, T rho, ExCounters& cnt) {
  const unsigned FULL = 0xffffffffu;
  const int lane = S.lane;
  T Uc = T(INFINITY), Lc = T(INFINITY), Ur = T(INFINITY);
  int te = 0, ts = 0;
  bool cert = false, zero = false;
  if (lane < n) {
    int idx = W.queue[lane];
    te = idx / W.ntf;
    ts = idx - te * W.ntf;
    V3<T> a[3], b[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      int ni = c_etri[W.p - 1][te][c], nj = c_ftri[W.q - 1][ts][c];
      a[c] = mkv(W.ex[ni], W.ey[ni], W.ez[ni]);
      b[c] = mkv(W.fx[nj], W.fy[nj], W.fz[nj]);
    }
    T U, L;
    V3<T> ca, cb;
    int xc;
    tritri<T>(a, b, U, L, ca, cb, xc);
    if (xc >= 0) {
      // a crossing: certify it against the rounding of the local copies
      const V3<T>* s = (xc < 3) ? b : a;
      const V3<T>* t = (xc < 3) ? a : b;
      int j = xc % 3;
      cert = certified_cross<T>(s[j], s[(j + 1) % 3], t[0], t[1], t[2], rho);
    }
    Uc = U + sigma;
    Lc = L - sigma;
    Ur = U;
    zero = (U == T(0));
  }
  cnt.bulk += (unsigned long long)n;
  S.U32 = fmin(S.U32, warp_min(Ur));
  if (__any_sync(FULL, cert)) {
    S.fringe_done = true;
    S.d_fringe = 0.0;
    S.Ucert = T(0);
    __syncwarp();
    return;
  }
  if (S.near_mode) {
    // only "is some pair within tol" matters: settle undecided pairs in FP64
    unsigned amb = __ballot_sync(FULL, (lane < n) && (Lc <= (T)W.in->tol));
    while (amb) {
      int src = __ffs(amb) - 1;
      amb &= amb - 1;
      int cte = __shfl_sync(FULL, te, src), cts = __shfl_sync(FULL, ts, src);
      double d64 = 0.0;
      if (lane == 0) {
        double r[7];
        pair64(*W.in, W.e, W.p, W.q, cte, f, cts, W.o, r);
        d64 = r[0];
      }
      d64 = __shfl_sync(FULL, d64, 0);
      cnt.recheck += 1;
      if (d64 <= W.in->tol) {
        S.fringe_done = true;
        S.d_fringe = d64;
        break;
      }
    }
    __syncwarp();
    return;
  }
  // a pair at distance exactly 0 without an edge crossing (coplanar contact):
  // confirm in FP64; a zero distance settles the element (d(E) = 0)
  unsigned zm = __ballot_sync(FULL, zero);
  if (zm) {
    int src = __ffs(zm) - 1;
    int cte = __shfl_sync(FULL, te, src), cts = __shfl_sync(FULL, ts, src);
    double d64 = 0.0;
    if (sizeof(T) == 4) {
      if (lane == 0) {
        double r[7];
        pair64(*W.in, W.e, W.p, W.q, cte, f, cts, W.o, r);
        d64 = r[0];
      }
      d64 = __shfl_sync(FULL, d64, 0);
      cnt.recheck += 1;
    }
    if (d64 == 0.0) {
      S.fringe_done = true;
      S.d_fringe = 0.0;
      S.Ucert = T(0);
      __syncwarp();
      return;
    }
  }
  S.Ucert = fmin(S.Ucert, warp_min(Uc));
  // keep the pairs that may reach the minimum for the FP64 re-solve
  bool keep = (lane < n) && (Lc <= S.Ucert);
  unsigned km = __ballot_sync(FULL, keep);
  int nk = __popc(km);
  if (nk && S.nrl + nk > RCAP) {
    // compact: drop entries the improved bound has excluded
    __syncwarp();
    int w = 0;
    for (int base = 0; base < S.nrl; base += 32) {
      int i = base + lane;
      bool k2 = i < S.nrl && W.rl_lc[i] <= (float)S.Ucert;
      int fi = 0; unsigned tt = 0; float lc = 0.f;
      if (i < S.nrl) { fi = W.rl_face[i]; tt = W.rl_tt[i]; lc = W.rl_lc[i]; }
      unsigned m2 = __ballot_sync(FULL, k2);
      __syncwarp();
      if (k2) {
        int pos = w + __popc(m2 & ((1u << lane) - 1u));
        W.rl_face[pos] = fi; W.rl_tt[pos] = tt; W.rl_lc[pos] = lc;
      }
      w += __popc(m2);
      __syncwarp();
    }
    S.nrl = w;
  }
  if (nk && S.nrl + nk > RCAP && S.labeled) {
    // the side is known, only the minimum matters: re-solve what is listed now
    flush_list<T>(W, S, cnt);
  }
  if (nk) {
    if (S.nrl + nk > RCAP) {
      S.overflow = true;
    } else {
      if (keep) {
        int pos = S.nrl + __popc(km & ((1u << lane) - 1u));
        W.rl_face[pos] = f;
        W.rl_tt[pos] = ((unsigned)te << 16) | (unsigned)ts;
        W.rl_lc[pos] = (float)Lc;
      }
      S.nrl += nk;
    }
  }
  __syncwarp();
}

// test the triangle pairs of face f against the element: element triangles
// are first pruned against the face's box, then pairs against each other;
// `thr` is the current threshold (tol in near mode, the best bound otherwise)
template <class T>
__device__ __noinline__ void process_face(WarpCtx<T>& W, WarpState<T>& S, int f, ExCounters& cnt) {
  const unsigned FULL = 0xffffffffu;
  const Inst& in = *W.in;
  const int lane = S.lane;
  const double* fn = in.surf + (long long)f * W.npf * 3;
  T smax = T(0);
  T flo[3] = {T(INFINITY), T(INFINITY), T(INFINITY)}, fhi[3] = {-T(INFINITY), -T(INFINITY), -T(INFINITY)};
  for (int k = lane; k < W.npf * 3; k += 32) {
    int nd = k / 3, a = k - nd * 3;
    T v = (T)(fn[k] - W.o[a]);
    (a == 0 ? W.fx : (a == 1 ? W.fy : W.fz))[nd] = v;
    smax = fmax(smax, fabs(v));
    flo[a] = fmin(flo[a], v);
    fhi[a] = fmax(fhi[a], v);
  }
  smax = warp_max(smax);
  for (int a = 0; a < 3; ++a) { flo[a] = warp_min(flo[a]); fhi[a] = warp_max(fhi[a]); }
  __syncwarp();
  for (int t = lane; t < W.ntf; t += 32) {
    T lo[3] = {T(INFINITY), T(INFINITY), T(INFINITY)}, hi[3] = {-T(INFINITY), -T(INFINITY), -T(INFINITY)};
    for (int c = 0; c < 3; ++c) {
      int nd = c_ftri[W.q - 1][t][c];
      T v[3] = {W.fx[nd], W.fy[nd], W.fz[nd]};
      for (int a = 0; a < 3; ++a) { lo[a] = fmin(lo[a], v[a]); hi[a] = fmax(hi[a], v[a]); }
    }
    for (int a = 0; a < 3; ++a) { W.fb[a * W.ntf + t] = lo[a]; W.fb[(3 + a) * W.ntf + t] = hi[a]; }
  }
  __syncwarp();
  const T Smag = fmax(W.Se, smax);
  const T sigma = (T)C_SIGMA * Eps<T>::u * Smag;
  const T rho = T(2) * Eps<T>::u * Smag;
  const int nte = W.nte, ntf = W.ntf, tpf = nte / 6;
  S.nq = 0;
  for (int t0 = 0; t0 < nte; t0 += 32) {
    // element triangles of this chunk near the face box
    int te = t0 + lane;
    bool near = false;
    if (te < nte && ((S.fmask >> (te / tpf)) & 1u)) {
      T lb = box_dist<T>(W.eb[te], W.eb[nte + te], W.eb[2 * nte + te], W.eb[3 * nte + te], W.eb[4 * nte + te],
                         W.eb[5 * nte + te], flo[0], flo[1], flo[2], fhi[0], fhi[1], fhi[2]);
      near = lb - sigma <= S.Ucert;
    }
    unsigned em = __ballot_sync(FULL, near);
    const int P = __popc(em) * ntf;
    for (int base = 0; base < P; base += 32) {
      int idx = base + lane;
      bool keep = false;
      int pi = 0;
      if (idx < P) {
        int k = idx / ntf, ts = idx - k * ntf;
        int tk = t0 + (int)__fns(em, 0, k + 1);
        T lb = box_dist<T>(W.eb[tk], W.eb[nte + tk], W.eb[2 * nte + tk], W.eb[3 * nte + tk], W.eb[4 * nte + tk],
                           W.eb[5 * nte + tk], W.fb[ts], W.fb[ntf + ts], W.fb[2 * ntf + ts], W.fb[3 * ntf + ts],
                           W.fb[4 * ntf + ts], W.fb[5 * ntf + ts]);
        keep = lb - sigma <= S.Ucert;
        pi = tk * ntf + ts;
      }
      unsigned m = __ballot_sync(FULL, keep);
      if (keep) W.queue[S.nq + __popc(m & ((1u << lane) - 1u))] = pi;
      S.nq += __popc(m);
      __syncwarp();
      if (S.nq >= 32) {
        eval_batch<T>(W, S, 32, f, sigma, rho, cnt);
        if (S.fringe_done) { S.nq = 0; return; }
        int rem = S.nq - 32;
        int v = (lane < rem) ? W.queue[32 + lane] : 0;
        __syncwarp();
        if (lane < rem) W.queue[lane] = v;
        S.nq = rem;
        __syncwarp();
      }
    }
  }
  if (S.nq > 0) eval_batch<T>(W, S, S.nq, f, sigma, rho, cnt);
  S.nq = 0;
  cnt.faces += 1;
}

// process the gathered faces in the paper's ranking order (box distance +
// 0.01 x centre distance), skipping those the current bound excludes
template <class T>
__device__ void process_list(WarpCtx<T>& W, WarpState<T>& S, ExCounters& cnt) {
  const unsigned FULL = 0xffffffffu;
  const int lane = S.lane;
  while (!S.fringe_done) {
    float bk = INFINITY;
    int bi = -1;
    for (int i = lane; i < S.nfl; i += 32)
      if (W.fl_key[i] < bk) { bk = W.fl_key[i]; bi = i; }
#pragma unroll
    for (int s = 16; s; s >>= 1) {
      float ok = __shfl_xor_sync(FULL, bk, s);
      int oi = __shfl_xor_sync(FULL, bi, s);
      if (ok < bk || (ok == bk && oi >= 0 && (bi < 0 || oi < bi))) { bk = ok; bi = oi; }
    }
    if (bi < 0) break;
    float lb = W.fl_lb[bi];
    int f = W.fl_id[bi];
    __syncwarp();
    if (lane == 0) W.fl_key[bi] = INFINITY;
    __syncwarp();
    if (isinf(bk)) break;
    if ((T)lb <= S.Ucert) process_face<T>(W, S, f, cnt);
  }
  S.nfl = 0;
  __syncwarp();
}

// side of an element from its FP64 tie set: ties sharing a surface closest
// point form a group whose normal is the angle-weighted average of its
// triangles' normals; across groups the largest |cos| decides (Sec. 4.1/4.2)
__device__ double tri_weight(const double* v, const double* x, double eps) {
  for (int k = 0; k < 3; ++k) {
    double dx = x[0] - v[3 * k], dy = x[1] - v[3 * k + 1], dz = x[2] - v[3 * k + 2];
    if (sqrt(dx * dx + dy * dy + dz * dz) <= eps) {
      int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
      double e1[3], e2[3];
      for (int a = 0; a < 3; ++a) { e1[a] = v[3 * k1 + a] - v[3 * k + a]; e2[a] = v[3 * k2 + a] - v[3 * k + a]; }
      double c = (e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2]) /
                 (sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]) * sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]));
      return acos(fmin(1.0, fmax(-1.0, c)));
    }
  }
  for (int k = 0; k < 3; ++k) {
    int k1 = (k + 1) % 3;
    double d[3], w[3];
    for (int a = 0; a < 3; ++a) { d[a] = v[3 * k1 + a] - v[3 * k + a]; w[a] = x[a] - v[3 * k + a]; }
    double L2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double t = L2 > 0.0 ? fmin(1.0, fmax(0.0, (w[0] * d[0] + w[1] * d[1] + w[2] * d[2]) / L2)) : 0.0;
    double r0 = w[0] - t * d[0], r1 = w[1] - t * d[1], r2 = w[2] - t * d[2];
    if (sqrt(r0 * r0 + r1 * r1 + r2 * r2) <= eps) return 3.14159265358979323846;
  }
  return 2.0 * 3.14159265358979323846;
}

__device__ __noinline__ int side_of(const Inst& in, int q, const double* o, const int* rl_face, const unsigned* rl_tt,
                                    const double* rres, int nt, double lim, double eps) {
  // rres rows: d, ce, cs (element frame)
  unsigned long long grouped[RCAP / 64 + 1] = {0ull};
  double best_mag = -1.0;
  int best_sign = 1;
  const int npf = (q + 1) * (q + 1);
  for (int i = 0; i < nt; ++i) {
    const double* ri = rres + 7 * i;
    if (ri[0] > lim || ((grouped[i >> 6] >> (i & 63)) & 1ull)) continue;
    double nsum[3] = {0.0, 0.0, 0.0};
    int lead = i;
    for (int j = i; j < nt; ++j) {
      const double* rj = rres + 7 * j;
      if (rj[0] > lim || ((grouped[j >> 6] >> (j & 63)) & 1ull)) continue;
      double dx = rj[4] - ri[4], dy = rj[5] - ri[5], dz = rj[6] - ri[6];
      if (sqrt(dx * dx + dy * dy + dz * dz) > eps) continue;
      grouped[j >> 6] |= 1ull << (j & 63);
      if (rj[0] < rres[7 * lead]) lead = j;
      // skip a surface triangle already counted in this group
      int fj = rl_face[j], tj = (int)(rl_tt[j] & 0xffffu);
      bool dup = false;
      for (int k = i; k < j; ++k) {
        const double* rk = rres + 7 * k;
        if (rk[0] > lim) continue;
        double ex = rk[4] - ri[4], ey = rk[5] - ri[5], ez = rk[6] - ri[6];
        if (sqrt(ex * ex + ey * ey + ez * ez) > eps) continue;
        if (rl_face[k] == fj && (int)(rl_tt[k] & 0xffffu) == tj) { dup = true; break; }
      }
      if (dup) continue;
      const double* fn = in.surf + (long long)fj * npf * 3;
      double v[9];
      for (int c = 0; c < 3; ++c) {
        int nd = c_ftri[q - 1][tj][c];
        for (int a = 0; a < 3; ++a) v[3 * c + a] = fn[3 * nd + a] - o[a];
      }
      double e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]}, e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
      double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
      double ln = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      if (!(ln > 0.0)) continue;
      double wgt = tri_weight(v, ri + 4, eps) / ln;
      for (int a = 0; a < 3; ++a) nsum[a] += wgt * n[a];
    }
    const double* rl = rres + 7 * lead;
    double vv[3] = {rl[1] - rl[4], rl[2] - rl[5], rl[3] - rl[6]};
    double den = sqrt(vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2]) *
                 sqrt(nsum[0] * nsum[0] + nsum[1] * nsum[1] + nsum[2] * nsum[2]);
    double c = den > 0.0 ? (vv[0] * nsum[0] + vv[1] * nsum[1] + vv[2] * nsum[2]) / den : 0.0;
    if (fabs(c) > best_mag) { best_mag = fabs(c); best_sign = c > 0.0 ? 1 : -1; }
  }
  return best_sign;
}

// gather the faces whose boxes come within radius r of the element box (bins
// not yet visited) into the face list, processing the list whenever it fills
template <class T>
__device__ void gather_round(WarpCtx<T>& W, WarpState<T>& S, double r, const float* fext, int* b0, int* b1, const int* pb0,
                             const int* pb1, ExCounters& cnt) {
  const unsigned FULL = 0xffffffffu;
  const Inst& in = *W.in;
  const int lane = S.lane;
  float gmax = 0.f;
  for (int a = 0; a < 6; ++a) gmax = fmaxf(gmax, fabsf(W.gbox[a]));
  const float ecx = 0.5f * (W.gbox[0] + W.gbox[3]), ecy = 0.5f * (W.gbox[1] + W.gbox[4]), ecz = 0.5f * (W.gbox[2] + W.gbox[5]);
  for (int a = 0; a < 3; ++a) {
    // float bin range, widened by 1e-3 bin plus the rounding of its inputs
    float rf = (float)r * 1.0001f;
    float glo = W.gbox[a] - rf - fext[a], ghi = W.gbox[3 + a] + rf;
    float o = in.origin_f[a];
    float slack = 1e-3f + 16.0f * 5.9604645e-8f * (fabsf(glo) + fabsf(ghi) + fabsf(o)) * in.inv_bs_f;
    b0[a] = clampi(cube_floor((double)((glo - o) * in.inv_bs_f - slack), in.bdims[a]), 0, in.bdims[a] - 1);
    b1[a] = clampi(cube_floor((double)((ghi - o) * in.inv_bs_f + slack), in.bdims[a]), 0, in.bdims[a] - 1);
  }
  for (int bz = b0[2]; bz <= b1[2] && !S.fringe_done; ++bz)
    for (int by = b0[1]; by <= b1[1] && !S.fringe_done; ++by)
      for (int bx = b0[0]; bx <= b1[0] && !S.fringe_done; ++bx) {
        if (bx >= pb0[0] && bx <= pb1[0] && by >= pb0[1] && by <= pb1[1] && bz >= pb0[2] && bz <= pb1[2]) continue;
        int bi = (bz * in.bdims[1] + by) * in.bdims[0] + bx;
        int f0 = in.bin_off[bi], f1 = in.bin_off[bi + 1];
        for (int base = f0; base < f1; base += 32) {
          int k = base + lane;
          bool keep = false;
          int f = 0;
          float lb = 0.f, key = 0.f;
          if (k < f1) {
            f = in.bin_faces[k];
            const float* fb = in.bin_fbox + 6 * (long long)k;  // the box beside the id
            float b[6] = {fb[0], fb[1], fb[2], fb[3], fb[4], fb[5]};
            float fm = 0.f;
            for (int a = 0; a < 6; ++a) fm = fmaxf(fm, fabsf(b[a]));
            lb = box_dist<float>(W.gbox[0], W.gbox[1], W.gbox[2], W.gbox[3], W.gbox[4], W.gbox[5], b[0], b[1], b[2],
                                 b[3], b[4], b[5]);
            lb -= 8.0f * 5.9604645e-8f * fmaxf(gmax, fm);  // rounding of the float box distance
            float cx = 0.5f * (b[0] + b[3]) - ecx, cy = 0.5f * (b[1] + b[4]) - ecy, cz = 0.5f * (b[2] + b[5]) - ecz;
            key = fmaxf(lb, 0.f) + 0.01f * sqrtf(cx * cx + cy * cy + cz * cz);  // Alg. cp0 ranking
            keep = (T)lb <= S.Ucert;
          }
          unsigned m = __ballot_sync(FULL, keep);
          int nk = __popc(m);
          if (S.nfl + nk > FMAX) {
            process_list<T>(W, S, cnt);
            if (S.fringe_done) break;
          }
          if (keep) {
            int pos = S.nfl + __popc(m & ((1u << lane) - 1u));
            W.fl_id[pos] = f;
            W.fl_key[pos] = key;
            W.fl_lb[pos] = lb;
          }
          S.nfl += nk;
          __syncwarp();
        }
      }
  if (!S.fringe_done) process_list<T>(W, S, cnt);
}

// one candidate element; returns false when it must be redone in FP64
template <class T>
__device__ bool process_element(WarpCtx<T>& W, WarpState<T>& S, ExCounters& cnt) {
  const unsigned FULL = 0xffffffffu;
  const Inst& in = *W.in;
  const int lane = S.lane;
  const long long e = W.e;
  const float* gb = in.eaabb + 6 * e;
  if (lane == 0) {
    for (int a = 0; a < 6; ++a) W.gbox[a] = gb[a];
    for (int a = 0; a < 3; ++a) W.o[a] = 0.5 * ((double)gb[a] + (double)gb[3 + a]);
  }
  __syncwarp();
  const double* en = in.nodes + e * W.npe * 3;
  T smax = T(0);
  for (int k = lane; k < W.npe * 3; k += 32) {
    int nd = k / 3, a = k - nd * 3;
    T v = (T)(en[k] - W.o[a]);
    (a == 0 ? W.ex : (a == 1 ? W.ey : W.ez))[nd] = v;
    smax = fmax(smax, fabs(v));
  }
  smax = warp_max(smax);
  if (lane == 0) W.Se = smax;
  __syncwarp();
  // side labels of the element's nodes from the hole map (node = frame
  // origin + local coordinate, in float; margin in cube units for rounding)
  int lab_or = 0;
  {
    const float ox = (float)W.o[0], oy = (float)W.o[1], oz = (float)W.o[2];
    const float gm = fmaxf(fmaxf(fabsf(ox), fabsf(oy)), fabsf(oz)) + (float)smax;
    const float m = 1e-5f + 16.0f * 5.9604645e-8f * gm * in.inv_ds_f;
    for (int nd = lane; nd < W.npe; nd += 32)
      lab_or |= point_label(in, ox + (float)W.ex[nd], oy + (float)W.ey[nd], oz + (float)W.ez[nd], m);
  }
  const bool any_in = __any_sync(FULL, lab_or & 1), any_out = __any_sync(FULL, lab_or & 2);
  int8_t flag;
  double dist = 0.0;
  S.Ucert = T(INFINITY);
  S.nfl = 0;
  S.nq = 0;
  S.nrl = 0;
  S.overflow = false;
  S.fringe_done = false;
  S.d_fringe = 0.0;
  S.near_mode = false;
  S.fmask = 0x3fu;
  S.labeled = any_in != any_out;
  S.dmin64 = INFINITY;
  S.U32 = T(INFINITY);
  if (any_in && any_out) {
    // nodes on both sides: the closed element boundary crosses the surface
    flag = DC_FRINGE_;
    dist = 0.0;
  } else {
    __syncwarp();
    for (int t = lane; t < W.nte; t += 32) {
      T lo[3] = {T(INFINITY), T(INFINITY), T(INFINITY)}, hi[3] = {-T(INFINITY), -T(INFINITY), -T(INFINITY)};
      for (int c = 0; c < 3; ++c) {
        int nd = c_etri[W.p - 1][t][c];
        T v[3] = {W.ex[nd], W.ey[nd], W.ez[nd]};
        for (int a = 0; a < 3; ++a) { lo[a] = fmin(lo[a], v[a]); hi[a] = fmax(hi[a], v[a]); }
      }
      for (int a = 0; a < 3; ++a) { W.eb[a * W.nte + t] = lo[a]; W.eb[(3 + a) * W.nte + t] = hi[a]; }
    }
    __syncwarp();
    const float fext[3] = {__uint_as_float(in.fext_bits[0]), __uint_as_float(in.fext_bits[1]),
                           __uint_as_float(in.fext_bits[2])};
    int pb0[3] = {1, 1, 1}, pb1[3] = {0, 0, 0}, b0[3], b1[3];
    if (!in.want_dist && (any_in || any_out)) {
      // the side is known: only "does any pair come within tol" is left
      S.near_mode = true;
      S.Ucert = (T)in.tol;
      gather_round<T>(W, S, in.tol, fext, b0, b1, pb0, pb1, cnt);
      flag = S.fringe_done ? DC_FRINGE_ : (any_in ? DC_HOLE_ : DC_FIELD_);
    } else {
      double r = 0.0;
      bool converged = false;
      for (int round = 0; round < 40 && !S.fringe_done; ++round) {
        gather_round<T>(W, S, r, fext, b0, b1, pb0, pb1, cnt);
        for (int a = 0; a < 3; ++a) { pb0[a] = b0[a]; pb1[a] = b1[a]; }
        if (S.fringe_done) { converged = true; break; }
        double U = (double)S.Ucert;
        if (U < INFINITY) {
          bool covered = true;
          for (int a = 0; a < 3; ++a) {
            double need_lo = (double)W.gbox[a] - U - (double)fext[a], need_hi = (double)W.gbox[3 + a] + U;
            if (b0[a] > 0 && in.origin[a] + b0[a] * in.bs > need_lo - 1e-9 * in.bs) covered = false;
            if (b1[a] < in.bdims[a] - 1 && in.origin[a] + (b1[a] + 1) * in.bs < need_hi + 1e-9 * in.bs) covered = false;
          }
          if (covered) { converged = true; break; }
          r = fmax(U, r);
        } else {
          r = (r == 0.0) ? in.bs : 2.0 * r;
        }
      }
      if (!converged && lane == 0) atomicOr((int*)&in.err, (int)ERR_ROUNDS);
      if (S.fringe_done) {
        flag = DC_FRINGE_;
        dist = S.d_fringe;
      } else {
        if (S.overflow) return false;
        // keep only the entries the final bound admits
        int w = 0;
        for (int base = 0; base < S.nrl; base += 32) {
          int i = base + lane;
          bool k2 = i < S.nrl && W.rl_lc[i] <= (float)S.Ucert;
          int fi = 0; unsigned tt = 0; float lc = 0.f;
          if (i < S.nrl) { fi = W.rl_face[i]; tt = W.rl_tt[i]; lc = W.rl_lc[i]; }
          unsigned m2 = __ballot_sync(FULL, k2);
          __syncwarp();
          if (k2) {
            int pos = w + __popc(m2 & ((1u << lane) - 1u));
            W.rl_face[pos] = fi; W.rl_tt[pos] = tt; W.rl_lc[pos] = lc;
          }
          w += __popc(m2);
          __syncwarp();
        }
        S.nrl = w;
        // FP64 re-solve
        double dmin = INFINITY;
        for (int base = 0; base < S.nrl; base += 32) {
          int i = base + lane;
          if (i < S.nrl) {
            unsigned tt = W.rl_tt[i];
            double* rr = W.rres + 7 * i;
            pair64(in, e, W.p, W.q, (int)(tt >> 16), W.rl_face[i], (int)(tt & 0xffffu), W.o, rr);
            dmin = fmin(dmin, rr[0]);
          }
        }
        cnt.recheck += (unsigned long long)S.nrl;
        dmin = fmin(warp_min(dmin), S.dmin64);
        __syncwarp();
        if (dmin <= in.tol) {
          flag = DC_FRINGE_;
          dist = dmin;
        } else if (S.labeled) {
          flag = any_in ? DC_HOLE_ : DC_FIELD_;
          dist = any_in ? -dmin : dmin;
        } else {
          int sgn = 1;
          if (lane == 0) {
            double scale = fmax((double)W.gbox[3] - W.gbox[0], fmax((double)W.gbox[4] - W.gbox[1], (double)W.gbox[5] - W.gbox[2]));
            sgn = side_of(in, W.q, W.o, W.rl_face, W.rl_tt, W.rres, S.nrl, dmin * (1.0 + 1e-9) + 1e-14, 1e-9 * scale);
          }
          sgn = __shfl_sync(FULL, sgn, 0);
          flag = sgn > 0 ? DC_FIELD_ : DC_HOLE_;
          dist = sgn > 0 ? dmin : -dmin;
        }
      }
    }
  }
  if (lane == 0) {
    in.flags[e] = flag;
    if (in.dist) in.dist[e] = dist;
    if (in.dist32) {
      // the bulk stage's own distance (FP32 instantiation only; an element
      // settled by its node labels alone computed none)
      const bool have = sizeof(T) == 4 && S.U32 < T(INFINITY);
      in.dist32[e] = have ? (dist < 0.0 ? -(float)S.U32 : (float)S.U32) : __int_as_float(0x7fc00000);
    }
  }
  if (flag == DC_FRINGE_) cnt.fringe++;
  else if (flag == DC_HOLE_) cnt.hole++;
  else cnt.field++;
  return true;
}

// Persistent exact-test kernel over a candidate list.  Elements whose FP32
// re-solve list overflowed are appended to `redo` for an FP64 pass.
template <class T>
__global__ void __launch_bounds__(256, 2) k_exact(Inst* __restrict__ I, CandList cl, CandList redo, int pmax, int qmax,
                                                  unsigned long long* __restrict__ gcnt) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const ExLayout Lo = ex_layout(pmax, qmax, (int)sizeof(T));
  __shared__ WarpCtx<T> s_ctx[8];
  unsigned char* ws = smem + (size_t)wid * Lo.total;
  WarpCtx<T>& W = s_ctx[wid];
  WarpState<T> S;
  S.lane = lane;
  if (lane == 0) {
    W.ex = reinterpret_cast<T*>(ws + Lo.en);
    W.eb = reinterpret_cast<T*>(ws + Lo.ebox);
    W.fx = reinterpret_cast<T*>(ws + Lo.fn);
    W.fb = reinterpret_cast<T*>(ws + Lo.fbx);
    W.fl_id = reinterpret_cast<int*>(ws + Lo.flist);
    W.fl_key = reinterpret_cast<float*>(W.fl_id + FMAX);
    W.fl_lb = W.fl_key + FMAX;
    W.queue = reinterpret_cast<int*>(ws + Lo.queue);
    W.rl_face = reinterpret_cast<int*>(ws + Lo.rlist);
    W.rl_tt = reinterpret_cast<unsigned*>(W.rl_face + RCAP);
    W.rl_lc = reinterpret_cast<float*>(W.rl_tt + RCAP);
    W.rres = reinterpret_cast<double*>(ws + Lo.rres);
  }
  __syncwarp();
  ExCounters cnt = {0, 0, 0, 0, 0, 0, 0};
  unsigned long long ncand = cl.count[0];
  if (ncand > cl.cap) ncand = cl.cap;
  while (true) {
    unsigned long long w = 0;
    if (lane == 0) w = atomicAdd(&cl.count[1], 1ull);
    w = __shfl_sync(FULL, w, 0);
    if (w >= ncand) break;
    unsigned long long ent = cl.cand[w];
    int ii = (int)(ent >> 40);
    __syncwarp();
    if (lane == 0) {
      W.in = &I[ii];
      W.e = (long long)(ent & ((1ull << 40) - 1ull));
      W.p = I[ii].p;
      W.q = I[ii].q;
      W.npe = (W.p + 1) * (W.p + 1) * (W.p + 1);
      W.nte = 12 * W.p * W.p;
      W.npf = (W.q + 1) * (W.q + 1);
      W.ntf = 2 * W.q * W.q;
      W.ey = W.ex + W.npe;
      W.ez = W.ey + W.npe;
      W.fy = W.fx + W.npf;
      W.fz = W.fy + W.npf;
    }
    __syncwarp();
    bool ok = process_element<T>(W, S, cnt);
    if (!ok) {
      if (sizeof(T) == 4) {
        // FP32 re-solve list overflowed: the element is redone by the FP64 pass
        cnt.fallback++;
        if (lane == 0) {
          unsigned long long pos = atomicAdd(&redo.count[0], 1ull);
          if (pos < redo.cap) redo.cand[pos] = ent;
        }
      } else if (lane == 0) {
        atomicOr((int*)&I[ii].err, (int)ERR_RECHECK);
      }
    }
    __syncwarp();
  }
  if (lane == 0) {
    atomicAdd(&gcnt[0], cnt.faces);
    atomicAdd(&gcnt[1], cnt.bulk);
    atomicAdd(&gcnt[2], cnt.recheck);
    atomicAdd(&gcnt[3], cnt.fringe);
    atomicAdd(&gcnt[4], cnt.hole);
    atomicAdd(&gcnt[5], cnt.field);
    atomicAdd(&gcnt[6], cnt.fallback);
  }
}

}  // namespace dc
