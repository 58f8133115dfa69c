// dc_heur.cuh -- the paper's truncating variant of the exact stage
// (DC_HEURISTIC), to compare its answers and its cost with the exact cut.
//
// Sec. 4.2 with Alg. cp0 / bboxdix / cp1 / cp2, for every candidate element:
//   * OBB of the element's 8 corner nodes: axes = eigenvectors of the corner
//     covariance (cyclic Jacobi), box of the rotated corners;
//   * Alg. cp0 key of every face of the surface: 0.01 x centroid distance +
//     distance between the OBB and the box of the face's rotated corners; the
//     16 smallest keys are kept (N_F^1, ties: lower face id);
//   * Alg. cp1 on each of them: the element corner nearest to the face's
//     centroid (lowest index on ties), distance D1 between the corner triangles
//     of the three element faces at that corner and the face's two corner
//     triangles, 0 below tol; the 4 smallest D1 are kept (N_F^2, ties: key
//     order);
//   * Alg. cp2: the order-p triangles of the three element faces at each kept
//     face's corner against the face's 2q^2 triangles; below tol: fringe,
//     otherwise the side rule on the pairs at the smallest distance.
// Every decision is taken as the FP64 computation would take it: the key scan
// runs in FP32 on world coordinates and keeps 24 faces, which are re-ranked in
// FP64 (certified by the FP32 error bound, else the element is rescanned in
// FP64); pass 1 runs in FP32 in the element frame with certified bounds and
// certified crossings, and the faces those cannot zero or order are re-solved
// in FP64; pass 2 is the
// exact stage's certified FP32 search with FP64 re-solves, restricted to the
// kept faces and their corner faces (k_heur_final).
#pragma once

#include "dc_exact.cuh"

namespace dc {

constexpr int HEUR_NF1 = 16;   // N_F^1
constexpr int HEUR_NF2 = 4;    // N_F^2
constexpr int HEUR_K = 24;     // FP32 key buffer (>= N_F^1, certified re-rank)
constexpr int HEUR_SEL = 8;    // ints per candidate in the selection array

// per face of an instance: 4 corner nodes (12 floats, world), the corners'
// mean (3), the face's largest |coordinate| (1)
__global__ void k_heur_faces(Inst* __restrict__ I) {
  pdl_enter();
  Inst& in = I[blockIdx.y];
  const int q = in.q, npf = (q + 1) * (q + 1);
  const int fc[4] = {0, q, npf - 1, q * (q + 1)};
  for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < in.n_faces;
       f += (long long)gridDim.x * blockDim.x) {
    const double* fn = in.surf + f * npf * 3;
    float* o = in.hface + 16 * f;
    double s[3] = {0.0, 0.0, 0.0};
    float m = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double v = fn[3 * fc[c] + a];
        s[a] += v;
        o[3 * c + a] = (float)v;
        m = fmaxf(m, fabsf((float)v));
      }
#pragma unroll
    for (int a = 0; a < 3; ++a) o[12 + a] = (float)(s[a] * 0.25);
    o[15] = m;
    atomicMax((int*)&in.hmax_bits, __float_as_int(m));
  }
}

// element node of corner c = i + 2j + 4k: (i p, j p, k p)
__device__ __forceinline__ int heur_corner_node(int p, int c) {
  const int i = (c & 1) * p, j = ((c >> 1) & 1) * p, k = ((c >> 2) & 1) * p;
  return i + (p + 1) * (j + (p + 1) * k);
}

// node (a, b) of element face f (0 xi-, 1 xi+, 2 eta-, 3 eta+, 4 zeta-, 5 zeta+),
// (a, b) over the two free directions in (xi, eta, zeta) order
__device__ __forceinline__ int heur_face_node(int p, int f, int a, int b) {
  const int fix = (f & 1) ? p : 0;
  const int ax = f >> 1;
  const int i = ax == 0 ? fix : a;
  const int j = ax == 0 ? a : (ax == 1 ? fix : b);
  const int k = ax == 2 ? fix : b;
  return i + (p + 1) * (j + (p + 1) * k);
}

// element corner triangle h of the corner quad of element face f:
// (00, 10, 11) or (00, 11, 01) over corner nodes
__device__ __forceinline__ void heur_ctri(int p, int f, int h, int nd[3]) {
  const int n00 = heur_face_node(p, f, 0, 0), n10 = heur_face_node(p, f, p, 0);
  const int n11 = heur_face_node(p, f, p, p), n01 = heur_face_node(p, f, 0, p);
  nd[0] = n00;
  nd[1] = h ? n11 : n10;
  nd[2] = h ? n01 : n11;
}

// cyclic Jacobi on a symmetric 3x3 (every lane the same values): rotations
// applied to A and accumulated into V (columns: eigenvectors once A is
// diagonal), until the off-diagonal sum is below rel x the diagonal sum
template <class T>
__device__ void heur_jacobi(T A[3][3], T V[3][3], int sweeps, T rel) {
  for (int sweep = 0; sweep < sweeps; ++sweep) {
    const T off = fabs(A[0][1]) + fabs(A[0][2]) + fabs(A[1][2]);
    const T scale = fabs(A[0][0]) + fabs(A[1][1]) + fabs(A[2][2]);
    if (off <= rel * scale || off == T(0)) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (A[p][q] == T(0)) continue;
        const T theta = (A[q][q] - A[p][p]) / (T(2) * A[p][q]);
        const T t = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
        const T c = T(1) / sqrt(t * t + T(1)), s = t * c;
        for (int k = 0; k < 3; ++k) {
          const T akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {
          const T apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          const T vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
}

// Alg. cp0 key in FP64 from the face's FP64 nodes
__device__ double heur_key64(const double R[9], const double Be[6], const double ecg[3], const double* fn, int q) {
  const int npf = (q + 1) * (q + 1);
  const int fc[4] = {0, q, npf - 1, q * (q + 1)};
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  double s[3] = {0.0, 0.0, 0.0};
  for (int c = 0; c < 4; ++c) {
    const double* x = fn + 3 * fc[c];
    for (int a = 0; a < 3; ++a) s[a] += x[a];
    for (int r = 0; r < 3; ++r) {
      const double v = R[3 * r] * x[0] + R[3 * r + 1] * x[1] + R[3 * r + 2] * x[2];
      lo[r] = fmin(lo[r], v);
      hi[r] = fmax(hi[r], v);
    }
  }
  double D = 0.0;
  for (int a = 0; a < 3; ++a)
    if (hi[a] < Be[a] || Be[3 + a] < lo[a]) {
      const double d = fmax(Be[a] - hi[a], lo[a] - Be[3 + a]);
      D += d * d;
    }
  const double dx = s[0] * 0.25 - ecg[0], dy = s[1] * 0.25 - ecg[1], dz = s[2] * 0.25 - ecg[2];
  return 0.01 * sqrt(dx * dx + dy * dy + dz * dz) + sqrt(D);
}

__device__ __forceinline__ bool heur_less(double ka, int ia, double kb, int ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// insert (k, id) into the sorted list held by lanes 0..n-1 (one entry per lane)
template <class K>
__device__ __forceinline__ void heur_insert(K& tk, int& ti, K k, int id, int n, int lane) {
  const unsigned FULL = 0xffffffffu;
  const bool below = lane < n && (tk < k || (tk == k && ti < id));
  const int pos = __popc(__ballot_sync(FULL, below));
  const K uk = __shfl_up_sync(FULL, tk, 1);
  const int ui = __shfl_up_sync(FULL, ti, 1);
  if (lane < n && lane > pos) { tk = uk; ti = ui; }
  if (lane == pos && pos < n) { tk = k; ti = id; }
}

// bitonic sort of one (key, id) entry per lane, ascending
__device__ __forceinline__ void heur_sort32(double& k, int& id, int lane) {
  const unsigned FULL = 0xffffffffu;
  for (int size = 2; size <= 32; size <<= 1)
    for (int stride = size >> 1; stride; stride >>= 1) {
      const double ok = __shfl_xor_sync(FULL, k, stride);
      const int oi = __shfl_xor_sync(FULL, id, stride);
      const bool up = (lane & size) == 0;
      const bool lower = (lane & stride) == 0;
      const bool other_less = heur_less(ok, oi, k, id);
      const bool take = lower == up ? other_less : !other_less && !(ok == k && oi == id);
      if (take) { k = ok; id = oi; }
    }
}

// FP64 D1 of one kept face: the 12 corner-triangle pairs on lanes 0..11
__device__ double heur_d1_64(const Inst& in, long long e, int p, int q, long long f, int c, const double* o, int lane) {
  const int npe = (p + 1) * (p + 1) * (p + 1), npf = (q + 1) * (q + 1);
  const int fc[4] = {0, q, npf - 1, q * (q + 1)};
  double d = INFINITY;
  if (lane < 12) {
    const int s = lane >> 2, h = (lane >> 1) & 1, j = lane & 1;
    const int fsel = s == 0 ? (c & 1) : (s == 1 ? 2 + ((c >> 1) & 1) : 4 + ((c >> 2) & 1));
    int nd[3];
    heur_ctri(p, fsel, h, nd);
    const double* en = in.nodes + e * npe * 3;
    const double* fn = in.surf + f * npf * 3;
    const int tf[3] = {fc[0], j ? fc[2] : fc[1], j ? fc[3] : fc[2]};
    V3<double> a[3], b[3];
    for (int v = 0; v < 3; ++v) {
      a[v] = mkv(en[3 * nd[v]] - o[0], en[3 * nd[v] + 1] - o[1], en[3 * nd[v] + 2] - o[2]);
      b[v] = mkv(fn[3 * tf[v]] - o[0], fn[3 * tf[v] + 1] - o[1], fn[3 * tf[v] + 2] - o[2]);
    }
    double U, L;
    V3<double> ca, cb;
    int xc;
    tritri<double>(a, b, U, L, ca, cb, xc);
    d = U;
  }
  return warp_min(d);
}

// One warp per candidate: OBB, keys, the 16 nearest faces, pass 1, the 4
// nearest.  sel[HEUR_SEL * w]: n2, 4 faces, corners (4 bits each), status.
// cnt[0] FP64 key rescans, [1] pass-1 FP64 re-solves.
__global__ void __launch_bounds__(256, 2) k_heur_select(Inst* __restrict__ I, CandList cl, int* __restrict__ sel,
                                                        unsigned long long* __restrict__ cnt) {
  pdl_enter();
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __shared__ float s_fc[8][HEUR_NF1][12];  // kept faces' corners in the element frame
  __shared__ float s_lo[8][HEUR_NF1], s_hi[8][HEUR_NF1];
  // the FP64 OBB (axes R[9], box Be[6], centroid[3]) and corners of each
  // warp's element, parked here during the face scan (registers are short)
  __shared__ double s_obb[8][18];
  __shared__ double s_cor[8][8][3];
  const unsigned long long ncand = cl.count[0] < cl.cap ? cl.count[0] : cl.cap;
  unsigned long long n_rescan = 0, n_resolve = 0;
  for (unsigned long long w = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + wid; w < ncand;
       w += (unsigned long long)gridDim.x * (blockDim.x >> 5)) {
    const unsigned long long ent = cl.cand[w];
    const Inst& in = I[(int)(ent >> 40)];
    const long long e = (long long)(ent & ((1ull << 40) - 1ull));
    const int p = in.p, q = in.q, npe = (p + 1) * (p + 1) * (p + 1), npf = (q + 1) * (q + 1);
    const long long nf = in.n_faces;
    float Rf[9], Bef[6], ecf[3], Xe = 0.f;
    {
    // corners (lane c < 8), FP64 world
    const double* en = in.nodes + e * npe * 3;
    double cx = 0.0, cy = 0.0, cz = 0.0;
    if (lane < 8) {
      const int nd = heur_corner_node(p, lane);
      cx = en[3 * nd]; cy = en[3 * nd + 1]; cz = en[3 * nd + 2];
    }
    double sx = cx, sy = cy, sz = cz;
#pragma unroll
    for (int s = 4; s; s >>= 1) {
      sx += __shfl_xor_sync(FULL, sx, s);
      sy += __shfl_xor_sync(FULL, sy, s);
      sz += __shfl_xor_sync(FULL, sz, s);
    }
    sx = __shfl_sync(FULL, sx, 0); sy = __shfl_sync(FULL, sy, 0); sz = __shfl_sync(FULL, sz, 0);
    const double ecg[3] = {sx * 0.125, sy * 0.125, sz * 0.125};
    double cv[6] = {0, 0, 0, 0, 0, 0};
    if (lane < 8) {
      const double dx = cx - ecg[0], dy = cy - ecg[1], dz = cz - ecg[2];
      cv[0] = dx * dx / 8.0; cv[1] = dx * dy / 8.0; cv[2] = dx * dz / 8.0;
      cv[3] = dy * dy / 8.0; cv[4] = dy * dz / 8.0; cv[5] = dz * dz / 8.0;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
#pragma unroll
      for (int s = 4; s; s >>= 1) cv[k] += __shfl_xor_sync(FULL, cv[k], s);
      cv[k] = __shfl_sync(FULL, cv[k], 0);
    }
    // eigenvectors: Jacobi in FP32 from the identity, then FP64 sweeps on
    // V32^T A V32 (already nearly diagonal) to the FP64 tolerance; the OBB key
    // does not depend on the order or sign of the axes
    double A[3][3] = {{cv[0], cv[1], cv[2]}, {cv[1], cv[3], cv[4]}, {cv[2], cv[4], cv[5]}}, V[3][3];
    {
      float Af[3][3], Vf[3][3];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) { Af[i][j] = (float)A[i][j]; Vf[i][j] = i == j ? 1.f : 0.f; }
      heur_jacobi<float>(Af, Vf, 20, 1e-7f);
      double B[3][3];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          V[i][j] = (double)Vf[i][j];
          double acc = 0.0;
          for (int k = 0; k < 3; ++k) acc += A[i][k] * (double)Vf[k][j];
          B[i][j] = acc;
        }
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          double acc = 0.0;
          for (int k = 0; k < 3; ++k) acc += (double)Vf[k][i] * B[k][j];
          A[i][j] = acc;
        }
      heur_jacobi<double>(A, V, 50, 1e-15);
    }
    double R[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int a = 0; a < 3; ++a) R[3 * r + a] = V[a][r];
    double Be[6];
    {
      double rv[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) rv[r] = R[3 * r] * cx + R[3 * r + 1] * cy + R[3 * r + 2] * cz;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        double lo = lane < 8 ? rv[r] : INFINITY, hi = lane < 8 ? rv[r] : -INFINITY;
        lo = warp_min(lo);
        hi = warp_max(hi);
        Be[r] = lo;
        Be[3 + r] = hi;
      }
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) Rf[k] = (float)R[k];
#pragma unroll
    for (int k = 0; k < 6; ++k) Bef[k] = (float)Be[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) ecf[k] = (float)ecg[k];
    {
      float m = lane < 8 ? fmaxf(fabsf((float)cx), fmaxf(fabsf((float)cy), fabsf((float)cz))) : 0.f;
      Xe = warp_max(m);
    }
    if (lane == 0) {
      for (int k = 0; k < 9; ++k) s_obb[wid][k] = R[k];
      for (int k = 0; k < 6; ++k) s_obb[wid][9 + k] = Be[k];
      for (int k = 0; k < 3; ++k) s_obb[wid][15 + k] = ecg[k];
    }
    if (lane < 8) { s_cor[wid][lane][0] = cx; s_cor[wid][lane][1] = cy; s_cor[wid][lane][2] = cz; }
    }
    __syncwarp();
    const double* R = s_obb[wid];
    const double* Be = R + 9;
    const double* ecg = R + 15;
    // FP32 key scan (world coordinates), the 24 smallest keys in lanes 0..23
    float tk = INFINITY;
    int ti = 0x7fffffff;
    float tau = INFINITY;
    for (long long f0 = 0; f0 < nf; f0 += 32) {
      const long long f = f0 + lane;
      float key = INFINITY;
      if (f < nf) {
        const float4* h4 = reinterpret_cast<const float4*>(in.hface + 16 * f);
        const float4 a0 = __ldg(h4), a1 = __ldg(h4 + 1), a2 = __ldg(h4 + 2), a3 = __ldg(h4 + 3);
        const float X[12] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, a2.x, a2.y, a2.z, a2.w};
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            const float v = Rf[3 * r] * X[3 * c] + Rf[3 * r + 1] * X[3 * c + 1] + Rf[3 * r + 2] * X[3 * c + 2];
            lo[r] = fminf(lo[r], v);
            hi[r] = fmaxf(hi[r], v);
          }
        float D = 0.f;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const float d = fmaxf(fmaxf(Bef[r] - hi[r], lo[r] - Bef[3 + r]), 0.f);
          D += d * d;
        }
        const float dx = a3.x - ecf[0], dy = a3.y - ecf[1], dz = a3.z - ecf[2];
        key = 0.01f * sqrtf(dx * dx + dy * dy + dz * dz) + sqrtf(D);
      }
      unsigned m = __ballot_sync(FULL, key < tau);
      while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const float k = __shfl_sync(FULL, key, src);
        if (!(k < tau)) continue;
        heur_insert<float>(tk, ti, k, (int)(f0 + src), HEUR_K, lane);
        tau = __shfl_sync(FULL, tk, HEUR_K - 1);
      }
    }
    // FP64 re-rank of the buffered faces
    const int nbuf = nf < HEUR_K ? (int)nf : HEUR_K;
    double k64 = INFINITY;
    int id64 = 0x7fffffff;
    if (lane < nbuf && ti >= 0 && (long long)ti < nf) {
      id64 = ti;
      k64 = heur_key64(R, Be, ecg, in.surf + (long long)ti * npf * 3, q);
    }
    heur_sort32(k64, id64, lane);
    const int n1 = nf < HEUR_NF1 ? (int)nf : HEUR_NF1;
    bool certain = true;
    if (nf > HEUR_K) {
      // a face outside the buffer has FP32 key >= tau, hence FP64 key >= tau - eps
      const float Xf = __int_as_float(in.hmax_bits);
      const double eps = 64.0 * (double)Eps<float>::u * ((double)Xe + (double)Xf + 1.0);
      const double k16 = __shfl_sync(FULL, k64, HEUR_NF1 - 1);
      certain = k16 < (double)tau - eps;
    }
    if (!certain) {
      // rescan every face in FP64
      n_rescan += (lane == 0);
      k64 = INFINITY;
      id64 = 0x7fffffff;
      double tau64 = INFINITY;
      for (long long f0 = 0; f0 < nf; f0 += 32) {
        const long long f = f0 + lane;
        const double key = f < nf ? heur_key64(R, Be, ecg, in.surf + f * npf * 3, q) : INFINITY;
        unsigned m = __ballot_sync(FULL, key < tau64);
        while (m) {
          const int src = __ffs(m) - 1;
          m &= m - 1;
          const double k = __shfl_sync(FULL, key, src);
          if (!(k < tau64)) continue;
          heur_insert<double>(k64, id64, k, (int)(f0 + src), HEUR_NF1, lane);
          tau64 = __shfl_sync(FULL, k64, HEUR_NF1 - 1);
        }
      }
    }
    // pass 1: lane i < n1 owns kept face i (rank i); nearest corner in FP64
    // the element frame (origin at the centre of the float box), as the exact
    // stage forms it
    const float* gbx = in.eaabb + 6 * e;
    const double o[3] = {0.5 * ((double)gbx[0] + (double)gbx[3]), 0.5 * ((double)gbx[1] + (double)gbx[4]),
                         0.5 * ((double)gbx[2] + (double)gbx[5])};
    const int fid = id64;
    int corner = 0;
    {
      double fcg[3] = {0.0, 0.0, 0.0};
      const int fcn[4] = {0, q, npf - 1, q * (q + 1)};
      const double* fn = in.surf + (long long)(lane < n1 ? fid : 0) * npf * 3;
      if (lane < n1) {
        for (int c = 0; c < 4; ++c)
          for (int a = 0; a < 3; ++a) fcg[a] += fn[3 * fcn[c] + a];
        for (int a = 0; a < 3; ++a) fcg[a] *= 0.25;
      }
      double best = INFINITY;
      for (int c = 0; c < 8; ++c) {
        const double xc = s_cor[wid][c][0], yc = s_cor[wid][c][1], zc = s_cor[wid][c][2];
        const double dx = xc - fcg[0], dy = yc - fcg[1], dz = zc - fcg[2];
        const double d = dx * dx + dy * dy + dz * dz;  // squared: the same nearest corner
        if (d < best) { best = d; corner = c; }
      }
      if (lane < n1)
        for (int c = 0; c < 4; ++c)
          for (int a = 0; a < 3; ++a) s_fc[wid][lane][3 * c + a] = (float)(fn[3 * fcn[c] + a] - o[a]);
      if (lane < HEUR_NF1) { s_lo[wid][lane] = INFINITY; s_hi[wid][lane] = INFINITY; }
    }
    __syncwarp();
    // FP32 corner-triangle pairs, 12 per kept face, certified bounds per face
    {
      const double* xn = in.nodes + e * 3 * npe;
      for (int base = 0; base < 12 * n1; base += 32) {
        const int P = base + lane;
        const int i = P / 12;
        const int c = __shfl_sync(FULL, corner, i < HEUR_NF1 ? i : 0);
        if (P < 12 * n1) {
          const int rem = P - 12 * i;
          const int s = rem >> 2, h = (rem >> 1) & 1, j = rem & 1;
          const int fsel = s == 0 ? (c & 1) : (s == 1 ? 2 + ((c >> 1) & 1) : 4 + ((c >> 2) & 1));
          int nd[3];
          heur_ctri(p, fsel, h, nd);
          const int tf[3] = {0, j ? 2 : 1, j ? 3 : 2};  // face corners (00, 10, 11, 01) -> triangles
          V3<float> a[3], b[3];
          float S = 0.f;
#pragma unroll
          for (int v = 0; v < 3; ++v) {
            a[v] = mkv((float)(xn[3 * nd[v]] - o[0]), (float)(xn[3 * nd[v] + 1] - o[1]), (float)(xn[3 * nd[v] + 2] - o[2]));
            const float* fc = &s_fc[wid][i][3 * tf[v]];
            b[v] = mkv(fc[0], fc[1], fc[2]);
            S = fmaxf(S, fmaxf(fmaxf(fabsf(a[v].x), fabsf(a[v].y)), fabsf(a[v].z)));
            S = fmaxf(S, fmaxf(fmaxf(fabsf(b[v].x), fabsf(b[v].y)), fabsf(b[v].z)));
          }
          float U, L;
          V3<float> ca, cb;
          int xc;
          tritri<float, false>(a, b, U, L, ca, cb, xc);
          const float sg = (float)C_SIGMA * Eps<float>::u * S;
          float lo = fmaxf(L - sg, 0.f), hi = U + sg;
          if (xc >= 0) {
            // a crossing certified against the rounding of the local copies:
            // the FP64 triangles meet, D1 is exactly 0
            const V3<float>* sv = xc < 3 ? b : a;
            const V3<float>* tv = xc < 3 ? a : b;
            const int jj = xc % 3;
            if (certified_cross<float>(sv[jj], sv[(jj + 1) % 3], tv[0], tv[1], tv[2], 2.f * Eps<float>::u * S)) {
              lo = 0.f;
              hi = 0.f;
            }
          }
          atomicMin((int*)&s_lo[wid][i], __float_as_int(lo));
          atomicMin((int*)&s_hi[wid][i], __float_as_int(hi));
        }
      }
    }
    __syncwarp();
    // D1 per kept face: certified zero, certified nonzero interval, or FP64
    float lo = lane < n1 ? s_lo[wid][lane] : INFINITY, hi = lane < n1 ? s_hi[wid][lane] : INFINITY;
    const float tolf = in.tol_f;
    bool exact = false;
    double v64 = 0.0;
    {
      unsigned um = __ballot_sync(FULL, lane < n1 && !(hi < tolf && (double)hi < in.tol) && !((double)lo >= in.tol));
      while (um) {
        const int src = __ffs(um) - 1;
        um &= um - 1;
        const int fs = __shfl_sync(FULL, fid, src), cs = __shfl_sync(FULL, corner, src);
        const double d = heur_d1_64(in, e, p, q, fs, cs, o, lane);
        n_resolve += (lane == 0);
        if (lane == src) { exact = true; v64 = d; }
      }
    }
    // value classes: zero (0), or the interval [lo, hi] / exact value
    bool zero = lane < n1 && (exact ? v64 < in.tol : (double)hi < in.tol);
    double vlo = exact ? v64 : (double)lo, vhi = exact ? v64 : (double)hi;
    if (zero) { vlo = 0.0; vhi = 0.0; }
    const int nz = __popc(__ballot_sync(FULL, zero));
    const int n2 = n1 < HEUR_NF2 ? n1 : HEUR_NF2;
    bool keep = false;
    if (nz >= n2) {
      // enough zeros: the lowest ranks among them
      const unsigned zmask = __ballot_sync(FULL, zero);  // every lane takes part
      keep = zero && __popc(zmask & ((1u << lane) - 1u)) < n2;
    } else {
      keep = zero;
      const int k = n2 - nz;
      // k-th smallest upper bound among the nonzero faces
      double h = (lane < n1 && !zero) ? vhi : INFINITY;
      int hid = lane;
      heur_sort32(h, hid, lane);
      const double kth = __shfl_sync(FULL, h, k - 1);
      // faces that could be among the k: re-solve those not yet exact
      const bool cand = lane < n1 && !zero && vlo <= kth;
      unsigned rm = __ballot_sync(FULL, cand && !exact);
      const unsigned cm = __ballot_sync(FULL, cand);
      if (__popc(cm) > k && rm) {
        while (rm) {
          const int src = __ffs(rm) - 1;
          rm &= rm - 1;
          const int fs = __shfl_sync(FULL, fid, src), cs = __shfl_sync(FULL, corner, src);
          const double d = heur_d1_64(in, e, p, q, fs, cs, o, lane);
          n_resolve += (lane == 0);
          if (lane == src) { exact = true; v64 = d; vlo = vhi = d; }
        }
      }
      // order the candidates by (value, rank); values are exact where it matters
      double key = cand ? vlo : INFINITY;
      int rk = lane;
      heur_sort32(key, rk, lane);
      unsigned chosen = 0;
      for (int t = 0; t < k; ++t) chosen |= 1u << __shfl_sync(FULL, rk, t);
      keep = keep || ((chosen >> lane) & 1u);
    }
    // the kept faces in (D1, rank) order
    double okey = keep ? (zero ? 0.0 : vlo) : INFINITY;
    int orank = lane;
    heur_sort32(okey, orank, lane);
    const int kf = __shfl_sync(FULL, fid, orank < 32 ? orank : 0);
    const int kc = __shfl_sync(FULL, corner, orank < 32 ? orank : 0);
    int cpack = 0, kfv[HEUR_NF2];
#pragma unroll
    for (int t = 0; t < HEUR_NF2; ++t) {
      cpack |= (__shfl_sync(FULL, kc, t) & 7) << (4 * t);
      const int ft = __shfl_sync(FULL, kf, t);
      kfv[t] = t < n2 ? ft : -1;
    }
    if (lane == 0) {
      int* o8 = sel + HEUR_SEL * w;
      o8[0] = n2;
#pragma unroll
      for (int t = 0; t < HEUR_NF2; ++t) o8[1 + t] = kfv[t];
      o8[5] = cpack;
      o8[6] = certain ? 0 : 1;
      o8[7] = 0;
    }
    __syncwarp();
  }
  if (lane == 0) {
    if (n_rescan) atomicAdd(&cnt[0], n_rescan);
    if (n_resolve) atomicAdd(&cnt[1], n_resolve);
  }
}

// Pass 2 (Alg. cp2) and the decision for one candidate whose kept faces are
// sel8: the exact stage's certified search over the kept faces only, each
// against the triangles of the three element faces at its corner; false when
// the FP32 re-solve list overflowed (the FP64 pass redoes the element).
template <class T>
__device__ bool heur_element(WarpCtx<T>& W, WarpState<T>& S, ExCounters& cnt, const int* sel8) {
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
    const int nd = k / 3, a = k - nd * 3;
    const T v = (T)(en[k] - W.o[a]);
    (a == 0 ? W.ex : (a == 1 ? W.ey : W.ez))[nd] = v;
    smax = fmax(smax, fabs(v));
  }
  smax = warp_max(smax);
  if (lane == 0) W.Se = smax;
  __syncwarp();
  for (int t = lane; t < W.nte; t += 32) {
    T lo[3] = {T(INFINITY), T(INFINITY), T(INFINITY)}, hi[3] = {-T(INFINITY), -T(INFINITY), -T(INFINITY)};
    for (int c = 0; c < 3; ++c) {
      const int nd = c_etri[W.p - 1][t][c];
      const T v[3] = {W.ex[nd], W.ey[nd], W.ez[nd]};
      for (int a = 0; a < 3; ++a) { lo[a] = fmin(lo[a], v[a]); hi[a] = fmax(hi[a], v[a]); }
    }
    for (int a = 0; a < 3; ++a) { W.eb[a * W.nte + t] = lo[a]; W.eb[(3 + a) * W.nte + t] = hi[a]; }
  }
  __syncwarp();
  S.Ucert = T(INFINITY);
  S.nfl = 0;
  S.nq = 0;
  S.nrl = 0;
  S.overflow = false;
  S.fringe_done = false;
  S.d_fringe = 0.0;
  S.near_mode = false;
  S.labeled = false;
  S.dmin64 = INFINITY;
  const int n2 = sel8[0], cpack = sel8[5];
  for (int t = 0; t < n2 && t < HEUR_NF2 && !S.fringe_done; ++t) {
    const int f = sel8[1 + t], c = (cpack >> (4 * t)) & 7;
    if (f < 0 || f >= in.n_faces) continue;
    S.fmask = (1u << (c & 1)) | (1u << (2 + ((c >> 1) & 1))) | (1u << (4 + ((c >> 2) & 1)));
    process_face<T>(W, S, f, cnt);
  }
  S.fmask = 0x3fu;
  int8_t flag;
  double dist;
  if (S.fringe_done) {
    flag = DC_FRINGE_;
    dist = S.d_fringe;
  } else {
    if (S.overflow) return false;
    int w = 0;
    for (int base = 0; base < S.nrl; base += 32) {
      const int i = base + lane;
      const bool k2 = i < S.nrl && W.rl_lc[i] <= (float)S.Ucert;
      int fi = 0;
      unsigned tt = 0;
      float lc = 0.f;
      if (i < S.nrl) { fi = W.rl_face[i]; tt = W.rl_tt[i]; lc = W.rl_lc[i]; }
      const unsigned m2 = __ballot_sync(FULL, k2);
      __syncwarp();
      if (k2) {
        const int pos = w + __popc(m2 & ((1u << lane) - 1u));
        W.rl_face[pos] = fi; W.rl_tt[pos] = tt; W.rl_lc[pos] = lc;
      }
      w += __popc(m2);
      __syncwarp();
    }
    S.nrl = w;
    double dmin = INFINITY;
    for (int base = 0; base < S.nrl; base += 32) {
      const int i = base + lane;
      if (i < S.nrl) {
        const unsigned tt = W.rl_tt[i];
        double* rr = W.rres + 7 * i;
        pair64(in, e, W.p, W.q, (int)(tt >> 16), W.rl_face[i], (int)(tt & 0xffffu), W.o, rr);
        dmin = fmin(dmin, rr[0]);
      }
    }
    cnt.recheck += (unsigned long long)S.nrl;
    dmin = fmin(warp_min(dmin), S.dmin64);
    __syncwarp();
    if (dmin < in.tol) {
      // Alg. cp2: a distance below tol makes the element intersecting
      flag = DC_FRINGE_;
      dist = dmin;
    } else {
      int sgn = 1;
      if (lane == 0) {
        const double scale =
            fmax((double)W.gbox[3] - W.gbox[0], fmax((double)W.gbox[4] - W.gbox[1], (double)W.gbox[5] - W.gbox[2]));
        sgn = side_of(in, W.q, W.o, W.rl_face, W.rl_tt, W.rres, S.nrl, dmin * (1.0 + 1e-9) + 1e-14, 1e-9 * scale);
      }
      sgn = __shfl_sync(FULL, sgn, 0);
      flag = sgn > 0 ? DC_FIELD_ : DC_HOLE_;
      dist = sgn > 0 ? dmin : -dmin;
    }
  }
  if (lane == 0) {
    in.flags[e] = flag;
    if (in.dist) in.dist[e] = dist;
  }
  if (flag == DC_FRINGE_) cnt.fringe++;
  else if (flag == DC_HOLE_) cnt.hole++;
  else cnt.field++;
  return true;
}

// Persistent pass-2 kernel over the candidates (from_redo = 0: the whole
// list, FP32 with FP64 re-solves; 1: the FP64 pass over the candidate indices
// the FP32 pass appended to `redo`).
template <class T>
__global__ void __launch_bounds__(256, 2) k_heur_final(Inst* __restrict__ I, CandList cl, CandList redo,
                                                       const int* __restrict__ sel, int from_redo, int pmax, int qmax,
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
  const CandList& src = from_redo ? redo : cl;
  unsigned long long n = src.count[0];
  if (n > src.cap) n = src.cap;
  while (true) {
    unsigned long long k = 0;
    if (lane == 0) k = atomicAdd(&src.count[1], 1ull);
    k = __shfl_sync(FULL, k, 0);
    if (k >= n) break;
    const unsigned long long w = from_redo ? src.cand[k] : k;
    const unsigned long long ent = cl.cand[w];
    const int ii = (int)(ent >> 40);
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
    const bool ok = heur_element<T>(W, S, cnt, sel + HEUR_SEL * w);
    if (!ok) {
      if (sizeof(T) == 4) {
        cnt.fallback++;
        if (lane == 0) {
          const unsigned long long pos = atomicAdd(&redo.count[0], 1ull);
          if (pos < redo.cap) redo.cand[pos] = w;
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
