// dc_pc.cuh -- donor search for receptor points (the point-connectivity step
// after the cut: "Donor/Receptor Point Connectivity on GPUs", Eqs. reftophys,
// ref-update, Jac).
//
// The donor grid's search tree is built once on the host (dc_pc_create): a
// balanced tree over the elements' boxes, one element per node, split at the
// median of the six box coordinates in turn (as an alternating digital tree
// is), each node holding the box of its subtree for pruning.  The grid moves
// rigidly, so a query point is taken into the grid's initial frame by the
// inverse motion instead of rebuilding the tree.
//
//   k_pc_search  one thread per point: depth-first traversal with a fixed
//                stack (PC_STACK entries: a balanced tree of 2^PC_STACK - 1
//                nodes), the elements whose FP64 box holds the point
//                appended to the point's candidate list (ascending index);
//                no containment work during the traversal, so threads of a
//                warp do not wait on each other's Newton solves;
//   k_pc_newton  one thread per point: its candidates in index order, the
//                clamped Newton inversion of the isoparametric map (FP32 in
//                the element frame, at most 10 steps, then FP64 steps on the
//                original nodes to the acceptance tolerance); the first
//                element that holds the point is its donor.
#pragma once

#include "dc_common.cuh"

namespace dc {

constexpr int PC_STACK = 32;        // traversal stack (trees up to 2^32 - 1 nodes)
constexpr int PC_CAND = 16;         // candidate elements per point
constexpr int PC_ITERS = 10;        // Newton steps (FP32 stage)
constexpr int PC_POLISH = 3;        // FP64 steps after it
constexpr double PC_CLAMP = 1e-4;   // xi is kept within [-1 - PC_CLAMP, 1 + PC_CLAMP]
constexpr double PC_INSIDE = 1e-8;  // accepted when max |xi_a| <= 1 + PC_INSIDE
constexpr double PC_RESID = 1e-10;  // ... and |x - x(xi)| <= PC_RESID h
constexpr int PC_MAXP = 4;

struct PcNode {                     // 64 bytes
  float slo[3]; int elem;           // subtree box (outward float), this node's element
  float shi[3]; int left;           // child nodes (-1: none)
  float elo[3]; int right;          // the element's box (outward float)
  float ehi[3]; int pad;
};

struct PcGrid {
  int p;
  long long n_elem;
  const double* nodes;              // [n_elem][(p+1)^3][3]
  const float* loc;                 // [n_elem][3][(p+1)^3] frame coordinates
  const double* org;                // [n_elem][3] frame origins
  const double* ebox;               // [n_elem][6] FP64 node boxes
  const float* h;                   // [n_elem] largest box side
  const PcNode* tree;
  int root;
};

struct PcQuery {
  long long n;
  const double* pts;                // [n][3], world frame
  int has_pose;
  double pose[12];                  // grid motion [R|t] (initial frame -> world)
  double* xloc;                     // [n][3] points in the grid's initial frame
  int* ncand;                       // [n]
  int* cand;                        // [n][PC_CAND]
  long long* donor;                 // [n]
  double* ref;                      // [n][3]
  unsigned long long* cnt;          // [0] candidates, [1] overflowed points, [2] FP64 steps, [3] found
};

__global__ void __launch_bounds__(256) k_pc_search(PcGrid G, PcQuery Q) {
  unsigned long long n_c = 0, n_over = 0;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < Q.n; k += (long long)gridDim.x * blockDim.x) {
    const double* P = Q.pts + 3 * k;
    double x[3];
    if (Q.has_pose) {
      const double q0 = P[0] - Q.pose[3], q1 = P[1] - Q.pose[7], q2 = P[2] - Q.pose[11];
#pragma unroll
      for (int a = 0; a < 3; ++a) x[a] = __dadd_rn(__dadd_rn(__dmul_rn(Q.pose[a], q0), __dmul_rn(Q.pose[4 + a], q1)),
                                                  __dmul_rn(Q.pose[8 + a], q2));
    } else {
      x[0] = P[0]; x[1] = P[1]; x[2] = P[2];
    }
    Q.xloc[3 * k] = x[0]; Q.xloc[3 * k + 1] = x[1]; Q.xloc[3 * k + 2] = x[2];
    const float xf[3] = {(float)x[0], (float)x[1], (float)x[2]};
    int stack[PC_STACK];
    int sp = 0, nc = 0;
    bool over = false;
    int* cl = Q.cand + (long long)PC_CAND * k;
    if (G.root >= 0) stack[sp++] = G.root;
    while (sp > 0) {
      const int nd = stack[--sp];
      const float4* n4 = reinterpret_cast<const float4*>(G.tree + nd);
      const float4 a = __ldg(n4), b = __ldg(n4 + 1);
      // the rounded point against the outward-rounded subtree box: a float
      // comparison that can only keep more (the FP64 element test decides)
      if (xf[0] < a.x || xf[1] < a.y || xf[2] < a.z || xf[0] > b.x || xf[1] > b.y || xf[2] > b.z) continue;
      const float4 c = __ldg(n4 + 2), d = __ldg(n4 + 3);
      if (!(xf[0] < c.x || xf[1] < c.y || xf[2] < c.z || xf[0] > d.x || xf[1] > d.y || xf[2] > d.z)) {
        const int e = __float_as_int(a.w);
        const double* eb = G.ebox + 6 * (long long)e;
        if (x[0] >= eb[0] && x[0] <= eb[3] && x[1] >= eb[1] && x[1] <= eb[4] && x[2] >= eb[2] && x[2] <= eb[5]) {
          if (nc < PC_CAND) {
            // insert in ascending element order
            int j = nc++;
            while (j > 0 && cl[j - 1] > e) { cl[j] = cl[j - 1]; --j; }
            cl[j] = e;
          } else {
            over = true;
          }
        }
      }
      const int l = __float_as_int(b.w), r = __float_as_int(c.w);
      if (r >= 0) { if (sp < PC_STACK) stack[sp++] = r; else over = true; }
      if (l >= 0) { if (sp < PC_STACK) stack[sp++] = l; else over = true; }
    }
    Q.ncand[k] = nc;
    n_c += nc;
    n_over += over;
    if (over) Q.ncand[k] = -1;
  }
  for (int s = 16; s; s >>= 1) {
    n_c += __shfl_xor_sync(0xffffffffu, n_c, s);
    n_over += __shfl_xor_sync(0xffffffffu, n_over, s);
  }
  if ((threadIdx.x & 31) == 0) {
    if (n_c) atomicAdd(&Q.cnt[0], n_c);
    if (n_over) atomicAdd(&Q.cnt[1], n_over);
  }
}

// Lagrange basis on the p+1 equispaced nodes of [-1, 1] and its derivative
template <class T>
__device__ __forceinline__ void pc_basis(int p, T x, T* l, T* dl) {
#pragma unroll
  for (int i = 0; i <= PC_MAXP; ++i) {
    if (i > p) break;
    T v = T(1), dv = T(0);
    const T xi = T(-1) + T(2 * i) / T(p);
#pragma unroll
    for (int j = 0; j <= PC_MAXP; ++j) {
      if (j > p) break;
      if (j == i) continue;
      const T xj = T(-1) + T(2 * j) / T(p);
      const T inv = T(1) / (xi - xj);
      dv = dv * (x - xj) * inv + v * inv;
      v *= (x - xj) * inv;
    }
    l[i] = v;
    dl[i] = dv;
  }
}

// x(xi) (and the Jacobian when J is given) of one element whose node k
// coordinate a is X(a, k)
template <class T, class F>
__device__ __forceinline__ void pc_map(int p, const F& X, const T xi[3], T x[3], T* J) {
  T lx[PC_MAXP + 1], ly[PC_MAXP + 1], lz[PC_MAXP + 1], dx[PC_MAXP + 1], dy[PC_MAXP + 1], dz[PC_MAXP + 1];
  pc_basis<T>(p, xi[0], lx, dx);
  pc_basis<T>(p, xi[1], ly, dy);
  pc_basis<T>(p, xi[2], lz, dz);
  x[0] = x[1] = x[2] = T(0);
  if (J)
    for (int a = 0; a < 9; ++a) J[a] = T(0);
  int nd = 0;
  for (int k = 0; k <= p; ++k)
    for (int j = 0; j <= p; ++j) {
      const T ljk = ly[j] * lz[k], djk = dy[j] * lz[k], ljd = ly[j] * dz[k];
      for (int i = 0; i <= p; ++i, ++nd) {
        const T N = lx[i] * ljk;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const T v = X(a, nd);
          x[a] += v * N;
          if (J) {
            J[3 * a] += v * (dx[i] * ljk);
            J[3 * a + 1] += v * (lx[i] * djk);
            J[3 * a + 2] += v * (lx[i] * ljd);
          }
        }
      }
    }
}

// one clamped Newton step (Eq. ref-update); false when J is singular
template <class T>
__device__ __forceinline__ bool pc_step(const T J[9], const T r[3], T xi[3]) {
  const T c00 = J[4] * J[8] - J[5] * J[7], c01 = J[5] * J[6] - J[3] * J[8], c02 = J[3] * J[7] - J[4] * J[6];
  const T det = J[0] * c00 + J[1] * c01 + J[2] * c02;
  if (!(fabs(det) > T(0))) return false;
  const T inv = T(1) / det;
  const T d0 = (r[0] * c00 + r[1] * (J[2] * J[7] - J[1] * J[8]) + r[2] * (J[1] * J[5] - J[2] * J[4])) * inv;
  const T d1 = (r[0] * c01 + r[1] * (J[0] * J[8] - J[2] * J[6]) + r[2] * (J[2] * J[3] - J[0] * J[5])) * inv;
  const T d2 = (r[0] * c02 + r[1] * (J[1] * J[6] - J[0] * J[7]) + r[2] * (J[0] * J[4] - J[1] * J[3])) * inv;
  const T lim = T(1) + T(PC_CLAMP);
  const T d[3] = {d0, d1, d2};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T v = xi[a] + d[a];
    xi[a] = v < -lim ? -lim : (v > lim ? lim : v);
  }
  return true;
}

__global__ void __launch_bounds__(128) k_pc_newton(PcGrid G, PcQuery Q) {
  unsigned long long n_steps = 0, n_found = 0;
  const int p = G.p, npe = (p + 1) * (p + 1) * (p + 1);
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < Q.n; k += (long long)gridDim.x * blockDim.x) {
    const int nc = Q.ncand[k];
    const double x[3] = {Q.xloc[3 * k], Q.xloc[3 * k + 1], Q.xloc[3 * k + 2]};
    long long found = -1;
    double xi64[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < nc && found < 0; ++c) {
      const int e = Q.cand[(long long)PC_CAND * k + c];
      const float* L = G.loc + (long long)e * 3 * npe;
      const double* o = G.org + 3 * (long long)e;
      const double hE = (double)G.h[e];
      // FP32 stage in the element frame
      const float xl[3] = {(float)(x[0] - o[0]), (float)(x[1] - o[1]), (float)(x[2] - o[2])};
      float xi[3] = {0.f, 0.f, 0.f}, X[3], J[9], r[3];
      auto Lf = [&](int a, int nd) { return L[a * npe + nd]; };
      float rn = INFINITY;
      for (int it = 0; it <= PC_ITERS; ++it) {
        pc_map<float>(p, Lf, xi, X, J);
#pragma unroll
        for (int a = 0; a < 3; ++a) r[a] = xl[a] - X[a];
        rn = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        if (rn <= 1e-5f * (float)hE || it == PC_ITERS) break;
        if (!pc_step<float>(J, r, xi)) break;
      }
      // far from converged at the clamp: the point is outside this element
      if (!(rn <= 1e-3f * (float)hE)) continue;
      // FP64 steps on the original nodes
      const double* N64 = G.nodes + (long long)e * npe * 3;
      auto Ld = [&](int a, int nd) { return N64[3 * nd + a]; };
      double t[3] = {(double)xi[0], (double)xi[1], (double)xi[2]}, Xd[3], Jd[9], rd[3];
      bool conv = false;
      for (int it = 0; it <= PC_POLISH; ++it) {
        // the Jacobian only where another step may follow
        pc_map<double>(p, Ld, t, Xd, it < PC_POLISH ? Jd : nullptr);
#pragma unroll
        for (int a = 0; a < 3; ++a) rd[a] = x[a] - Xd[a];
        if (sqrt(rd[0] * rd[0] + rd[1] * rd[1] + rd[2] * rd[2]) <= PC_RESID * hE) { conv = true; break; }
        if (it == PC_POLISH) break;
        ++n_steps;
        if (!pc_step<double>(Jd, rd, t)) break;
      }
      const double mx = fmax(fabs(t[0]), fmax(fabs(t[1]), fabs(t[2])));
      if (conv && mx <= 1.0 + PC_INSIDE) {
        found = e;
        xi64[0] = t[0]; xi64[1] = t[1]; xi64[2] = t[2];
      }
    }
    Q.donor[k] = found;
    Q.ref[3 * k] = xi64[0]; Q.ref[3 * k + 1] = xi64[1]; Q.ref[3 * k + 2] = xi64[2];
    n_found += found >= 0;
  }
  for (int s = 16; s; s >>= 1) {
    n_steps += __shfl_xor_sync(0xffffffffu, n_steps, s);
    n_found += __shfl_xor_sync(0xffffffffu, n_found, s);
  }
  if ((threadIdx.x & 31) == 0) {
    if (n_steps) atomicAdd(&Q.cnt[2], n_steps);
    if (n_found) atomicAdd(&Q.cnt[3], n_found);
  }
}

}  // namespace dc
