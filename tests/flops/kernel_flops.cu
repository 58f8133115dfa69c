// kernel_flops.cu -- counts the arithmetic of the kernels' triangle-triangle routine
// (the per-unit figure of the exact-test roofline).
//
// The same tritri template the kernels use is instantiated on the host with a
// value type that counts every +, -, *, / and sqrt (a fused multiply-add in
// the kernel is a * and a + here: 2 flops); comparisons, min/max and |x| are
// not counted.  Inputs are pairs of triangles of edge ~1 whose separations are
// drawn uniformly from [0, 2] edge lengths (the near pairs that survive box
// pruning), from a fixed xorshift stream.  Prints: mean, min, max flops/pair.
#include <cmath>
#include <cstdio>

#include "dc_exact.cuh"  // from paper_1711_07663_gb300/csrc (-I)

namespace fc {
long long g_ops = 0;
#ifdef __CUDA_ARCH__
#define FC_COUNT()
#else
#define FC_COUNT() (++g_ops)
#endif
#define HD __host__ __device__
struct CF {
  double v;
  HD CF() : v(0) {}
  HD CF(double x) : v(x) {}
};
HD inline CF operator+(CF a, CF b) { FC_COUNT(); return CF(a.v + b.v); }
HD inline CF operator-(CF a, CF b) { FC_COUNT(); return CF(a.v - b.v); }
HD inline CF operator*(CF a, CF b) { FC_COUNT(); return CF(a.v * b.v); }
HD inline CF operator/(CF a, CF b) { FC_COUNT(); return CF(a.v / b.v); }
HD inline CF operator-(CF a) { return CF(-a.v); }
HD inline bool operator<(CF a, CF b) { return a.v < b.v; }
HD inline bool operator>(CF a, CF b) { return a.v > b.v; }
HD inline bool operator<=(CF a, CF b) { return a.v <= b.v; }
HD inline bool operator>=(CF a, CF b) { return a.v >= b.v; }
HD inline bool operator==(CF a, CF b) { return a.v == b.v; }
HD inline bool operator!=(CF a, CF b) { return a.v != b.v; }
HD inline CF sqrt(CF a) { FC_COUNT(); return CF(::sqrt(a.v)); }
HD inline CF fmin(CF a, CF b) { return CF(a.v < b.v ? a.v : b.v); }
HD inline CF fmax(CF a, CF b) { return CF(a.v > b.v ? a.v : b.v); }
HD inline CF fabs(CF a) { return CF(a.v < 0 ? -a.v : a.v); }
}  // namespace fc

static unsigned long long s_state = 0x9E3779B97F4A7C15ull;
static double urand() {
  s_state ^= s_state << 13;
  s_state ^= s_state >> 7;
  s_state ^= s_state << 17;
  return (double)(s_state >> 11) * (1.0 / 9007199254740992.0);
}

int main() {
  using fc::CF;
  const int N = 200000;
  long long tot = 0, mn = 1LL << 60, mx = 0;
  for (int it = 0; it < N; ++it) {
    dc::V3<CF> a[3], b[3];
    double sep = 2.0 * urand();
    double dir[3] = {urand() - 0.5, urand() - 0.5, urand() - 0.5};
    double dn = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    for (int c = 0; c < 3; ++c) {
      a[c] = dc::mkv(CF(urand()), CF(urand()), CF(urand()));
      b[c] = dc::mkv(CF(urand() + sep * dir[0] / dn), CF(urand() + sep * dir[1] / dn), CF(urand() + sep * dir[2] / dn));
    }
    CF U, L;
    dc::V3<CF> ca, cb;
    fc::g_ops = 0;
    int xc;
    dc::tritri<CF>(a, b, U, L, ca, cb, xc);
    tot += fc::g_ops;
    if (fc::g_ops < mn) mn = fc::g_ops;
    if (fc::g_ops > mx) mx = fc::g_ops;
  }
  printf("%.1f %lld %lld\n", (double)tot / N, mn, mx);
  return 0;
}
