// oracle_flops.cpp -- counts the arithmetic of the oracle's triangle-triangle
// distance (orc_tritri in oracle/oracle.c), the per-unit cost C_tt of the
// exact test's algorithmic flop count.
//
// oracle.c is compiled here as C++ with every `double` replaced by a number
// type that counts each +, -, *, / and sqrt (comparisons, min/max, |x| and
// sign changes are not counted; the oracle is built without FMA contraction,
// so each multiply and add is a separate operation).  Nothing of the oracle is
// changed: the same source, the same branches, only the type differs.
//
// Inputs: the same seeded distribution as kernel_flops.cu -- triangles with
// vertices uniform in a unit cube, the second shifted by a separation drawn
// uniformly from [0, 2] edge lengths in a random direction (the near pairs
// that survive box pruning).  Prints: mean, min, max flops per pair.
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <cstdio>

namespace fc {
long long g_ops = 0;
struct FD {
  double v;
  FD() : v(0) {}
  FD(double x) : v(x) {}
  explicit operator int() const { return (int)v; }
  explicit operator long() const { return (long)v; }
  explicit operator long long() const { return (long long)v; }
  explicit operator unsigned long() const { return (unsigned long)v; }
};
inline FD operator+(FD a, FD b) { ++g_ops; return FD(a.v + b.v); }
inline FD operator-(FD a, FD b) { ++g_ops; return FD(a.v - b.v); }
inline FD operator*(FD a, FD b) { ++g_ops; return FD(a.v * b.v); }
inline FD operator/(FD a, FD b) { ++g_ops; return FD(a.v / b.v); }
inline FD operator-(FD a) { return FD(-a.v); }
inline FD& operator+=(FD& a, FD b) { a = a + b; return a; }
inline FD& operator-=(FD& a, FD b) { a = a - b; return a; }
inline FD& operator*=(FD& a, FD b) { a = a * b; return a; }
inline FD& operator/=(FD& a, FD b) { a = a / b; return a; }
inline bool operator<(FD a, FD b) { return a.v < b.v; }
inline bool operator>(FD a, FD b) { return a.v > b.v; }
inline bool operator<=(FD a, FD b) { return a.v <= b.v; }
inline bool operator>=(FD a, FD b) { return a.v >= b.v; }
inline bool operator==(FD a, FD b) { return a.v == b.v; }
inline bool operator!=(FD a, FD b) { return a.v != b.v; }
inline FD sqrt(FD a) { ++g_ops; return FD(std::sqrt(a.v)); }
inline FD fabs(FD a) { return FD(std::fabs(a.v)); }
inline FD fmin(FD a, FD b) { return FD(std::fmin(a.v, b.v)); }
inline FD fmax(FD a, FD b) { return FD(std::fmax(a.v, b.v)); }
inline FD atan2(FD a, FD b) { ++g_ops; return FD(std::atan2(a.v, b.v)); }
inline FD acos(FD a) { ++g_ops; return FD(std::acos(a.v)); }
}  // namespace fc

using fc::FD;
using fc::sqrt;
using fc::fabs;
using fc::fmin;
using fc::fmax;
using fc::atan2;
using fc::acos;

#define double FD
#include "../../oracle/oracle.c"
#undef double

static unsigned long long s_state = 0x9E3779B97F4A7C15ull;
static double urand() {
  s_state ^= s_state << 13;
  s_state ^= s_state >> 7;
  s_state ^= s_state << 17;
  return (double)(s_state >> 11) * (1.0 / 9007199254740992.0);
}

int main() {
  const int N = 200000;
  long long tot = 0, mn = 1LL << 60, mx = 0;
  for (int it = 0; it < N; ++it) {
    FD A[9], B[9], ca[3], cb[3];
    double sep = 2.0 * urand();
    double dir[3] = {urand() - 0.5, urand() - 0.5, urand() - 0.5};
    double dn = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    for (int c = 0; c < 3; ++c) {
      A[3 * c] = FD(urand());
      A[3 * c + 1] = FD(urand());
      A[3 * c + 2] = FD(urand());
      B[3 * c] = FD(urand() + sep * dir[0] / dn);
      B[3 * c + 1] = FD(urand() + sep * dir[1] / dn);
      B[3 * c + 2] = FD(urand() + sep * dir[2] / dn);
    }
    fc::g_ops = 0;
    orc_tritri(A, B, ca, cb);
    tot += fc::g_ops;
    if (fc::g_ops < mn) mn = fc::g_ops;
    if (fc::g_ops > mx) mx = fc::g_ops;
  }
  printf("%.1f %lld %lld\n", (double)tot / N, mn, mx);
  return 0;
}
