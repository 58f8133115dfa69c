// dc_common.cuh -- shared device-side definitions of libdirectcut.
//
// One cut "instance" = one resident background grid + one cut surface.  Every
// kernel of the pipeline runs over a batch of instances at once (a single cut
// is a batch of one), reading its parameters from a device array of Inst.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dc {

constexpr int MAX_P = 4, MAX_Q = 4;
constexpr int MAX_NPE = (MAX_P + 1) * (MAX_P + 1) * (MAX_P + 1);  // nodes per element
constexpr int MAX_NTE = 12 * MAX_P * MAX_P;                       // boundary triangles per element
constexpr int MAX_NPF = (MAX_Q + 1) * (MAX_Q + 1);                // nodes per cut face
constexpr int MAX_NTF = 2 * MAX_Q * MAX_Q;                        // triangles per cut face
constexpr int MAX_CELLS = 80;                                     // hole-map cubes, longest side
constexpr int MAX_DIM = MAX_CELLS + 2;                            // + one padding cube per side
constexpr int ROW_XCAP = 24;  // surface crossings recorded per hole-map row (a row with more stays NEAR)

// hole-map cube states (Sec. 4.2 hole maps, after the 0/1 flip):
//   OUT  = outside the surface (winding number 0)
//   IN   = inside the surface (winding number 1)
//   NEAR = overlapped by a face box inflated by the fringe margin ("2"), or
//          on a row whose crossings could not be certified
constexpr uint8_t CUBE_OUT = 0, CUBE_IN = 1, CUBE_NEAR = 2;

// flag values written to the per-element int8 output
constexpr int8_t DC_HOLE_ = 0, DC_FIELD_ = 1, DC_FRINGE_ = -1;

// error bits reported per instance
enum : int {
  ERR_ROUNDS = 1,        // face gather did not converge
  ERR_RECHECK = 8,       // FP64 tie list overflow in the FP64 path
  ERR_DEGENERATE = 16,   // zero-extent surface
  ERR_NONFINITE = 64,    // a face node is NaN or infinite
};

struct Inst {
  // background grid (resident)
  const double* nodes;   // [n_elem][(p+1)^3][3]
  const float* eaabb;    // [n_elem][6] element node boxes, rounded outward (the element
                         // frame's origin is the centre of this box)
  long long n_elem;
  int p;
  // cut surface
  const double* faces_in;  // [n_faces][(q+1)^2][3]
  long long n_faces;
  int q;
  int has_pose;
  double pose[12];
  // outputs
  int8_t* flags;
  double* dist;            // may be null
  float* dist32;           // may be null: each exact-test element's distance from
                           // the FP32 bulk alone (signed as dist), before the FP64
                           // re-solve; NaN where the FP32 stage computed none
  // scratch (per instance)
  double* surf;            // posed face nodes [n_faces][(q+1)^2][3]
  float* fbox;             // face node boxes [n_faces][6], float, rounded outward
  int* fbin;               // bin of each face
  uint8_t* cube;           // hole map [dims z][y][x]
  int* bin_cnt;            // [nbins]
  int* bin_off;            // [nbins + 1]
  int* bin_faces;          // [n_faces]
  float* bin_fbox;         // [n_faces][6] the face boxes in bin order (beside bin_faces)
  int nbins_cap;
  int* row_cnt;            // surface crossings per hole-map row [rows] (+ROW_UNDECIDED: undecided)
  int* row_x;              // crossings (cube x << 1 | entering) [rows][ROW_XCAP]
  float* hface;            // truncating variant: face corners, centroid, max |x| [n_faces][16]
  int hmax_bits;           // truncating variant: largest |face coordinate| (float bits)
  // parameters
  double tol;
  float tol_f;             // tol rounded up to float
  int holemap_cells;        // 0: automatic, from h_elem
  float h_elem;             // mean longest box side of the grid's elements
  float cubes_per_edge;     // automatic resolution: cubes per mean element edge
  int bin_cubes;
  int want_dist;
  // derived on the device
  unsigned long long sbox_key[6];  // order-preserving keys of the surface box
  unsigned int fext_bits[3];       // largest face-box extent per axis (float bits)
  unsigned int surf_done;          // blocks of k_surface finished
  double origin[3];
  double ds;
  int dims[3];
  double bs;
  int bdims[3];
  float origin_f[3];               // float copies for the bulk lookups (margins cover
  float inv_ds_f, inv_bs_f;        // their rounding)
  int rows_undecided;              // hole-map rows left NEAR
  int err;
  // counters
  unsigned long long n_cand, n_fringe, n_hole, n_field;
  unsigned long long faces_visited, pairs_bulk, pairs_recheck, fallbacks;
};

// ---------------------------------------------------------------- helpers
// Programmatic dependent launch: a kernel of the cut waits here until the
// kernel before it has completed and its writes are visible (a no-op when it
// was launched without the programmatic attribute), then lets the next kernel
// be launched, so that launch overlaps this kernel's run.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ unsigned long long dkey(double d) {
  unsigned long long b = (unsigned long long)__double_as_longlong(d);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}
__host__ __device__ inline double dkey_decode(unsigned long long k) {
  unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFULL) : ~k;
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  __builtin_memcpy(&d, &b, 8);
  return d;
#endif
}

// instance owning global index g, given exclusive prefix offsets off[0..n]
__device__ __forceinline__ int find_inst(const long long* off, int n, long long g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

}  // namespace dc
