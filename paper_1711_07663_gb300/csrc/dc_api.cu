// dc_api.cu -- the C ABI of libdirectcut (declared in include/directcut.h).
//
// Host side of the parallel direct cut: resident background grids, per-slot
// device arenas, the launch sequence of one (batched) cut, and the serving
// calls (dc_submit / dc_poll) that let requests in different slots overlap on
// the GPU.
#include <cuda_runtime.h>
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define DC_HAVE_NVTX 1
#endif

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/directcut.h"
#include "dc_near.cuh"
#include "dc_overset.cuh"
#include "dc_heur.cuh"
#include "dc_pc.cuh"
#include "dc_frames.cuh"

using namespace dc;

namespace {

thread_local std::string g_err;

// NVTX range over a host-side phase of a call (visible in a profiler's
// timeline; no cost when no tool is attached)
struct NvtxRange {
#ifdef DC_HAVE_NVTX
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
#else
  explicit NvtxRange(const char*) {}
#endif
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Every device and pinned-host allocation of the library goes through
// dev_alloc / host_alloc: they count allocations, and dc_fail_alloc can arm a
// one-shot failure of a later one, so that the handling of DC_ENOMEM (by the
// library and by its callers) can be exercised without exhausting memory.
std::atomic<long long> g_allocs{0};
std::atomic<long long> g_fail_at{-1};

bool alloc_fails() {
  const long long k = g_allocs.fetch_add(1);
  long long f = g_fail_at.load();
  return f >= 0 && k == f && g_fail_at.compare_exchange_strong(f, -1);
}
template <class T>
cudaError_t dev_alloc(T** p, size_t n) {
  if (alloc_fails()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(reinterpret_cast<void**>(p), n);
}
template <class T>
cudaError_t host_alloc(T** p, size_t n) {
  if (alloc_fails()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocHost(reinterpret_cast<void**>(p), n);
}

dc_status fail(dc_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define CK(call)                                                                            \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return fail(DC_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)
// an allocation: its failure is DC_ENOMEM, and the sticky error is cleared
#define CKA(call)                                                                            \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      cudaGetLastError();                                                                    \
      return fail(DC_ENOMEM, "%s: %s", #call, cudaGetErrorString(e_));                       \
    }                                                                                        \
  } while (0)

// ------------------------------------------------------------------ element boxes
// Node boxes rounded outward and, when loc/org are given, the element frame of
// the exact test (k_elem_frames, dc_frames.cuh): a persistent grid of blocks
// over tiles of consecutive elements.  bad[0] is set for a non-finite node,
// bad[1] when a bulk copy never completed; ext_sum (may be null) receives the
// sum of the elements' longest box sides.
cudaError_t launch_frames(const double* nodes, long long n_elem, int npe, float* box, float* loc, double* org,
                          int* bad, double* ext_sum, int n_sm, cudaStream_t st) {
  const int eb = frames_tile_elems(npe);
  const size_t sm = frames_smem(npe);
  cudaError_t e = cudaFuncSetAttribute(k_elem_frames, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_elem_frames, FR_THREADS, sm);
  if (e != cudaSuccess) return e;
  const long long tiles = (n_elem + eb - 1) / eb;
  const long long grid = std::min<long long>(tiles, (long long)n_sm * std::max(occ, 1));
  k_elem_frames<<<(unsigned)grid, FR_THREADS, sm, st>>>(nodes, n_elem, npe, eb, box, loc, org, bad, ext_sum, bad + 1);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ triangle tables
// Element faces: 0 xi=-1, 1 xi=+1, 2 eta=-1, 3 eta=+1, 4 zeta=-1, 5 zeta=+1;
// face grid coordinates (a, b) run over the two free reference directions in
// (xi, eta, zeta) order; each grid quad (a,b) becomes triangles (00,10,11) and
// (00,11,01).  Cut faces: node (i,j) at i + (q+1) j, same quad split, which
// keeps d/dxi x d/deta as the triangle normal.
void build_tables(unsigned char et[MAX_P][MAX_NTE][3], unsigned char ft[MAX_Q][MAX_NTF][3]) {
  memset(et, 0, sizeof(unsigned char) * MAX_P * MAX_NTE * 3);
  memset(ft, 0, sizeof(unsigned char) * MAX_Q * MAX_NTF * 3);
  for (int p = 1; p <= MAX_P; ++p) {
    auto nid = [p](int i, int j, int k) { return i + (p + 1) * (j + (p + 1) * k); };
    int t = 0;
    for (int face = 0; face < 6; ++face) {
      int axis = face / 2, fix = (face % 2) ? p : 0;
      auto at = [&](int a, int b) {
        int ijk[3];
        ijk[axis] = fix;
        int u = 0;
        for (int d = 0; d < 3; ++d)
          if (d != axis) ijk[d] = (u++ == 0) ? a : b;
        return nid(ijk[0], ijk[1], ijk[2]);
      };
      for (int b = 0; b < p; ++b)
        for (int a = 0; a < p; ++a) {
          int q00 = at(a, b), q10 = at(a + 1, b), q11 = at(a + 1, b + 1), q01 = at(a, b + 1);
          int tri[2][3] = {{q00, q10, q11}, {q00, q11, q01}};
          for (int h = 0; h < 2; ++h, ++t)
            for (int c = 0; c < 3; ++c) et[p - 1][t][c] = (unsigned char)tri[h][c];
        }
    }
  }
  for (int q = 1; q <= MAX_Q; ++q) {
    int t = 0;
    for (int b = 0; b < q; ++b)
      for (int a = 0; a < q; ++a) {
        int q00 = a + (q + 1) * b, q10 = q00 + 1, q01 = q00 + (q + 1), q11 = q01 + 1;
        int tri[2][3] = {{q00, q10, q11}, {q00, q11, q01}};
        for (int h = 0; h < 2; ++h, ++t)
          for (int c = 0; c < 3; ++c) ft[q - 1][t][c] = (unsigned char)tri[h][c];
      }
  }
}

// ------------------------------------------------------------------ context
struct Mesh {
  int p = 0;
  long long n_elem = 0;
  double* nodes = nullptr;
  float* box = nullptr;
  float h_elem = 0.f;      // mean longest box side of the elements
};

struct Arena {
  char* base = nullptr;
  size_t cap = 0;
};

// Everything the kernel sequence of one cut depends on.  A slot keeps the
// CUDA graphs it captured, keyed by these values; the per-request data (pose,
// input/output pointers) lives in the instance table, which is copied to the
// device before each launch, so one graph serves every request of a shape.
struct LaunchParams {
  int n = 0;
  long long nf_total = 0, ne_total = 0, max_tri = 0, max_f = 0;
  int pmax = 1, qmax = 1, precision = 0, prof = 0;
  Inst* d_inst = nullptr;
  long long* d_off = nullptr;
  unsigned long long *cand = nullptr, *redo = nullptr, *d_cnt = nullptr;
  // flags-only form of the exact stage (k_near_*), when some instance
  // asks for flags only
  bool near = false;
  bool uniform = false;  // every instance has element order pmax and face order qmax
  int wpc = 8, cpw = 1;  // its warps per block and candidates per cursor step
  int* hsel = nullptr;   // truncating variant: kept faces per candidate
  unsigned long long* full = nullptr;  // flags-only stage: candidates for the full search
  bool operator==(const LaunchParams& o) const {
    return n == o.n && nf_total == o.nf_total && ne_total == o.ne_total && max_tri == o.max_tri && max_f == o.max_f &&
           pmax == o.pmax &&
           qmax == o.qmax && precision == o.precision && prof == o.prof && d_inst == o.d_inst && d_off == o.d_off &&
           cand == o.cand && redo == o.redo && d_cnt == o.d_cnt && near == o.near && uniform == o.uniform &&
           wpc == o.wpc && cpw == o.cpw &&
           hsel == o.hsel && full == o.full;
  }
};

struct GraphEntry {
  LaunchParams key;
  cudaGraphExec_t exec = nullptr;
  unsigned long long last_use = 0;
};

struct Slot {
  cudaStream_t stream = nullptr;
  std::vector<GraphEntry> graphs;   // captured launch sequences of this slot
  unsigned long long use_clock = 0;
  cudaEvent_t done = nullptr;
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  Arena arena;
  // Pinned staging of the instance table, reused round-robin: an entry is
  // rewritten only after the event recorded behind its upload has completed,
  // so back-to-back asynchronous cuts never overwrite a pending copy.
  static constexpr int RING = 4;
  Inst* ring_inst[RING] = {nullptr, nullptr, nullptr, nullptr};
  long long* ring_off[RING] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t ring_ev[RING] = {nullptr, nullptr, nullptr, nullptr};
  bool ring_used[RING] = {false, false, false, false};
  int ring_pos = 0;
  Inst* h_inst = nullptr;        // current ring entry
  long long* h_off = nullptr;    // current ring entry: foff then eoff
  size_t h_inst_cap = 0;
  unsigned long long* h_cnt = nullptr;  // pinned counters readback
  int8_t* h_flags = nullptr;     // pinned output staging (serving, host outputs)
  double* h_dist = nullptr;
  size_t h_out_cap = 0;
  size_t h_dist_cap = 0;
  // completion of a submitted request's upload of host face nodes: dc_submit
  // waits on it before it returns, so the caller may reuse its buffer at once
  cudaEvent_t in_done = nullptr;
  bool busy = false;
  uint64_t ticket = 0;
  // in-flight bookkeeping
  int n_inst = 0;
  Inst* d_inst = nullptr;
  unsigned long long* d_cnt = nullptr;
  int8_t* user_flags = nullptr;
  double* user_dist = nullptr;
  long long out_n = 0;
  bool host_out = false;
  bool want_dist = false;
  bool near = false;       // the flags-only split ran
  int cur_ring = 0;
};

// face order the slots' reservation at dc_create is sized for
constexpr int RESERVE_Q = 2;
// elements up to which the fused prep kernel also classifies (beyond, a
// separate k_classify launch does)
constexpr long long PREP_CLASSIFY_MAX = 1LL << 20;
// prefix offsets over a batch's instances, each n + 1 long: faces, elements,
// k_prep's surface tiles, surface triangles
constexpr int NOFF = 4;

constexpr int NCNT = 24;  // [0,1] candidates/cursor, [2,3] redo/cursor, [4..10] exact counters,
                          // [22] the prep kernel's barrier count (low half) and time-out flag,
                          // [11] near faces tested, [12] holes decided by the hole map,
                          // [14] near full searches, [16] near pairs given the
                          // full FP32 test, [17] truncating variant: FP64 key
                          // rescans, [18] FP64 pass-1 re-solves, [20,21]
                          // full-search list of the flags-only stage/cursor

}  // namespace

struct dc_ctx {
  dc_config cfg;
  int n_sm = 0;
  std::vector<Mesh> meshes;
  std::vector<Slot> slots;
  std::mutex mu;
  uint64_t next_ticket = 1;
  size_t mesh_bytes = 0;
  size_t arena_bytes = 0;
  dc_stats last{};
  int pmax = 1;
  int smem_optin = 0;  // per-block opt-in shared memory limit of the device
  int near_dyn_max = 0;  // dynamic shared memory k_near_main may take per block
  dc_tuning tune{1.8f, 4, 8, 1, 0.f};  // launch shapes (dc_set_tuning, dc_autotune)
  bool use_graphs = true;  // replay captured launch sequences (DC_NO_GRAPHS=1 disables)
  // the slots' reservation made at creation: one pinned host block and one
  // device block, carved into every slot's staging and arena (buffers a slot
  // later outgrows are replaced by its own allocations)
  char* pin_block = nullptr;
  size_t pin_bytes = 0;
  char* dev_block = nullptr;
  size_t dev_bytes = 0;
};

namespace {

struct InstReq {
  int mesh;
  const dc_request* req;
};

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// the smallest float >= x (x finite, positive)
float float_up(double x) {
  float f = (float)x;
  if ((double)f < x) f = std::nextafter(f, INFINITY);
  return f;
}

int nbins_cap(int bin_cubes) {
  int b = (MAX_DIM + bin_cubes - 1) / bin_cubes;
  return b * b * b;
}

// the smallest bins a context's arenas are sized for: the configured size, or
// 2 cubes when that is larger (so a tuned size of 2 still fits)
int bin_floor(const dc_config& cfg) { return cfg.bin_cubes < 2 ? cfg.bin_cubes : 2; }

size_t cube_bytes() { return (size_t)MAX_DIM * MAX_DIM * CUBE_PITCH; }

// hole-map row tables of one instance: crossing counts and crossings
size_t run_bytes() {
  const size_t rows = (size_t)MAX_DIM * MAX_DIM;
  return al256(sizeof(int) * rows) + al256(sizeof(int) * rows * ROW_XCAP);
}

// Launch k on st; with pdl, as a programmatic dependent launch: it may start
// while the previous kernel of the stream finishes, its pdl_enter() waiting for
// that kernel's completion (captured into graphs as programmatic edges).
template <typename... KArgs, typename... Args>
cudaError_t launch_k(bool pdl, void (*k)(KArgs...), dim3 g, dim3 b, size_t sm, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

// face bins filled and row crossings found (one launch), then row labels
cudaError_t launch_rows(bool pdl, Inst* d_inst, const long long* foff, int n, long long nf_total, long long max_tri,
                        cudaStream_t st) {
  const int fill_blocks = (int)((nf_total + 255) / 256);
  cudaError_t e = launch_k(pdl, k_fill_cross, dim3((unsigned)(fill_blocks + (max_tri + 255) / 256), n), dim3(256), 0,
                           st, d_inst, foff, n, nf_total, fill_blocks);
  if (e != cudaSuccess) return e;
  return launch_k(pdl, k_row_label, dim3((MAX_DIM * MAX_DIM + 7) / 8, n), dim3(256), 0, st, d_inst);
}

// the flags-only stage's kernel for a batch: compiled for its orders when
// every instance has the same element order p and face order q (p = q, the
// workloads' case), otherwise the form that reads the orders per instance
using NearKernel = void (*)(Inst*, CandList, CandList, NearBufs, int, int, int, unsigned long long*);
NearKernel near_kernel(int pmax, int qmax, bool uniform) {
  if (uniform && pmax == qmax) {
    switch (pmax) {
      case 1: return k_near_main<1, 1>;
      case 2: return k_near_main<2, 2>;
      case 3: return k_near_main<3, 3>;
      case 4: return k_near_main<4, 4>;
      default: break;
    }
  }
  return k_near_main<0, 0>;
}
const NearKernel NEAR_KERNELS[] = {k_near_main<0, 0>, k_near_main<1, 1>, k_near_main<2, 2>, k_near_main<3, 3>,
                                   k_near_main<4, 4>};

// one instance's surface as far as the arena is concerned
struct SurfNeed {
  long long F;  // faces
  int q;        // their order
  bool staged;  // host faces, uploaded into the arena
};

// bytes of arena a batch of surfaces over ne_total elements needs
size_t arena_bytes(const dc_ctx* c, const std::vector<SurfNeed>& v, long long ne_total) {
  size_t s = al256(sizeof(Inst) * v.size()) + al256(sizeof(long long) * NOFF * (v.size() + 1));
  int nb = nbins_cap(bin_floor(c->cfg));
  for (auto& r : v) {
    long long F = r.F;
    int npf = (r.q + 1) * (r.q + 1);
    if (r.staged) s += al256(sizeof(double) * F * npf * 3);  // staged input faces
    if (c->cfg.precision == DC_HEURISTIC) s += al256(sizeof(float) * 16 * F);
    s += al256(sizeof(double) * F * npf * 3) + al256(sizeof(float) * F * 6) * 2 +
         al256(sizeof(int) * F) * 2 + al256(cube_bytes()) + al256(sizeof(int) * nb) + al256(sizeof(int) * (nb + 1)) +
         run_bytes();
  }
  s += al256(sizeof(unsigned long long) * ne_total) * 3;  // candidates, redo, full-search list
  if (c->cfg.precision == DC_HEURISTIC) s += al256(sizeof(int) * HEUR_SEL * ne_total);  // kept faces
  s += al256(sizeof(unsigned long long) * NCNT);
  s += al256(ne_total) + al256(sizeof(double) * ne_total) + al256(sizeof(float) * ne_total);  // output staging
  return s;
}

size_t arena_need(const dc_ctx* c, const std::vector<InstReq>& v, long long ne_total) {
  std::vector<SurfNeed> sv;
  sv.reserve(v.size());
  for (auto& r : v) sv.push_back({r.req->n_faces, r.req->q, !r.req->on_device});
  return arena_bytes(c, sv, ne_total);
}

// free a slot's buffer unless it is part of the context's reservation
void host_free(const dc_ctx* c, void* p) {
  if (!p) return;
  const char* q = static_cast<const char*>(p);
  if (c->pin_block && q >= c->pin_block && q < c->pin_block + c->pin_bytes) return;
  cudaFreeHost(p);
}
void dev_free(const dc_ctx* c, void* p) {
  if (!p) return;
  const char* q = static_cast<const char*>(p);
  if (c->dev_block && q >= c->dev_block && q < c->dev_block + c->dev_bytes) return;
  cudaFree(p);
}

dc_status ensure_arena(dc_ctx* c, Slot& s, size_t need) {
  if (s.arena.cap >= need) return DC_OK;
  size_t grow = std::max(need, s.arena.cap + s.arena.cap / 2);
  if (c->cfg.mem_budget_bytes &&
      c->mesh_bytes + c->arena_bytes - s.arena.cap + grow > c->cfg.mem_budget_bytes) {
    grow = need;
    if (c->mesh_bytes + c->arena_bytes - s.arena.cap + grow > c->cfg.mem_budget_bytes)
      return fail(DC_EBUSY, "memory budget of %zu bytes exhausted (need %zu more)", c->cfg.mem_budget_bytes, grow);
  }
  if (s.arena.base) {
    CK(cudaStreamSynchronize(s.stream));
    for (auto& g : s.graphs) cudaGraphExecDestroy(g.exec);
    s.graphs.clear();
    dev_free(c, s.arena.base);
    c->arena_bytes -= s.arena.cap;
    s.arena.base = nullptr;
    s.arena.cap = 0;
  }
  cudaError_t e = dev_alloc(&s.arena.base, grow);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(DC_ENOMEM, "cudaMalloc(%zu) for the cut arena failed: %s", grow, cudaGetErrorString(e));
  }
  s.arena.cap = grow;
  c->arena_bytes += grow;
  return DC_OK;
}

// host staging of a slot: the instance ring, counters, the flags of host
// outputs, and (want_host_dist: a submitted request with host distances) their
// distances
dc_status ensure_host(dc_ctx* c, Slot& s, size_t n_inst, long long ne_total, bool want_host_dist) {
  if (s.h_inst_cap < n_inst) {
    for (int r = 0; r < Slot::RING; ++r) {
      if (s.ring_used[r]) CK(cudaEventSynchronize(s.ring_ev[r]));
      host_free(c, s.ring_inst[r]);
      host_free(c, s.ring_off[r]);
      s.ring_inst[r] = nullptr;
      s.ring_off[r] = nullptr;
      s.ring_used[r] = false;
    }
    // capacity 0 until every buffer exists: a failed allocation leaves the
    // ring to be rebuilt by the next call
    s.h_inst_cap = 0;
    for (int r = 0; r < Slot::RING; ++r) {
      CKA(host_alloc(&s.ring_inst[r], sizeof(Inst) * n_inst));
      CKA(host_alloc(&s.ring_off[r], sizeof(long long) * NOFF * (n_inst + 1)));
    }
    s.h_inst_cap = n_inst;
  }
  {
    int r = s.ring_pos;
    s.ring_pos = (s.ring_pos + 1) % Slot::RING;
    if (s.ring_used[r]) CK(cudaEventSynchronize(s.ring_ev[r]));
    s.h_inst = s.ring_inst[r];
    s.h_off = s.ring_off[r];
    s.ring_used[r] = false;
    s.cur_ring = r;
  }
  if (!s.h_cnt) CKA(host_alloc(&s.h_cnt, sizeof(unsigned long long) * NCNT));
  if ((long long)s.h_out_cap < ne_total) {
    host_free(c, s.h_flags);
    s.h_flags = nullptr;
    s.h_out_cap = 0;
    CKA(host_alloc(&s.h_flags, (size_t)ne_total));
    s.h_out_cap = (size_t)ne_total;
  }
  if (want_host_dist && (long long)s.h_dist_cap < ne_total) {
    host_free(c, s.h_dist);
    s.h_dist = nullptr;
    s.h_dist_cap = 0;
    CKA(host_alloc(&s.h_dist, sizeof(double) * ne_total));
    s.h_dist_cap = (size_t)ne_total;
  }
  return DC_OK;
}


dc_status validate_req(dc_ctx* c, int mesh, const dc_request* r) {
  if (!r) return fail(DC_EINVAL, "request is NULL");
  if (mesh < 0 || mesh >= (int)c->meshes.size()) return fail(DC_ENOTFOUND, "mesh %d does not exist", mesh);
  if (r->q < 1 || r->q > MAX_Q) return fail(DC_EINVAL, "face order q=%d outside 1..%d", r->q, MAX_Q);
  if (r->n_faces < 1 || r->n_faces > (1LL << 30)) return fail(DC_EINVAL, "n_faces=%lld out of range", (long long)r->n_faces);
  if (!r->face_nodes || !r->flags_out) return fail(DC_EINVAL, "face_nodes and flags_out are required");
  if (r->pose)
    for (int i = 0; i < 12; ++i)
      if (!std::isfinite(r->pose[i])) return fail(DC_EINVAL, "pose has a non-finite entry");
  if (r->fp32_dist_out && (!r->dist_out || c->cfg.precision != DC_FP32_RECHECK))
    return fail(DC_EINVAL, "fp32_dist_out needs dist_out and the DC_FP32_RECHECK precision");
  // face nodes are checked on the device as they are posed (k_surface), for
  // host and device inputs alike
  return DC_OK;
}

// Phase events: inside a stream capture they must become event-record nodes.
cudaError_t record(cudaEvent_t ev, cudaStream_t st, bool capturing) {
  return capturing ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal) : cudaEventRecord(ev, st);
}

// The kernel sequence of one (batched) cut on stream st.
dc_status launch_cut(dc_ctx* c, Slot& s, const LaunchParams& P, cudaStream_t st, bool capturing) {
  const int n = P.n;
  const long long nf_total = P.nf_total, ne_total = P.ne_total, max_tri = P.max_tri;
  const int pmax = P.pmax, qmax = P.qmax;
  Inst* d_inst = P.d_inst;
  long long* d_off = P.d_off;
  unsigned long long *cand = P.cand, *redo = P.redo, *d_cnt = P.d_cnt;
  CK(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long) * NCNT, st));
  const bool prof = P.prof != 0;
  if (prof) CK(record(s.ev[0], st, capturing));

  const int TB = 256;
  (void)max_tri;
  CandList cl{cand, (unsigned long long)ne_total, d_cnt};
  CandList rl{redo, (unsigned long long)ne_total, d_cnt + 2};
  {
    // a1-a4 in one cooperative launch (every block resident for its grid
    // barriers); its barrier counters are in d_cnt[22], zeroed above
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_prep, TB, 0));
    occ = std::max(1, std::min(occ, 4));
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)(c->n_sm * occ));
    lc.blockDim = dim3(TB);
    lc.dynamicSmemBytes = 0;
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    // a batch of millions of elements is classified by its own full-width
    // launch; a single grid's elements are a phase of the fused kernel
    const bool fused_classify = ne_total <= PREP_CLASSIFY_MAX;
    CK(cudaLaunchKernelEx(&lc, k_prep, d_inst, (const long long*)d_off, n, nf_total, ne_total, cl, d_cnt,
                          reinterpret_cast<unsigned*>(d_cnt + 22), fused_classify ? 1 : 0));
    if (!fused_classify)
      CK(launch_k(true, k_classify, dim3((unsigned)((ne_total + TB - 1) / TB)), dim3(TB), 0, st, d_inst,
                  (const long long*)(d_off + n + 1), n, ne_total, cl, d_cnt));
  }
  if (prof) {
    // the three phases are one kernel: their times are reported together
    CK(record(s.ev[1], st, capturing));
    CK(record(s.ev[2], st, capturing));
    CK(record(s.ev[3], st, capturing));
  }
  const ExLayout Lf = ex_layout(pmax, qmax, 4), Ld = ex_layout(pmax, qmax, 8);
  const int WPB = TB / 32;
  if ((long long)Ld.total * WPB > c->smem_optin)
    return fail(DC_EINVAL, "orders p=%d q=%d need %d bytes of shared memory per block", pmax, qmax, Ld.total * WPB);
  CandList none{redo, 0, d_cnt + 2};
  if (P.precision == DC_HEURISTIC) {
    // the paper's truncating variant: kept faces per candidate, then pass 2
    // (FP32 with FP64 re-solves; FP64 for the elements whose list overflowed)
    CK(launch_k(true, k_heur_faces, dim3((unsigned)((P.max_f + TB - 1) / TB), n), dim3(TB), 0, st, d_inst));
    int occs = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occs, k_heur_select, TB, 0);
    occs = std::max(occs, 1);
    CK(launch_k(true, k_heur_select, dim3(c->n_sm * occs), dim3(TB), 0, st, d_inst, cl, P.hsel, d_cnt + 17));
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_heur_final<float>, TB, (size_t)Lf.total * WPB);
    occ = std::max(occ, 1);
    CK(launch_k(true, k_heur_final<float>, dim3(c->n_sm * occ), dim3(TB), (size_t)Lf.total * WPB, st, d_inst, cl, rl,
                (const int*)P.hsel, 0, pmax, qmax, d_cnt + 4));
    if (prof) CK(record(s.ev[5], st, capturing));
    CK(launch_k(true, k_heur_final<double>, dim3(std::min(c->n_sm, 16)), dim3(TB), (size_t)Ld.total * WPB, st, d_inst,
                cl, rl, (const int*)P.hsel, 1, pmax, qmax, d_cnt + 4));
  } else if (P.precision == DC_FP32_RECHECK && P.near) {
    // flags-only form: one kernel settles every candidate (full searches and
    // their FP64 redo included)
    NearBufs nb{d_cnt + 11};
    const size_t per = (size_t)near_region(pmax, qmax);
    int wpc = std::min(P.wpc, NEAR_MAX_WARPS);
    while (wpc > 1 && per * wpc > (size_t)c->near_dyn_max) wpc >>= 1;
    if (per * wpc > (size_t)c->near_dyn_max)
      return fail(DC_EINVAL, "orders p=%d q=%d need %zu bytes of shared memory per warp", pmax, qmax, per);
    const size_t sm = per * wpc;
    const NearKernel kn = near_kernel(pmax, qmax, P.uniform);
    int occn = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occn, kn, 32 * wpc, sm);
    occn = std::max(occn, 1);
    CandList fl{P.full, (unsigned long long)ne_total, d_cnt + 20};
    CK(launch_k(true, kn, dim3(c->n_sm * occn), dim3(32 * wpc), sm, st, d_inst, cl, fl, nb, pmax, qmax, P.cpw,
                d_cnt + 4));
    if (prof) CK(record(s.ev[5], st, capturing));  // (the FP64 pass below is the "redo" phase)
    // the candidates it listed for the full per-element search -- only
    // elements with no labelled node that are not fringe (distances are never
    // asked for in this form), almost always none: a small FP64 pass
    CK(launch_k(true, k_exact<double>, dim3(std::min(c->n_sm, 16)), dim3(TB), (size_t)Ld.total * WPB, st, d_inst, fl,
                none, pmax, qmax, d_cnt + 4));
  } else if (P.precision == DC_FP32_RECHECK) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_exact<float>, TB, (size_t)Lf.total * WPB);
    occ = std::max(occ, 1);
    CK(launch_k(true, k_exact<float>, dim3(c->n_sm * occ), dim3(TB), (size_t)Lf.total * WPB, st, d_inst, cl, rl, pmax,
                qmax, d_cnt + 4));
    if (prof) CK(record(s.ev[5], st, capturing));
    // the FP64 redo pass is rarely non-empty: a small persistent grid keeps
    // its launch cheap
    CK(launch_k(true, k_exact<double>, dim3(std::min(c->n_sm, 16)), dim3(TB), (size_t)Ld.total * WPB, st, d_inst, rl,
                none, pmax, qmax, d_cnt + 4));
  } else {
    int occd = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occd, k_exact<double>, TB, (size_t)Ld.total * WPB);
    occd = std::max(occd, 1);
    CK(launch_k(true, k_exact<double>, dim3(c->n_sm * occd), dim3(TB), (size_t)Ld.total * WPB, st, d_inst, cl, none,
                pmax, qmax, d_cnt + 4));
    if (prof) CK(record(s.ev[5], st, capturing));
  }
  if (prof) CK(record(s.ev[4], st, capturing));
  return DC_OK;
}

// Replay (capturing on first use) the graph of this launch shape.
dc_status launch_graph(dc_ctx* c, Slot& s, const LaunchParams& P, cudaStream_t st) {
  GraphEntry* hit = nullptr;
  for (auto& g : s.graphs)
    if (g.key == P) hit = &g;
  if (!hit) {
    NvtxRange nr("directcut: capture launch graph");
    if (s.graphs.size() >= 8) {
      auto lru = std::min_element(s.graphs.begin(), s.graphs.end(),
                                  [](const GraphEntry& a, const GraphEntry& b) { return a.last_use < b.last_use; });
      cudaGraphExecDestroy(lru->exec);
      s.graphs.erase(lru);
    }
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeThreadLocal));
    dc_status rc = launch_cut(c, s, P, s.stream, true);
    cudaError_t ec = cudaStreamEndCapture(s.stream, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (ec != cudaSuccess) return fail(DC_ECUDA, "stream capture failed: %s", cudaGetErrorString(ec));
    GraphEntry e;
    e.key = P;
    cudaError_t ei = cudaGraphInstantiate(&e.exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return fail(DC_ECUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(ei));
    s.graphs.push_back(e);
    hit = &s.graphs.back();
  }
  hit->last_use = ++s.use_clock;
  CK(cudaGraphLaunch(hit->exec, st));
  return DC_OK;
}

// Enqueue the whole cut of a batch on slot s.  Host face nodes are uploaded
// straight from the caller's buffer.  copy_inputs: the call returns before the
// cut has run (dc_submit), so enqueue waits for those uploads before it
// returns (on any return once they are queued) and the caller may reuse its
// buffer at once; the synchronous calls need no wait, their caller's buffer
// stays valid until they return.
dc_status enqueue(dc_ctx* c, Slot& s, const std::vector<InstReq>& v, cudaStream_t st, bool copy_inputs) {
  NvtxRange nr("directcut: enqueue");
  const int n = (int)v.size();
  long long nf_total = 0, ne_total = 0, max_tri = 0, max_f = 0;
  int pmax = 1, qmax = 1, pmin = MAX_P, qmin = MAX_Q;
  for (auto& r : v) {
    pmin = std::min(pmin, c->meshes[r.mesh].p);
    qmin = std::min(qmin, r.req->q);
    nf_total += r.req->n_faces;
    max_f = std::max<long long>(max_f, r.req->n_faces);
    ne_total += c->meshes[r.mesh].n_elem;
    max_tri = std::max<long long>(max_tri, r.req->n_faces * 2LL * r.req->q * r.req->q);
    pmax = std::max(pmax, c->meshes[r.mesh].p);
    qmax = std::max(qmax, r.req->q);
  }
  dc_status rc = ensure_arena(c, s, arena_need(c, v, ne_total));
  if (rc) return rc;
  bool host_dist = false;
  if (copy_inputs)
    for (auto& r : v) host_dist |= !r.req->on_device && r.req->dist_out != nullptr;
  rc = ensure_host(c, s, (size_t)n, ne_total, host_dist);
  if (rc) return rc;
  bool uploaded = false;  // host face nodes queued for upload
  struct UploadWait {
    cudaEvent_t ev = nullptr;
    ~UploadWait() {
      if (ev) cudaEventSynchronize(ev);
    }
  } upload_wait;
  // carve the arena
  char* p = s.arena.base;
  auto take = [&](size_t bytes) { char* r = p; p += al256(bytes); return r; };
  Inst* d_inst = (Inst*)take(sizeof(Inst) * n);
  long long* d_off = (long long*)take(sizeof(long long) * NOFF * (n + 1));
  const int nb = nbins_cap(bin_floor(c->cfg));
  long long fo = 0, eo = 0, to = 0, tro = 0;
  for (int i = 0; i < n; ++i) {
    const dc_request* r = v[i].req;
    const Mesh& m = c->meshes[v[i].mesh];
    Inst& in = s.h_inst[i];
    memset(&in, 0, sizeof(Inst));
    long long F = r->n_faces;
    int npf = (r->q + 1) * (r->q + 1);
    in.nodes = m.nodes;
    in.eaabb = m.box;
    in.n_elem = m.n_elem;
    in.p = m.p;
    in.q = r->q;
    in.n_faces = F;
    if (r->on_device) {
      in.faces_in = r->face_nodes;
    } else {
      double* stage = (double*)take(sizeof(double) * F * npf * 3);
      const size_t nd = (size_t)F * npf * 3;
      CK(cudaMemcpyAsync(stage, r->face_nodes, sizeof(double) * nd, cudaMemcpyHostToDevice, st));
      in.faces_in = stage;
      uploaded = true;
    }
    in.has_pose = r->pose ? 1 : 0;
    if (r->pose) memcpy(in.pose, r->pose, sizeof(double) * 12);
    in.surf = (double*)take(sizeof(double) * F * npf * 3);
    if (c->cfg.precision == DC_HEURISTIC) in.hface = (float*)take(sizeof(float) * 16 * F);
    in.fbox = (float*)take(sizeof(float) * F * 6);
    in.fbin = (int*)take(sizeof(int) * F);
    in.bin_faces = (int*)take(sizeof(int) * F);
    in.bin_fbox = (float*)take(sizeof(float) * F * 6);
    in.cube = (uint8_t*)take(cube_bytes());
    in.bin_cnt = (int*)take(sizeof(int) * nb);
    in.bin_off = (int*)take(sizeof(int) * (nb + 1));
    in.nbins_cap = nb;
    {
      const size_t rows = (size_t)MAX_DIM * MAX_DIM;
      in.row_cnt = (int*)take(sizeof(int) * rows);
      in.row_x = (int*)take(sizeof(int) * rows * ROW_XCAP);
    }
    in.tol = c->cfg.tol;
    in.tol_f = float_up(c->cfg.tol);
    in.holemap_cells = c->cfg.holemap_cells;
    in.h_elem = m.h_elem;
    in.cubes_per_edge = c->tune.cubes_per_edge;
    in.bin_cubes = c->tune.bin_cubes;
    in.want_dist = r->dist_out ? 1 : 0;
    for (int a = 0; a < 3; ++a) { in.sbox_key[a] = ~0ULL; in.sbox_key[3 + a] = 0ULL; }
    s.h_off[i] = fo;
    s.h_off[n + 1 + i] = eo;
    s.h_off[2 * (n + 1) + i] = to;
    s.h_off[3 * (n + 1) + i] = tro;
    fo += F;
    eo += m.n_elem;
    to += (F + SURF_FPB - 1) / SURF_FPB;
    tro += F * 2LL * r->q * r->q;
  }
  s.h_off[n] = fo;
  s.h_off[2 * n + 1] = eo;
  s.h_off[3 * n + 2] = to;
  s.h_off[4 * n + 3] = tro;
  unsigned long long* cand = (unsigned long long*)take(sizeof(unsigned long long) * ne_total);
  unsigned long long* redo = (unsigned long long*)take(sizeof(unsigned long long) * ne_total);
  unsigned long long* fulll = (unsigned long long*)take(sizeof(unsigned long long) * ne_total);
  int* hsel = c->cfg.precision == DC_HEURISTIC ? (int*)take(sizeof(int) * HEUR_SEL * ne_total) : nullptr;
  unsigned long long* d_cnt = (unsigned long long*)take(sizeof(unsigned long long) * NCNT);
  int8_t* oflags = (int8_t*)take(ne_total);
  double* odist = (double*)take(sizeof(double) * ne_total);
  float* od32 = (float*)take(sizeof(float) * ne_total);
  // outputs: caller's device buffers, or staging for host buffers
  long long off = 0;
  for (int i = 0; i < n; ++i) {
    const dc_request* r = v[i].req;
    Inst& in = s.h_inst[i];
    if (r->on_device) {
      in.flags = r->flags_out;
      in.dist = r->dist_out;
      in.dist32 = r->fp32_dist_out;
    } else {
      in.flags = oflags + off;
      in.dist = r->dist_out ? odist + off : nullptr;
      in.dist32 = r->fp32_dist_out ? od32 + off : nullptr;
    }
    off += in.n_elem;
  }

  if (copy_inputs && uploaded) {
    CK(cudaEventRecord(s.in_done, st));
    upload_wait.ev = s.in_done;
  }
  CK(cudaMemcpyAsync(d_inst, s.h_inst, sizeof(Inst) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_off, s.h_off, sizeof(long long) * NOFF * (n + 1), cudaMemcpyHostToDevice, st));
  CK(cudaEventRecord(s.ring_ev[s.cur_ring], st));
  s.ring_used[s.cur_ring] = true;
  LaunchParams lp;
  lp.n = n; lp.nf_total = nf_total; lp.ne_total = ne_total; lp.max_tri = max_tri; lp.max_f = max_f;
  lp.pmax = pmax; lp.qmax = qmax; lp.precision = c->cfg.precision; lp.prof = c->cfg.profile != 0;
  lp.d_inst = d_inst; lp.d_off = d_off; lp.cand = cand; lp.redo = redo; lp.d_cnt = d_cnt; lp.hsel = hsel;
  lp.full = fulll;
  lp.wpc = c->tune.warps_per_cta; lp.cpw = c->tune.cands_per_warp;
  lp.uniform = pmin == pmax && qmin == qmax;
  {
    // the flags-only form when no instance asks for distances (a batch that
    // mixes both runs the distance form for all)
    bool flags_only = true;
    for (auto& r : v) flags_only &= r.req->dist_out == nullptr;
    lp.near = c->cfg.precision == DC_FP32_RECHECK && flags_only && ne_total < (1LL << 31);
  }
  {
    const ExLayout Ld = ex_layout(pmax, qmax, 8);
    if ((long long)Ld.total * (256 / 32) > c->smem_optin)
      return fail(DC_EINVAL, "orders p=%d q=%d need %d bytes of shared memory per block", pmax, qmax, Ld.total * 8);
  }
  dc_status lrc = c->use_graphs ? launch_graph(c, s, lp, st) : launch_cut(c, s, lp, st, false);
  if (lrc) return lrc;
  CK(cudaGetLastError());
  s.n_inst = n;
  s.d_inst = d_inst;
  s.d_cnt = d_cnt;
  s.near = lp.near;
  return DC_OK;  // (a submitted request's upload is waited for on the way out)
}

// copy results of a finished (synchronised) batch back and turn device error
// bits into a status; fills ctx->last
dc_status finish(dc_ctx* c, Slot& s, const std::vector<InstReq>& v, cudaStream_t st) {
  NvtxRange nr("directcut: wait and read back");
  const int n = s.n_inst;
  CK(cudaMemcpyAsync(s.h_cnt, s.d_cnt, sizeof(unsigned long long) * NCNT, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(s.h_inst, s.d_inst, sizeof(Inst) * n, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  s.ring_used[s.cur_ring] = false;
  dc_stats& S = c->last;
  memset(&S, 0, sizeof(S));
  int err = 0;
  for (int i = 0; i < n; ++i) {
    err |= s.h_inst[i].err;
    S.n_elem += s.h_inst[i].n_elem;
    S.holemap_rows_undecided += s.h_inst[i].rows_undecided;
  }
  S.n_candidates = (int64_t)s.h_cnt[0];
  S.faces_visited = (int64_t)s.h_cnt[4];
  S.pairs_bulk = (int64_t)s.h_cnt[5];
  S.pairs_recheck = (int64_t)s.h_cnt[6];
  S.n_fringe = (int64_t)s.h_cnt[7];
  S.n_hole = (int64_t)(s.h_cnt[8] + s.h_cnt[12]);
  S.n_field = S.n_elem - S.n_fringe - S.n_hole;
  S.fallbacks = (int64_t)s.h_cnt[10];
  S.near_tasks = s.near ? (int64_t)s.h_cnt[11] : 0;
  S.n_full_search = s.near ? (int64_t)s.h_cnt[14] : (int64_t)s.h_cnt[0];
  S.near_pairs_full = s.near ? (int64_t)s.h_cnt[16] : 0;
  S.heur_rescans = (int64_t)s.h_cnt[17];
  S.heur_resolves = (int64_t)s.h_cnt[18];
  if (c->cfg.profile) {
    cudaEventElapsedTime(&S.ms_surface, s.ev[0], s.ev[1]);
    cudaEventElapsedTime(&S.ms_holemap, s.ev[1], s.ev[2]);
    cudaEventElapsedTime(&S.ms_classify, s.ev[2], s.ev[3]);
    cudaEventElapsedTime(&S.ms_exact, s.ev[3], s.ev[5]);
    cudaEventElapsedTime(&S.ms_redo, s.ev[5], s.ev[4]);
    cudaEventElapsedTime(&S.ms_total, s.ev[0], s.ev[4]);
  }
  if ((s.h_cnt[22] >> 32) != 0) return fail(DC_EINTERNAL, "a grid barrier of the hole-map kernel timed out");
  if (err & ERR_NONFINITE) return fail(DC_EINVAL, "a face node is NaN or infinite");
  if (err & ERR_DEGENERATE) return fail(DC_EINVAL, "the cut surface has zero extent");
  if (err & (ERR_ROUNDS | ERR_RECHECK))
    return fail(DC_EINTERNAL, "exact test capacity exceeded (error bits 0x%x)", err);
  (void)v;
  return DC_OK;
}

// host outputs: the kernels wrote into the arena staging area; the copies
// are queued behind the cut (the caller synchronises)
dc_status copy_out_host(Slot& s, const std::vector<InstReq>& v, cudaStream_t st) {
  for (size_t i = 0; i < v.size(); ++i) {
    const dc_request* r = v[i].req;
    const long long ne = s.h_inst[i].n_elem;
    if (!r->on_device) {
      CK(cudaMemcpyAsync(r->flags_out, s.h_inst[i].flags, (size_t)ne, cudaMemcpyDeviceToHost, st));
      if (r->dist_out) CK(cudaMemcpyAsync(r->dist_out, s.h_inst[i].dist, sizeof(double) * ne, cudaMemcpyDeviceToHost, st));
      if (r->fp32_dist_out)
        CK(cudaMemcpyAsync(r->fp32_dist_out, s.h_inst[i].dist32, sizeof(float) * ne, cudaMemcpyDeviceToHost, st));
    }
  }
  return DC_OK;
}

dc_status init_slot(Slot& s, int prof) {
  CK(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
  for (int r = 0; r < Slot::RING; ++r) CK(cudaEventCreateWithFlags(&s.ring_ev[r], cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&s.in_done, cudaEventDisableTiming));
  if (prof)
    for (int i = 0; i < 6; ++i) CK(cudaEventCreate(&s.ev[i]));
  return DC_OK;
}

void free_slot(dc_ctx* c, Slot& s) {
  if (s.stream) cudaStreamSynchronize(s.stream);
  for (auto& g : s.graphs) cudaGraphExecDestroy(g.exec);
  s.graphs.clear();
  if (s.arena.base) { dev_free(c, s.arena.base); c->arena_bytes -= s.arena.cap; }
  for (int r = 0; r < Slot::RING; ++r) {
    host_free(c, s.ring_inst[r]);
    host_free(c, s.ring_off[r]);
    if (s.ring_ev[r]) cudaEventDestroy(s.ring_ev[r]);
  }
  host_free(c, s.h_cnt);
  host_free(c, s.h_flags);
  host_free(c, s.h_dist);
  if (s.in_done) cudaEventDestroy(s.in_done);
  for (int i = 0; i < 6; ++i)
    if (s.ev[i]) cudaEventDestroy(s.ev[i]);
  if (s.done) cudaEventDestroy(s.done);
  if (s.stream) cudaStreamDestroy(s.stream);
  s = Slot();
}

}  // namespace

// ------------------------------------------------------------------ public ABI
extern "C" {

const char* dc_last_error(const dc_ctx* ctx) {
  (void)ctx;  // the message belongs to the calling thread, whatever the context
  return g_err.c_str();
}

const char* dc_version(void) { return "directcut 0.1 (sm_103a)"; }

int64_t dc_fail_alloc(int64_t after) {
  const long long n = g_allocs.load();
  g_fail_at.store(after >= 0 ? n + after : -1);
  return n;
}

dc_status dc_config_default(dc_config* cfg) {
  if (!cfg) return fail(DC_EINVAL, "cfg is NULL");
  memset(cfg, 0, sizeof(*cfg));
  cfg->device = 0;
  cfg->precision = DC_FP32_RECHECK;
  cfg->tol = 1e-7;
  cfg->holemap_cells = 0;
  cfg->bin_cubes = 4;
  cfg->max_inflight = 4;
  cfg->reserve_faces = 8192;
  return DC_OK;
}

dc_status dc_create(const dc_config* cfg_in, const dc_mesh_desc* meshes, int32_t n_meshes, dc_ctx** out) {
  g_err.clear();
  NvtxRange nr("directcut: dc_create");
  if (!out) return fail(DC_EINVAL, "out is NULL");
  *out = nullptr;
  dc_config cfg;
  if (cfg_in) cfg = *cfg_in; else dc_config_default(&cfg);
  if (cfg.tol == 0.0) cfg.tol = 1e-7;
  if (cfg.bin_cubes == 0) cfg.bin_cubes = 4;
  if (cfg.max_inflight == 0) cfg.max_inflight = 4;
  if (cfg.reserve_faces == 0) cfg.reserve_faces = 8192;
  if (cfg.reserve_faces < -1 || cfg.reserve_faces > (1 << 24))
    return fail(DC_EINVAL, "reserve_faces outside -1..%d", 1 << 24);
  if (!(cfg.tol > 0.0) || !std::isfinite(cfg.tol)) return fail(DC_EINVAL, "tol must be positive and finite");
  if (cfg.holemap_cells != 0 && (cfg.holemap_cells < 8 || cfg.holemap_cells > MAX_CELLS))
    return fail(DC_EINVAL, "holemap_cells outside 8..%d (or 0: automatic)", MAX_CELLS);
  if (cfg.bin_cubes < 1 || cfg.bin_cubes > 16) return fail(DC_EINVAL, "bin_cubes outside 1..16");
  if (cfg.max_inflight < 1 || cfg.max_inflight > 64) return fail(DC_EINVAL, "max_inflight outside 1..64");
  if (cfg.precision != DC_FP64 && cfg.precision != DC_FP32_RECHECK && cfg.precision != DC_HEURISTIC)
    return fail(DC_EINVAL, "unknown precision %d", cfg.precision);
  if (n_meshes < 1 || !meshes) return fail(DC_EINVAL, "at least one mesh is required");
  for (int i = 0; i < n_meshes; ++i) {
    const dc_mesh_desc& m = meshes[i];
    if (m.p < 1 || m.p > MAX_P) return fail(DC_EINVAL, "mesh %d: order p=%d outside 1..%d", i, m.p, MAX_P);
    if (m.n_elem < 1 || m.n_elem >= (1LL << 40)) return fail(DC_EINVAL, "mesh %d: n_elem=%lld out of range", i, (long long)m.n_elem);
    if (!m.nodes) return fail(DC_EINVAL, "mesh %d: nodes is NULL", i);
  }
  int ndev = 0;
  CK(cudaGetDeviceCount(&ndev));
  if (cfg.device < 0 || cfg.device >= ndev) return fail(DC_EINVAL, "device %d not present (%d devices)", cfg.device, ndev);
  CK(cudaSetDevice(cfg.device));
  dc_ctx* c = new dc_ctx();
  c->cfg = cfg;
  {
    const char* ng = getenv("DC_NO_GRAPHS");
    c->use_graphs = !(ng && ng[0] == '1');
  }
  auto bail = [&](dc_status st) { dc_destroy(c); return st; };
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, cfg.device) != cudaSuccess) return bail(fail(DC_ECUDA, "cudaGetDeviceProperties failed"));
  c->n_sm = prop.multiProcessorCount;
  static unsigned char et[MAX_P][MAX_NTE][3], ft[MAX_Q][MAX_NTF][3];
  build_tables(et, ft);
  if (cudaMemcpyToSymbol(c_etri, et, sizeof(et)) != cudaSuccess || cudaMemcpyToSymbol(c_ftri, ft, sizeof(ft)) != cudaSuccess)
    return bail(fail(DC_ECUDA, "uploading triangle tables failed"));
  {
    c->smem_optin = prop.sharedMemPerBlockOptin;
    cudaFuncAttributes fe, fd;
    if (cudaFuncGetAttributes(&fe, k_exact<float>) != cudaSuccess || cudaFuncGetAttributes(&fd, k_exact<double>) != cudaSuccess)
      return bail(fail(DC_ECUDA, "cudaFuncGetAttributes failed"));
    size_t near_static = 0;
    for (NearKernel kn : NEAR_KERNELS) {
      cudaFuncAttributes fa;
      if (cudaFuncGetAttributes(&fa, kn) != cudaSuccess) return bail(fail(DC_ECUDA, "cudaFuncGetAttributes failed"));
      near_static = std::max(near_static, fa.sharedSizeBytes);
    }
    if (cudaFuncSetAttribute(k_exact<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(c->smem_optin - fe.sharedSizeBytes)) != cudaSuccess ||
        cudaFuncSetAttribute(k_exact<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(c->smem_optin - fd.sharedSizeBytes)) != cudaSuccess)
      return bail(fail(DC_ECUDA, "cudaFuncSetAttribute failed"));
    c->near_dyn_max = (int)(c->smem_optin - near_static);
    for (NearKernel kn : NEAR_KERNELS)
      if (cudaFuncSetAttribute(kn, cudaFuncAttributeMaxDynamicSharedMemorySize, c->near_dyn_max) != cudaSuccess)
        return bail(fail(DC_ECUDA, "cudaFuncSetAttribute failed"));
    cudaFuncAttributes fhf, fhd;
    if (cudaFuncGetAttributes(&fhf, k_heur_final<float>) != cudaSuccess ||
        cudaFuncGetAttributes(&fhd, k_heur_final<double>) != cudaSuccess ||
        cudaFuncSetAttribute(k_heur_final<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(c->smem_optin - fhf.sharedSizeBytes)) != cudaSuccess ||
        cudaFuncSetAttribute(k_heur_final<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(c->smem_optin - fhd.sharedSizeBytes)) != cudaSuccess)
      return bail(fail(DC_ECUDA, "cudaFuncSetAttribute failed"));
  }
  c->tune.bin_cubes = cfg.bin_cubes;
  c->slots.resize(cfg.max_inflight);
  for (auto& s : c->slots) {
    dc_status st = init_slot(s, cfg.profile);
    if (st) return bail(st);
  }
  int* d_bad = nullptr;  // [0]: a node is not finite; bytes 8..15: sum of element extents
  if (dev_alloc(&d_bad, 16) != cudaSuccess) return bail(fail(DC_ENOMEM, "cudaMalloc failed"));
  double* d_ext = reinterpret_cast<double*>(reinterpret_cast<char*>(d_bad) + 8);
  cudaStream_t st = c->slots[0].stream;
  c->meshes.resize(n_meshes);
  for (int i = 0; i < n_meshes; ++i) {
    const dc_mesh_desc& md = meshes[i];
    Mesh& m = c->meshes[i];
    m.p = md.p;
    m.n_elem = md.n_elem;
    c->pmax = std::max(c->pmax, md.p);
    size_t npe = (size_t)(md.p + 1) * (md.p + 1) * (md.p + 1);
    size_t nb = sizeof(double) * npe * 3 * md.n_elem, bb = sizeof(float) * 6 * md.n_elem;
    if (cfg.mem_budget_bytes && c->mesh_bytes + nb + bb > cfg.mem_budget_bytes) {
      cudaFree(d_bad);
      return bail(fail(DC_ENOMEM, "mesh %d does not fit the memory budget", i));
    }
    if (dev_alloc(&m.nodes, nb) != cudaSuccess || dev_alloc(&m.box, bb) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(d_bad);
      return bail(fail(DC_ENOMEM, "mesh %d: cudaMalloc of %zu bytes failed", i, nb + bb));
    }
    c->mesh_bytes += nb + bb;
    cudaMemcpyKind kind = md.nodes_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpyAsync(m.nodes, md.nodes, nb, kind, st) != cudaSuccess) {
      cudaFree(d_bad);
      return bail(fail(DC_ECUDA, "mesh %d: copying nodes failed", i));
    }
    cudaMemsetAsync(d_bad, 0, 16, st);
    k_elem_boxes<<<fb_grid(md.n_elem, c->n_sm), 256, 0, st>>>(
        m.nodes, md.n_elem, (int)npe, m.box, d_bad, d_ext);
    const cudaError_t fe = cudaGetLastError();
    int bad[2] = {0, 0};
    double ext = 0.0;
    if (fe != cudaSuccess || cudaMemcpyAsync(bad, d_bad, 2 * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&ext, d_ext, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaStreamSynchronize(st);
      cudaFree(d_bad);
      return bail(fail(DC_ECUDA, "mesh %d: element boxes failed: %s", i,
                       cudaGetErrorString(fe != cudaSuccess ? fe : cudaGetLastError())));
    }
    if (bad[0]) {
      cudaFree(d_bad);
      return bail(fail(DC_EINVAL, "mesh %d has a NaN or infinite node", i));
    }
    m.h_elem = (float)(ext / (double)md.n_elem);
  }
  cudaFree(d_bad);
  if (cfg.reserve_faces > 0) {
    // every slot sized now for one request on the largest mesh, so that
    // dc_cut and dc_submit of such requests allocate nothing while serving
    long long ne_max = 0;
    for (auto& m : c->meshes) ne_max = std::max(ne_max, m.n_elem);
    const std::vector<SurfNeed> one{{(long long)cfg.reserve_faces, RESERVE_Q, true}};
    const size_t need = al256(arena_bytes(c, one, ne_max));
    const size_t n_slots = c->slots.size();
    // host staging of one slot: instance ring, counters, host flags
    const size_t ring_one = al256(sizeof(Inst)) + al256(sizeof(long long) * NOFF * 2);
    const size_t host_one = Slot::RING * ring_one + al256(sizeof(unsigned long long) * NCNT) + al256((size_t)ne_max);
    const size_t host_total = host_one * n_slots;
    if (!cfg.mem_budget_bytes || c->mesh_bytes + need * n_slots <= cfg.mem_budget_bytes) {
      if (dev_alloc(&c->dev_block, need * n_slots) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(DC_ENOMEM, "cudaMalloc(%zu) for the slots' arenas failed", need * n_slots));
      }
      c->dev_bytes = need * n_slots;
      if (host_alloc(&c->pin_block, host_total) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(DC_ENOMEM, "cudaMallocHost(%zu) for the slots' staging failed", host_total));
      }
      c->pin_bytes = host_total;
      char* hp = c->pin_block;
      auto take = [&](size_t bytes) { char* r = hp; hp += al256(bytes); return r; };
      for (size_t i = 0; i < n_slots; ++i) {
        Slot& s = c->slots[i];
        s.arena.base = c->dev_block + i * need;
        s.arena.cap = need;
        c->arena_bytes += need;
        for (int r = 0; r < Slot::RING; ++r) {
          s.ring_inst[r] = reinterpret_cast<Inst*>(take(sizeof(Inst)));
          s.ring_off[r] = reinterpret_cast<long long*>(take(sizeof(long long) * NOFF * 2));
        }
        s.h_inst_cap = 1;
        s.h_cnt = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * NCNT));
        s.h_flags = reinterpret_cast<int8_t*>(take((size_t)ne_max));
        s.h_out_cap = (size_t)ne_max;
      }
    }
  }
  *out = c;
  return DC_OK;
}

static dc_status run_sync(dc_ctx* c, const std::vector<InstReq>& v, bool async_ok, cudaStream_t user) {
  Slot& s = c->slots[0];
  cudaStream_t st = user ? user : s.stream;
  dc_status rc = enqueue(c, s, v, st, false);
  if (rc) return rc;
  if (async_ok) return DC_OK;
  // host outputs are copied in the same stream order, so finish's one
  // synchronisation covers them
  dc_status rc2 = copy_out_host(s, v, st);
  rc = finish(c, s, v, st);
  return rc ? rc : rc2;
}

dc_status dc_cut(dc_ctx* c, int32_t mesh, const dc_request* req) {
  g_err.clear();
  NvtxRange nr("directcut: dc_cut");
  if (!c) return fail(DC_EINVAL, "ctx is NULL");
  std::lock_guard<std::mutex> lk(c->mu);
  dc_status rc = validate_req(c, mesh, req);
  if (rc) return rc;
  if (req->async && !req->on_device) return fail(DC_EINVAL, "async requires device pointers");
  CK(cudaSetDevice(c->cfg.device));
  std::vector<InstReq> v{{mesh, req}};
  return run_sync(c, v, req->async != 0, (cudaStream_t)req->stream);
}

dc_status dc_cut_batch(dc_ctx* c, int32_t n, const int32_t* meshes, const dc_request* reqs) {
  g_err.clear();
  NvtxRange nr("directcut: dc_cut_batch");
  if (!c) return fail(DC_EINVAL, "ctx is NULL");
  if (n < 1 || !meshes || !reqs) return fail(DC_EINVAL, "empty batch");
  std::lock_guard<std::mutex> lk(c->mu);
  std::vector<InstReq> v;
  v.reserve(n);
  for (int i = 0; i < n; ++i) {
    dc_status rc = validate_req(c, meshes[i], &reqs[i]);
    if (rc) return rc;
    if (reqs[i].async) return fail(DC_EINVAL, "dc_cut_batch is synchronous; async must be 0");
    v.push_back({meshes[i], &reqs[i]});
  }
  CK(cudaSetDevice(c->cfg.device));
  return run_sync(c, v, false, (cudaStream_t)reqs[0].stream);
}

// ---------------------------------------------------------------- tuning

static dc_status check_tuning(const dc_ctx* c, const dc_tuning& t) {
  if (!(t.cubes_per_edge >= 0.5f && t.cubes_per_edge <= 4.0f))
    return fail(DC_EINVAL, "cubes_per_edge outside 0.5..4");
  if (t.bin_cubes < bin_floor(c->cfg) || t.bin_cubes > 16)
    return fail(DC_EINVAL, "bin_cubes outside %d..16", bin_floor(c->cfg));
  if (t.warps_per_cta != 4 && t.warps_per_cta != 8 && t.warps_per_cta != 16)
    return fail(DC_EINVAL, "warps_per_cta must be 4, 8 or 16");
  if (t.cands_per_warp != 1 && t.cands_per_warp != 2 && t.cands_per_warp != 4 && t.cands_per_warp != 8)
    return fail(DC_EINVAL, "cands_per_warp must be 1, 2, 4 or 8");
  return DC_OK;
}

dc_status dc_get_tuning(dc_ctx* c, dc_tuning* out) {
  g_err.clear();
  if (!c || !out) return fail(DC_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(c->mu);
  *out = c->tune;
  return DC_OK;
}

dc_status dc_set_tuning(dc_ctx* c, const dc_tuning* t) {
  g_err.clear();
  if (!c || !t) return fail(DC_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(c->mu);
  dc_status rc = check_tuning(c, *t);
  if (rc) return rc;
  c->tune = *t;
  c->tune.ms = 0.f;
  return DC_OK;
}

dc_status dc_autotune(dc_ctx* c, int32_t n, const int32_t* meshes, const dc_request* reqs, int32_t repeats,
                      dc_tuning* best, int32_t* n_trials) {
  g_err.clear();
  if (!c) return fail(DC_EINVAL, "ctx is NULL");
  if (n < 1 || !meshes || !reqs) return fail(DC_EINVAL, "empty batch");
  if (repeats < 1 || repeats > 50) return fail(DC_EINVAL, "repeats outside 1..50");
  std::lock_guard<std::mutex> lk(c->mu);
  std::vector<InstReq> v;
  v.reserve(n);
  for (int i = 0; i < n; ++i) {
    dc_status rc = validate_req(c, meshes[i], &reqs[i]);
    if (rc) return rc;
    if (reqs[i].async) return fail(DC_EINVAL, "dc_autotune is synchronous; async must be 0");
    v.push_back({meshes[i], &reqs[i]});
  }
  CK(cudaSetDevice(c->cfg.device));
  Slot& s = c->slots[0];
  const cudaStream_t st = reqs[0].stream ? (cudaStream_t)reqs[0].stream : s.stream;
  const dc_tuning saved = c->tune;
  std::vector<float> cpes;
  if (c->cfg.holemap_cells == 0) cpes = {1.2f, 1.8f, 2.7f};
  else cpes = {saved.cubes_per_edge};
  std::vector<int> bins;
  for (int b : {2, 4, 8})
    if (b >= bin_floor(c->cfg)) bins.push_back(b);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(DC_ECUDA, "cudaEventCreate failed");
  }
  auto done = [&](dc_status rc) {
    if (rc) c->tune = saved;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
  };
  dc_tuning bt = saved;
  float bms = INFINITY;
  int trials = 0;
  std::vector<float> t(repeats);
  // launch shapes outermost: each graph of a shape is captured once and
  // replayed for the hole-map settings (instance data, not graph keys)
  for (int wpc : {4, 8, 16})
    for (int cpw : {1, 2, 4, 8})
      for (float cpe : cpes)
        for (int bc : bins) {
          c->tune = dc_tuning{cpe, bc, wpc, cpw, 0.f};
          dc_status rc = run_sync(c, v, false, st);  // untimed
          if (rc) return done(rc);
          for (int r = 0; r < repeats; ++r) {
            if (cudaEventRecord(e0, st) != cudaSuccess) return done(fail(DC_ECUDA, "cudaEventRecord failed"));
            rc = enqueue(c, s, v, st, false);
            if (rc) return done(rc);
            if (cudaEventRecord(e1, st) != cudaSuccess) return done(fail(DC_ECUDA, "cudaEventRecord failed"));
            rc = finish(c, s, v, st);
            if (rc) return done(rc);
            if (cudaEventElapsedTime(&t[r], e0, e1) != cudaSuccess) return done(fail(DC_ECUDA, "cudaEventElapsedTime failed"));
          }
          std::vector<float> u = t;
          std::nth_element(u.begin(), u.begin() + repeats / 2, u.end());
          const float med = u[repeats / 2];
          ++trials;
          if (med < bms) {
            bms = med;
            bt = c->tune;
          }
        }
  bt.ms = bms;
  c->tune = bt;
  dc_status rc = run_sync(c, v, false, st);  // the outputs, with the chosen setting
  if (rc) return done(rc);
  if (best) *best = bt;
  if (n_trials) *n_trials = trials;
  return done(DC_OK);
}

dc_status dc_get_stats(dc_ctx* c, dc_stats* out) {
  if (!c || !out) return fail(DC_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(c->mu);
  *out = c->last;
  return DC_OK;
}

dc_status dc_submit(dc_ctx* c, int32_t mesh, const dc_request* req, uint64_t* ticket) {
  g_err.clear();
  NvtxRange nr("directcut: dc_submit");
  if (!c || !ticket) return fail(DC_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(c->mu);
  dc_status rc = validate_req(c, mesh, req);
  if (rc) return rc;
  if (req->fp32_dist_out) return fail(DC_EINVAL, "fp32_dist_out is for dc_cut and dc_cut_batch");
  CK(cudaSetDevice(c->cfg.device));
  // slot 0 stays reserved for dc_cut; serving uses the others (or slot 0 when
  // only one exists)
  int pick = -1;
  for (int i = (c->slots.size() > 1 ? 1 : 0); i < (int)c->slots.size(); ++i)
    if (!c->slots[i].busy) { pick = i; break; }
  if (pick < 0) return fail(DC_EBUSY, "all %zu serving slots are in flight", c->slots.size());
  Slot& s = c->slots[pick];
  std::vector<InstReq> v{{mesh, req}};
  rc = enqueue(c, s, v, s.stream, true);
  if (rc) return rc;
  long long ne = c->meshes[mesh].n_elem;
  s.host_out = !req->on_device;
  s.user_flags = req->flags_out;
  s.user_dist = req->dist_out;
  s.out_n = ne;
  if (s.host_out) {
    CK(cudaMemcpyAsync(s.h_flags, s.h_inst[0].flags, (size_t)ne, cudaMemcpyDeviceToHost, s.stream));
    if (req->dist_out) CK(cudaMemcpyAsync(s.h_dist, s.h_inst[0].dist, sizeof(double) * ne, cudaMemcpyDeviceToHost, s.stream));
  }
  CK(cudaMemcpyAsync(s.h_cnt, s.d_cnt, sizeof(unsigned long long) * NCNT, cudaMemcpyDeviceToHost, s.stream));
  CK(cudaEventRecord(s.done, s.stream));
  s.busy = true;
  s.ticket = c->next_ticket++;
  *ticket = s.ticket;
  return DC_OK;
}

dc_status dc_poll(dc_ctx* c, uint64_t ticket, int64_t timeout_us) {
  g_err.clear();
  if (!c) return fail(DC_EINVAL, "ctx is NULL");
  auto t0 = std::chrono::steady_clock::now();
  while (true) {
    {
      std::lock_guard<std::mutex> lk(c->mu);
      Slot* s = nullptr;
      for (auto& x : c->slots)
        if (x.busy && x.ticket == ticket) s = &x;
      if (!s) return fail(DC_ENOTFOUND, "ticket %llu is not in flight", (unsigned long long)ticket);
      cudaError_t q = cudaEventQuery(s->done);
      if (q == cudaSuccess) {
        std::vector<InstReq> none;
        CK(cudaMemcpyAsync(s->h_inst, s->d_inst, sizeof(Inst) * s->n_inst, cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        int err = 0;
        for (int i = 0; i < s->n_inst; ++i) err |= s->h_inst[i].err;
        const bool barrier_out = (s->h_cnt[22] >> 32) != 0;
        if (s->host_out) {
          memcpy(s->user_flags, s->h_flags, (size_t)s->out_n);
          if (s->user_dist) memcpy(s->user_dist, s->h_dist, sizeof(double) * s->out_n);
        }
        s->busy = false;
        if (barrier_out) return fail(DC_EINTERNAL, "a grid barrier of the hole-map kernel timed out");
        if (err & ERR_NONFINITE) return fail(DC_EINVAL, "a face node is NaN or infinite");
        if (err & ERR_DEGENERATE) return fail(DC_EINVAL, "the cut surface has zero extent");
        if (err & (ERR_ROUNDS | ERR_RECHECK)) return fail(DC_EINTERNAL, "exact test capacity exceeded (0x%x)", err);
        return DC_OK;
      }
      if (q != cudaErrorNotReady) {
        s->busy = false;
        return fail(DC_ECUDA, "ticket %llu failed: %s", (unsigned long long)ticket, cudaGetErrorString(q));
      }
    }
    auto el = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count();
    if (timeout_us >= 0 && el >= timeout_us) return DC_PENDING;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

void dc_destroy(dc_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->cfg.device);
  for (auto& s : c->slots) free_slot(c, s);
  if (c->pin_block) cudaFreeHost(c->pin_block);
  if (c->dev_block) cudaFree(c->dev_block);
  for (auto& m : c->meshes) {
    if (m.nodes) cudaFree(m.nodes);
    if (m.box) cudaFree(m.box);
  }
  delete c;
}

}  // extern "C"

// ------------------------------------------------------------------ allocation-free cut
// Some callers cannot allocate device memory when they cut: real-time loops
// that forbid allocation after start-up (cudaMalloc and cudaFree may block and
// synchronise the device, so their latency has no bound), and hosts whose own
// allocator owns every device byte (a framework's caching pool that reserves
// the GPU's memory up front, where a second allocator would fail or fragment
// it).  dc_cut_noalloc serves them: the same cut as dc_cut for one grid, with
// every scratch buffer carved from the fixed array below, which each GPU that
// loads this library holds until the process exits.  In host code
// `g_noalloc_scratch` only names a host-side stand-in for the symbol, never a
// device address: the address the kernels get comes from
// cudaGetSymbolAddress, once per device, with that device current.
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(8) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {
struct NoallocDevice {
  bool ready = false;
  unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch
  int n_sm = 0;
  int smem_optin = 0;
};
std::mutex g_noalloc_mu;
NoallocDevice g_noalloc_dev[64];

// first call on a device: symbol address, triangle tables, kernel attributes
dc_status noalloc_setup(int dev, NoallocDevice& d) {
  if (d.ready) return DC_OK;
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess) return fail(DC_ECUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
  static unsigned char et[MAX_P][MAX_NTE][3], ft[MAX_Q][MAX_NTF][3];
  build_tables(et, ft);
  CK(cudaMemcpyToSymbol(c_etri, et, sizeof(et)));
  CK(cudaMemcpyToSymbol(c_ftri, ft, sizeof(ft)));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, dev));
  cudaFuncAttributes fe, fd;
  CK(cudaFuncGetAttributes(&fe, k_exact<float>));
  CK(cudaFuncGetAttributes(&fd, k_exact<double>));
  d.smem_optin = (int)prop.sharedMemPerBlockOptin;
  CK(cudaFuncSetAttribute(k_exact<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(d.smem_optin - fe.sharedSizeBytes)));
  CK(cudaFuncSetAttribute(k_exact<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(d.smem_optin - fd.sharedSizeBytes)));
  d.n_sm = prop.multiProcessorCount;
  d.scratch = (unsigned char*)ptr;
  d.ready = true;
  return DC_OK;
}
}  // namespace

extern "C" dc_status dc_cut_noalloc(int32_t p, int64_t n_elem, const double* nodes, int32_t q, int64_t n_faces,
                                    const double* face_nodes, const double* pose, double tol, int8_t* flags_out,
                                    double* dist_out, void* stream) {
  g_err.clear();
  if (p < 1 || p > MAX_P) return fail(DC_EINVAL, "element order p=%d outside 1..%d", p, MAX_P);
  if (q < 1 || q > MAX_Q) return fail(DC_EINVAL, "face order q=%d outside 1..%d", q, MAX_Q);
  if (n_elem < 1 || n_faces < 1) return fail(DC_EINVAL, "n_elem and n_faces must be positive");
  if (!nodes || !face_nodes || !flags_out) return fail(DC_EINVAL, "nodes, face_nodes and flags_out are required");
  if (tol == 0.0) tol = 1e-7;
  if (!(tol > 0.0) || !std::isfinite(tol)) return fail(DC_EINVAL, "tol must be positive and finite");
  if (pose)
    for (int i = 0; i < 12; ++i)
      if (!std::isfinite(pose[i])) return fail(DC_EINVAL, "pose has a non-finite entry");
  const int bin_cubes = 4, cells = 64;
  const int nb = nbins_cap(bin_cubes);
  const int npe = (p + 1) * (p + 1) * (p + 1), npf = (q + 1) * (q + 1);
  // scratch plan (bytes, 256-aligned pieces)
  size_t need = al256(sizeof(Inst)) + al256(sizeof(long long) * 4) + al256(sizeof(float) * 6 * n_elem) +
                al256(sizeof(unsigned long long) * n_elem) * 2 + al256(sizeof(unsigned long long) * NCNT) +
                al256(sizeof(double) * n_faces * npf * 3) +
                al256(sizeof(float) * n_faces * 6) * 2 + al256(sizeof(int) * n_faces) * 2 + al256(cube_bytes()) +
                al256(sizeof(int) * nb) + al256(sizeof(int) * (nb + 1)) + run_bytes() + al256(sizeof(int));
  if (need > NOALLOC_SCRATCH_BYTES)
    return fail(DC_EINVAL, "dc_cut_noalloc: %lld elements (p=%d) and %lld faces (q=%d) need %zu bytes of scratch; "
                "the fixed array holds %zu", (long long)n_elem, p, (long long)n_faces, q, need, NOALLOC_SCRATCH_BYTES);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(DC_EINVAL, "device ordinal %d not supported", dev);
  NoallocDevice& D = g_noalloc_dev[dev];
  dc_status rc = noalloc_setup(dev, D);
  if (rc) return rc;
  // every check and query that can fail comes before the first queued copy:
  // once work is on the stream, a failure waits for it before returning, so
  // the lock is never released with work still running on the shared array
  const int TB = 256;
  const ExLayout Lf = ex_layout(p, q, 4), Ld = ex_layout(p, q, 8);
  const int WPB = TB / 32;
  if ((long long)Ld.total * WPB > D.smem_optin)
    return fail(DC_EINVAL, "orders p=%d q=%d need %d bytes of shared memory per block", p, q, Ld.total * WPB);
  int occ = 0, occd = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_exact<float>, TB, (size_t)Lf.total * WPB));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occd, k_exact<double>, TB, (size_t)Ld.total * WPB));
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* pp = D.scratch;
  auto take = [&](size_t bytes) { unsigned char* r = pp; pp += al256(bytes); return r; };
  Inst* d_inst = (Inst*)take(sizeof(Inst));
  long long* d_off = (long long*)take(sizeof(long long) * 4);
  float* ebox = (float*)take(sizeof(float) * 6 * n_elem);
  unsigned long long* cand = (unsigned long long*)take(sizeof(unsigned long long) * n_elem);
  unsigned long long* redo = (unsigned long long*)take(sizeof(unsigned long long) * n_elem);
  unsigned long long* d_cnt = (unsigned long long*)take(sizeof(unsigned long long) * NCNT);
  Inst h;
  memset(&h, 0, sizeof(h));
  h.nodes = nodes;
  h.eaabb = ebox;
  h.n_elem = n_elem;
  h.p = p;
  h.faces_in = face_nodes;
  h.n_faces = n_faces;
  h.q = q;
  h.has_pose = pose ? 1 : 0;
  if (pose) memcpy(h.pose, pose, sizeof(double) * 12);
  h.flags = flags_out;
  h.dist = dist_out;
  h.surf = (double*)take(sizeof(double) * n_faces * npf * 3);
  h.fbox = (float*)take(sizeof(float) * n_faces * 6);
  h.fbin = (int*)take(sizeof(int) * n_faces);
  h.bin_faces = (int*)take(sizeof(int) * n_faces);
  h.bin_fbox = (float*)take(sizeof(float) * n_faces * 6);
  h.cube = (uint8_t*)take(cube_bytes());
  h.bin_cnt = (int*)take(sizeof(int) * nb);
  h.bin_off = (int*)take(sizeof(int) * (nb + 1));
  {
    const size_t rows = (size_t)MAX_DIM * MAX_DIM;
    h.row_cnt = (int*)take(sizeof(int) * rows);
    h.row_x = (int*)take(sizeof(int) * rows * ROW_XCAP);
  }
  int* d_bad = (int*)take(sizeof(int) * 2);  // [0] a non-finite node
  h.nbins_cap = nb;
  h.tol = tol;
  h.tol_f = float_up(tol);
  h.holemap_cells = cells;
  h.bin_cubes = bin_cubes;
  h.want_dist = dist_out ? 1 : 0;
  for (int a = 0; a < 3; ++a) { h.sbox_key[a] = ~0ULL; h.sbox_key[3 + a] = 0ULL; }
  long long off[4] = {0, n_faces, 0, n_elem};
  // from here on a failure first drains what was queued
  auto queued_fail = [&](const char* what, cudaError_t e) {
    cudaStreamSynchronize(st);
    return fail(DC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  };
#define CKQ(call)                                 \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return queued_fail(#call, e_); \
  } while (0)
  // the array keeps the previous call's contents: the instance record and
  // offsets are rewritten and the counters and the bad-node flag set to zero
  // here; the hole map, bins and row tables are cleared by the kernels
  // themselves (k_clear, k_tag, k_bin_scan), exactly as in a context's arena,
  // which is also reused from cut to cut
  CKQ(cudaMemcpyAsync(d_inst, &h, sizeof(Inst), cudaMemcpyHostToDevice, st));
  CKQ(cudaMemcpyAsync(d_off, off, sizeof(off), cudaMemcpyHostToDevice, st));
  CKQ(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long) * NCNT, st));
  CKQ(cudaMemsetAsync(d_bad, 0, sizeof(int) * 2, st));
  k_elem_boxes<<<fb_grid(n_elem, D.n_sm), 256, 0, st>>>(
      nodes, n_elem, npe, ebox, d_bad, nullptr);
  unsigned gf = (unsigned)((n_faces * TAG_R + TB - 1) / TB);
  k_surface<<<dim3((unsigned)((n_faces + SURF_FPB - 1) / SURF_FPB), 1), TB, 0, st>>>(d_inst);
  k_clear<<<dim3(64, 1), TB, 0, st>>>(d_inst);
  k_tag<<<gf, TB, 0, st>>>(d_inst, d_off, 1, n_faces);
  k_bin_scan<<<1, 1024, 0, st>>>(d_inst);
  CKQ(launch_rows(false, d_inst, d_off, 1, n_faces, n_faces * 2LL * q * q, st));
  CandList cl{cand, (unsigned long long)n_elem, d_cnt};
  CandList rl{redo, (unsigned long long)n_elem, d_cnt + 2};
  CandList none{redo, 0, d_cnt + 2};
  k_classify<<<(unsigned)((n_elem + TB - 1) / TB), TB, 0, st>>>(d_inst, d_off + 2, 1, n_elem, cl, d_cnt);
  k_exact<float><<<D.n_sm * std::max(occ, 1), TB, (size_t)Lf.total * WPB, st>>>(d_inst, cl, rl, p, q, d_cnt + 4);
  k_exact<double><<<D.n_sm * std::max(occd, 1), TB, (size_t)Ld.total * WPB, st>>>(d_inst, rl, none, p, q, d_cnt + 4);
  CKQ(cudaGetLastError());
  int bad[2] = {0, 0};
  CKQ(cudaMemcpyAsync(&h, d_inst, sizeof(Inst), cudaMemcpyDeviceToHost, st));
  CKQ(cudaMemcpyAsync(bad, d_bad, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
  CKQ(cudaStreamSynchronize(st));
#undef CKQ
  if (bad[0]) return fail(DC_EINVAL, "an element node is NaN or infinite");
  if (h.err & ERR_NONFINITE) return fail(DC_EINVAL, "a face node is NaN or infinite");
  if (h.err & ERR_DEGENERATE) return fail(DC_EINVAL, "the cut surface has zero extent");
  if (h.err & (ERR_ROUNDS | ERR_RECHECK)) return fail(DC_EINTERNAL, "exact test capacity exceeded (error bits 0x%x)", h.err);
  return DC_OK;
}

// ------------------------------------------------------------------ after the cut
// Union of cuts, artificial-boundary faces and the unblank step (Sec. 4.2
// final paragraphs; Algorithm "Artificial Boundary unblank procedure").  The
// element-parallel kernels are in dc_overset.cuh; their counts come back
// through a small library-owned device array, so these calls allocate nothing.
namespace {

static __device__ unsigned long long g_ov_count[64];  // one counter per device ordinal
std::mutex g_ov_mu;

dc_status ov_counter(unsigned long long** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(DC_EINVAL, "device ordinal %d beyond 63", dev);
  void* p = nullptr;
  CK(cudaGetSymbolAddress(&p, g_ov_count));
  *out = static_cast<unsigned long long*>(p) + dev;
  return DC_OK;
}

// blocks of 256 threads for n elements: at most 16 per SM of the current device
unsigned ov_grid(long long n) {
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      n_sm < 1)
    n_sm = 1;
  return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)n_sm * 16));
}

}  // namespace

extern "C" {

dc_status dc_blank_union(int32_t n_cuts, const int8_t* const* flags, const int32_t* kinds, int64_t n_elem,
                         int8_t* iblank_out, void* stream) {
  g_err.clear();
  if (n_cuts < 1 || n_cuts > OV_MAX_CUTS) return fail(DC_EINVAL, "n_cuts must be 1..%d", OV_MAX_CUTS);
  if (!flags || !kinds || !iblank_out || n_elem < 1) return fail(DC_EINVAL, "NULL argument or n_elem < 1");
  CutSet cs{};
  cs.n = n_cuts;
  for (int k = 0; k < n_cuts; ++k) {
    if (!flags[k]) return fail(DC_EINVAL, "flags[%d] is NULL", k);
    if (kinds[k] != DC_WALL && kinds[k] != DC_OVERSET) return fail(DC_EINVAL, "kinds[%d] is not DC_WALL or DC_OVERSET", k);
    cs.flags[k] = flags[k];
    cs.kind[k] = kinds[k] == DC_WALL ? OV_WALL : OV_OVERSET;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_blank_union<<<ov_grid(n_elem), 256, 0, st>>>(cs, (long long)n_elem, iblank_out);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return DC_OK;
}

dc_status dc_ab_faces(int64_t n_elem, const int8_t* iblank, const int64_t* neighbours, uint8_t* ab_mask,
                      int64_t* n_ab, void* stream) {
  g_err.clear();
  if (!iblank || !neighbours || !ab_mask || n_elem < 1) return fail(DC_EINVAL, "NULL argument or n_elem < 1");
  std::lock_guard<std::mutex> lk(g_ov_mu);
  unsigned long long* cnt = nullptr;
  dc_status rc = ov_counter(&cnt);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
  k_ab_faces<<<ov_grid(n_elem), 256, 0, st>>>((long long)n_elem, iblank, reinterpret_cast<const long long*>(neighbours),
                                               ab_mask, cnt);
  CK(cudaGetLastError());
  unsigned long long h = 0;
  CK(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (n_ab) *n_ab = (int64_t)h;
  return DC_OK;
}

dc_status dc_unblank(int32_t kind, int64_t n_elem, const int8_t* iblank_prev, const int8_t* flags_t,
                     const int8_t* flags_tp, int8_t* iblank_out, uint8_t* unblank_out, int64_t* n_unblank,
                     void* stream) {
  g_err.clear();
  if (kind != DC_WALL && kind != DC_OVERSET) return fail(DC_EINVAL, "kind is not DC_WALL or DC_OVERSET");
  if (!iblank_prev || !flags_t || !flags_tp || !iblank_out || !unblank_out || n_elem < 1)
    return fail(DC_EINVAL, "NULL argument or n_elem < 1");
  std::lock_guard<std::mutex> lk(g_ov_mu);
  unsigned long long* cnt = nullptr;
  dc_status rc = ov_counter(&cnt);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
  k_unblank<<<ov_grid(n_elem), 256, 0, st>>>(kind == DC_WALL ? OV_WALL : OV_OVERSET, (long long)n_elem, iblank_prev,
                                              flags_t, flags_tp, iblank_out, unblank_out, cnt);
  CK(cudaGetLastError());
  unsigned long long h = 0;
  CK(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (n_unblank) *n_unblank = (int64_t)h;
  return DC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- point connectivity
struct dc_pc {
  int device = 0, p = 0, n_sm = 0, root = -1, depth = 0;
  long long n_elem = 0;
  double* nodes = nullptr;
  float* loc = nullptr;
  double* org = nullptr;
  float* fbox = nullptr;
  double* ebox = nullptr;
  float* h = nullptr;
  PcNode* tree = nullptr;
  cudaStream_t stream = nullptr;
  size_t cap = 0;  // points the scratch below holds
  double *pts = nullptr, *xloc = nullptr, *ref = nullptr;
  int *ncand = nullptr, *cand = nullptr;
  long long* donor = nullptr;
  unsigned long long* cnt = nullptr;
  dc_pc_stats last{};
  std::mutex mu;
};

namespace {

float round_down(double x) {
  float f = (float)x;
  if ((double)f > x) f = std::nextafter(f, -INFINITY);
  return f;
}
float round_up(double x) {
  float f = (float)x;
  if ((double)f < x) f = std::nextafter(f, INFINITY);
  return f;
}

// balanced tree over the element boxes: the median of box coordinate
// (depth mod 6) of (min x, min y, min z, max x, max y, max z) splits each
// range; returns the node index (-1: empty range)
int pc_build(std::vector<PcNode>& T, std::vector<int>& idx, int lo, int hi, int depth, const std::vector<double>& box,
             int& maxdepth) {
  if (lo >= hi) return -1;
  maxdepth = std::max(maxdepth, depth + 1);
  const int axis = depth % 6, mid = lo + (hi - lo) / 2;
  std::nth_element(idx.begin() + lo, idx.begin() + mid, idx.begin() + hi, [&](int a, int b) {
    const double ka = box[6 * (size_t)a + axis], kb = box[6 * (size_t)b + axis];
    return ka < kb || (ka == kb && a < b);
  });
  const int node = (int)T.size();
  T.emplace_back();
  const int e = idx[mid];
  const int l = pc_build(T, idx, lo, mid, depth + 1, box, maxdepth);
  const int r = pc_build(T, idx, mid + 1, hi, depth + 1, box, maxdepth);
  PcNode& N = T[node];
  N.elem = e;
  N.left = l;
  N.right = r;
  N.pad = 0;
  for (int a = 0; a < 3; ++a) {
    N.elo[a] = round_down(box[6 * (size_t)e + a]);
    N.ehi[a] = round_up(box[6 * (size_t)e + 3 + a]);
    N.slo[a] = N.elo[a];
    N.shi[a] = N.ehi[a];
    for (int c : {l, r})
      if (c >= 0) {
        N.slo[a] = std::min(N.slo[a], T[c].slo[a]);
        N.shi[a] = std::max(N.shi[a], T[c].shi[a]);
      }
  }
  return node;
}

void pc_free(dc_pc* pc) {
  for (void* q : std::initializer_list<void*>{pc->nodes, pc->loc, pc->org, pc->fbox, pc->ebox, pc->h, pc->tree, pc->pts,
                                              pc->xloc, pc->ref, pc->ncand, pc->cand, pc->donor, pc->cnt})
    if (q) cudaFree(q);
  if (pc->stream) cudaStreamDestroy(pc->stream);
  delete pc;
}

dc_status pc_reserve(dc_pc* pc, size_t n) {
  if (pc->cap >= n) return DC_OK;
  const size_t m = std::max(n, pc->cap + pc->cap / 2);
  for (void* q : std::initializer_list<void*>{pc->pts, pc->xloc, pc->ref, pc->ncand, pc->cand, pc->donor})
    if (q) cudaFree(q);
  pc->pts = pc->xloc = pc->ref = nullptr;
  pc->ncand = pc->cand = nullptr;
  pc->donor = nullptr;
  pc->cap = 0;
  if (dev_alloc(&pc->pts, sizeof(double) * 3 * m) != cudaSuccess ||
      dev_alloc(&pc->xloc, sizeof(double) * 3 * m) != cudaSuccess ||
      dev_alloc(&pc->ref, sizeof(double) * 3 * m) != cudaSuccess || dev_alloc(&pc->ncand, sizeof(int) * m) != cudaSuccess ||
      dev_alloc(&pc->cand, sizeof(int) * PC_CAND * m) != cudaSuccess ||
      dev_alloc(&pc->donor, sizeof(long long) * m) != cudaSuccess)
    return fail(DC_ENOMEM, "point scratch for %zu points: cudaMalloc failed", m);
  pc->cap = m;
  return DC_OK;
}

}  // namespace

extern "C" {

dc_status dc_pc_create(int32_t device, int32_t p, int64_t n_elem, const double* nodes, int32_t nodes_on_device,
                       dc_pc** out) {
  g_err.clear();
  if (!out) return fail(DC_EINVAL, "out is NULL");
  *out = nullptr;
  if (p < 1 || p > PC_MAXP) return fail(DC_EINVAL, "order p=%d outside 1..%d", p, PC_MAXP);
  if (n_elem < 1 || n_elem >= (1LL << 31) - 1) return fail(DC_EINVAL, "n_elem=%lld out of range", (long long)n_elem);
  if (!nodes) return fail(DC_EINVAL, "nodes is NULL");
  int ndev = 0;
  CK(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(DC_EINVAL, "device %d does not exist", device);
  CK(cudaSetDevice(device));
  const int npe = (p + 1) * (p + 1) * (p + 1);
  const size_t nn = (size_t)n_elem * npe * 3;
  std::vector<double> hn;
  const double* hp = nodes;
  if (nodes_on_device) {
    hn.resize(nn);
    CK(cudaMemcpy(hn.data(), nodes, sizeof(double) * nn, cudaMemcpyDeviceToHost));
    hp = hn.data();
  }
  // FP64 boxes, sizes, the tree (host)
  std::vector<double> box(6 * (size_t)n_elem);
  std::vector<float> hs((size_t)n_elem);
  for (long long e = 0; e < n_elem; ++e) {
    const double* x = hp + (size_t)e * npe * 3;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int k = 0; k < npe; ++k)
      for (int a = 0; a < 3; ++a) {
        const double v = x[3 * k + a];
        if (!std::isfinite(v)) return fail(DC_EINVAL, "element %lld has a NaN or infinite node", e);
        lo[a] = std::min(lo[a], v);
        hi[a] = std::max(hi[a], v);
      }
    for (int a = 0; a < 3; ++a) { box[6 * e + a] = lo[a]; box[6 * e + 3 + a] = hi[a]; }
    hs[e] = (float)std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
  }
  std::vector<PcNode> T;
  T.reserve((size_t)n_elem);
  std::vector<int> idx((size_t)n_elem);
  for (long long e = 0; e < n_elem; ++e) idx[e] = (int)e;
  int depth = 0;
  const int root = pc_build(T, idx, 0, (int)n_elem, 0, box, depth);
  if (depth > PC_STACK) return fail(DC_EINVAL, "search tree depth %d exceeds the traversal stack", depth);
  dc_pc* pc = new dc_pc();
  pc->device = device;
  pc->p = p;
  pc->n_elem = n_elem;
  pc->root = root;
  pc->depth = depth;
  auto bail = [&](dc_status st) { pc_free(pc); return st; };
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return bail(fail(DC_ECUDA, "cudaGetDeviceProperties failed"));
  pc->n_sm = prop.multiProcessorCount;
  if (cudaStreamCreateWithFlags(&pc->stream, cudaStreamNonBlocking) != cudaSuccess ||
      dev_alloc(&pc->nodes, sizeof(double) * nn) != cudaSuccess ||
      dev_alloc(&pc->loc, sizeof(float) * nn) != cudaSuccess ||
      dev_alloc(&pc->org, sizeof(double) * 3 * n_elem) != cudaSuccess ||
      dev_alloc(&pc->fbox, sizeof(float) * 6 * n_elem) != cudaSuccess ||
      dev_alloc(&pc->ebox, sizeof(double) * 6 * n_elem) != cudaSuccess ||
      dev_alloc(&pc->h, sizeof(float) * n_elem) != cudaSuccess ||
      dev_alloc(&pc->tree, sizeof(PcNode) * T.size()) != cudaSuccess ||
      dev_alloc(&pc->cnt, sizeof(unsigned long long) * 4) != cudaSuccess)
    return bail(fail(DC_ENOMEM, "donor grid of %lld elements: cudaMalloc failed", (long long)n_elem));
  cudaStream_t st = pc->stream;
  if (cudaMemcpyAsync(pc->nodes, nodes, sizeof(double) * nn,
                      nodes_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(pc->ebox, box.data(), sizeof(double) * box.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(pc->h, hs.data(), sizeof(float) * hs.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(pc->tree, T.data(), sizeof(PcNode) * T.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return bail(fail(DC_ECUDA, "uploading the donor grid failed"));
  int* d_bad = nullptr;
  if (dev_alloc(&d_bad, 2 * sizeof(int)) != cudaSuccess) return bail(fail(DC_ENOMEM, "cudaMalloc failed"));
  cudaMemsetAsync(d_bad, 0, 2 * sizeof(int), st);
  int n_sm = 0;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
  cudaError_t ke = launch_frames(pc->nodes, (long long)n_elem, npe, pc->fbox, pc->loc, pc->org, d_bad, nullptr,
                                 std::max(n_sm, 1), st);
  int hb[2] = {0, 0};
  if (ke == cudaSuccess) ke = cudaMemcpyAsync(hb, d_bad, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
  const cudaError_t ks = cudaStreamSynchronize(st);
  if (ke == cudaSuccess) ke = ks;
  cudaFree(d_bad);
  if (ke != cudaSuccess) return bail(fail(DC_ECUDA, "element frames failed: %s", cudaGetErrorString(ke)));
  if (hb[1]) return bail(fail(DC_EINTERNAL, "a bulk copy of element nodes did not complete"));
  *out = pc;
  return DC_OK;
}

dc_status dc_pc_locate(dc_pc* pc, int64_t n_pts, const double* pts, const double* pose, int64_t* donor_out,
                       double* ref_out, int32_t on_device, void* stream) {
  g_err.clear();
  if (!pc) return fail(DC_EINVAL, "pc is NULL");
  if (n_pts < 0) return fail(DC_EINVAL, "n_pts < 0");
  if (n_pts > 0 && (!pts || !donor_out || !ref_out)) return fail(DC_EINVAL, "NULL argument");
  if (pose)
    for (int i = 0; i < 12; ++i)
      if (!std::isfinite(pose[i])) return fail(DC_EINVAL, "pose has a non-finite entry");
  std::lock_guard<std::mutex> lk(pc->mu);
  CK(cudaSetDevice(pc->device));
  pc->last = dc_pc_stats{};
  pc->last.n_points = n_pts;
  if (n_pts == 0) return DC_OK;
  dc_status rc = pc_reserve(pc, (size_t)n_pts);
  if (rc) return rc;
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : pc->stream;
  PcGrid G{pc->p, pc->n_elem, pc->nodes, pc->loc, pc->org, pc->ebox, pc->h, pc->tree, pc->root};
  PcQuery Q{};
  Q.n = n_pts;
  if (on_device) {
    Q.pts = pts;
  } else {
    CK(cudaMemcpyAsync(pc->pts, pts, sizeof(double) * 3 * n_pts, cudaMemcpyHostToDevice, st));
    Q.pts = pc->pts;
  }
  Q.has_pose = pose ? 1 : 0;
  if (pose) memcpy(Q.pose, pose, sizeof(Q.pose));
  Q.xloc = pc->xloc;
  Q.ncand = pc->ncand;
  Q.cand = pc->cand;
  Q.donor = on_device ? reinterpret_cast<long long*>(donor_out) : pc->donor;
  Q.ref = on_device ? ref_out : pc->ref;
  Q.cnt = pc->cnt;
  CK(cudaMemsetAsync(pc->cnt, 0, sizeof(unsigned long long) * 4, st));
  const unsigned gs = (unsigned)std::min<long long>((n_pts + 255) / 256, (long long)pc->n_sm * 16);
  k_pc_search<<<gs, 256, 0, st>>>(G, Q);
  CK(cudaGetLastError());
  const unsigned gn = (unsigned)std::min<long long>((n_pts + 127) / 128, (long long)pc->n_sm * 32);
  k_pc_newton<<<gn, 128, 0, st>>>(G, Q);
  CK(cudaGetLastError());
  if (!on_device) {
    CK(cudaMemcpyAsync(donor_out, pc->donor, sizeof(long long) * n_pts, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ref_out, pc->ref, sizeof(double) * 3 * n_pts, cudaMemcpyDeviceToHost, st));
  }
  unsigned long long h[4];
  CK(cudaMemcpyAsync(h, pc->cnt, sizeof(h), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  pc->last.candidates = (int64_t)h[0];
  pc->last.fp64_steps = (int64_t)h[2];
  pc->last.n_found = (int64_t)h[3];
  if (h[1]) return fail(DC_EINTERNAL, "%llu points had more than %d candidate elements", h[1], PC_CAND);
  return DC_OK;
}

dc_status dc_pc_get_stats(dc_pc* pc, dc_pc_stats* out) {
  g_err.clear();
  if (!pc || !out) return fail(DC_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(pc->mu);
  *out = pc->last;
  out->tree_depth = pc->depth;
  return DC_OK;
}

void dc_pc_destroy(dc_pc* pc) {
  if (!pc) return;
  cudaSetDevice(pc->device);
  cudaStreamSynchronize(pc->stream);
  pc_free(pc);
}

}  // extern "C"
