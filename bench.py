#!/usr/bin/env python3
"""Benchmark of the GB300 parallel direct cut.

Workload (one step = one full cut, every phase of the hot path): background
64^3 Q2 hexes (262,144 elements) on [-2,2]^3 curved by a sinusoidal node
displacement of 0.1 h, cut by a dimpled sphere (336 Gaussian dimples, 6144 Q2
faces).  The mesh is resident in HBM (created once); each step cuts it with
the surface (1.33 MB of face nodes, already on the device for `value`).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on stdout (rank 0).  value = |S*| / cut time: the necessary
element-face tests of one cut (the pairs any box-pruned exact method must
evaluate, counted once by the oracle into tests/golden/necessary_pairs.json)
resolved per second, summed over ranks; `effective_rate` = N_E * N_F / cut
time.  `e2e` is the same metric through the C ABI with host buffers (face
upload and flag download inside the timed region); `roofline` is the
flags-only exact stage (k_near_main, the dominant kernel) against the FP32 ALU
peak, with the algorithmic arithmetic of the exact test on S*; `cut_roofline`
is the whole cut against max(bytes / HBM peak, flops / FP32 peak);
`cpu_baseline` is the CPU oracle on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cut ms & element-face tests/s at 64^3 Q2 hexes; p50/p99 cut latency, vs plain"
UNIT = "element-face tests/s"
WORKLOAD = "dimpled sphere (6144 Q2 faces, 336 dimples) cutting 64^3 Q2 hexes (262,144 elements, sinusoidal 0.1h)"
# C_tt, the arithmetic of one triangle-triangle distance as the oracle's
# routine computes it (tests/flops/oracle_flops.cpp: orc_tritri counted with a
# counting number type, mean over near pairs): the per-unit cost of the
# algorithmic count
FLOPS_PER_PAIR = 2887.6
# the same for the kernels' own FP32 routine (tests/flops/kernel_flops.cu; a
# fused multiply-add counts 2): the per-pair cost of the executed-work figures
FLOPS_PER_PAIR_KERNEL = 936.5
# arithmetic of the plane-separation test every listed pair of the flags-only
# stage takes (two normals 30, two norms 12, two thresholds 18, six signed
# volumes 48, extrema and compares 16) plus its box test (15)
FLOPS_PER_SEP = 139.0
# Alg. cp0 key of one (element, face) pair: 4 corners rotated into the OBB
# axes (60), box distance (12), centroid distance (9), key (2)
FLOPS_PER_KEY = 83.0
# one Newton step of the donor search on a Q2 element: the 27-node map and
# Jacobian (27 x 32), the 1-D bases (72) and the 3x3 solve (60)
FLOPS_PER_NEWTON_STEP_Q2 = 996.0
# DRAM bytes (read + write) of one k_near_main launch at the scale workload,
# from the ncu capture summarised in profiles/k_near_main_scale64.md
# (8.338432 MB read + 0.046592 MB written); None once the kernel changes
K_NEAR_MAIN_TRAFFIC = 8_385_024
# resident-mesh bytes one cut must move: a FP32 box read and a flag written per
# element, the FP64 nodes of each element that needs the exact test (Q2: 27
# nodes x 3 x 8 B; its frame is formed from them), the FP64 face nodes (Q2:
# 9 x 3 x 8 B)
BYTES_PER_ELEM = 25
BYTES_PER_EXACT_ELEM = 648
BYTES_PER_FACE = 216
# kernels of one flags-only cut: the fused prep (pose, hole map, bins,
# classification), the flags-only exact stage, its small FP64 full-search pass
LAUNCHES_PER_CUT = 3


def bench_config(workload, n_elem, n_faces):
    """The `config` object of both arms' JSON lines (the same keys and values
    for the same workload)."""
    return {"workload": WORKLOAD if workload == "scale64" else workload, "n_elem": int(n_elem),
            "n_faces": int(n_faces), "p": 2, "q": 2,
            "l2": "GPU arm: flushed (256 MB write) between timed steps; CPU oracle arm: not applicable"}


def necessary(workload):
    """The oracle's count of the necessary pair set S* of a workload."""
    with open(os.path.join(ROOT, "tests", "golden", "necessary_pairs.json")) as f:
        return json.load(f)[workload]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def alu_peaks(dev_index):
    """FP32 and FP64 FMA peaks of this GPU, measured by bench_peaks.cu (8
    independent FMA chains per thread, full occupancy, best of several
    launches timed with CUDA events): the denominators of every ALU roofline
    here.  Returns TFLOP/s and the SM count the device reports."""
    import ctypes
    import torch
    from paper_1711_07663_gb300 import build as B
    lib = ctypes.CDLL(B.build_peaks())
    lib.bp_fma.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.c_int, ctypes.c_int,
                           ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double)]
    lib.bp_fma.restype = ctypes.c_int
    torch.cuda.set_device(dev_index)
    out = {"sm_count": torch.cuda.get_device_properties(dev_index).multi_processor_count}
    for name, fp64, iters, reps in (("fp32", 0, 1 << 16, 7), ("fp64", 1, 1 << 10, 5)):
        ms, fl = ctypes.c_float(0.0), ctypes.c_double(0.0)
        rc = lib.bp_fma(fp64, iters, 8, reps, ctypes.byref(ms), ctypes.byref(fl))
        if rc != 0:
            raise RuntimeError(f"FMA peak microbenchmark failed ({rc})")
        out[f"{name}_tflops"] = fl.value / (ms.value * 1e-3) / 1e12
        out[f"{name}_ms"] = ms.value
    out["how"] = ("bench_peaks.cu: 8 independent FMA chains per thread, 8 blocks of 256 threads per SM, "
                  "best of several launches by CUDA events; 1 FMA = 2 flops")
    return out


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return None


def _scale64():
    import workloads as W
    return W.dimpled_sphere_case()


def _mid32():
    import workloads as W
    return W.dimpled_sphere_case(n=32, m=16, seed=12)


def _plain16():
    import workloads as W
    return W.sphere_in_box(n=16, p=2, m=8, q=2, seed=1)


WORKLOADS = {"scale64": _scale64, "mid32": _mid32, "plain16": _plain16}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plain-steps", type=int, default=10)
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--tuning", default=None,
                    help="launch shapes cubes_per_edge,bin_cubes,warps_per_cta,cands_per_warp instead of the "
                         "autotuner's (for runs under a profiler, whose timings would mislead the tuner)")
    ap.add_argument("--serving-seconds", type=float, default=10.0,
                    help="length of the open-loop serving measurement (0: skip it)")
    ap.add_argument("--batch-steps", type=int, default=5,
                    help="timed runs of the 256-instance batch (0: skip it)")
    ap.add_argument("--precision-steps", type=int, default=3,
                    help="timed cuts of the 128^3 Q3 precision-stress workload per form (0: skip it)")
    ap.add_argument("--no-peaks", action="store_true",
                    help="skip the FMA peak measurement (rooflines then use the unit-count figure)")
    ap.add_argument("--locate-points", type=int, default=1 << 20,
                    help="points of the donor-search measurement (0: skip it)")
    ap.add_argument("--heuristic-steps", type=int, default=10,
                    help="timed cuts of the paper's truncating variant (0: skip it)")
    ap.add_argument("--workload", default="scale64", choices=sorted(WORKLOADS),
                    help="scale64 is the benchmark; the others are small cases for profiling")
    return ap.parse_args()


# ----------------------------------------------------------------- clocks
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------- distributed
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, world):
    """The largest x over the ranks of the default process group (a CUDA
    tensor under NCCL, a host tensor under gloo)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as D
    dev = "cuda" if D.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    D.all_reduce(t, op=D.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as D
        D.barrier()


# ----------------------------------------------------------------- CPU oracle leg
def cpu_oracle_sample(case, seconds, seed=0, threads=0):
    """Time the oracle (as it stands; `threads` host threads, 0 = all cores) on
    random elements of the workload until ~`seconds` of wall time.  Returns
    (elements done, seconds, threads); one whole cut takes seconds * N_E / done."""
    import oracle as O
    g = np.random.default_rng(seed)
    ncpu = threads or (os.cpu_count() or 1)
    done = 0
    t0 = time.perf_counter()
    # batches of ~1 s of work for long samples; short ones still give every
    # thread a full chunk (the oracle schedules 16 elements at a time)
    batch = max(16 * ncpu, int(64 * ncpu * min(1.0, seconds)))
    while time.perf_counter() - t0 < seconds:
        ids = g.choice(case.n_elem, size=batch, replace=False)
        O.cut(case.p, case.nodes, case.q, case.faces, ids=ids, nthreads=threads)
        done += batch
    dt = time.perf_counter() - t0
    return done, dt, ncpu


def config1_oracle(n_sample=256, seed=7):
    """The oracle's two modes on the 16^3 Q2 plain workload (4096 elements, 384
    Q2 faces): branch and bound on the whole grid, and brute force (every
    triangle pair of every element-face pair) on a seeded sample of elements,
    scaled to the grid; both on all host threads, flags compared on the
    sample."""
    import oracle as O
    case = _plain16()
    t0 = time.perf_counter()
    flags, _, _, st = O.cut(case.p, case.nodes, case.q, case.faces)
    t_pruned = time.perf_counter() - t0
    ids = np.sort(np.random.default_rng(seed).choice(case.n_elem, size=n_sample, replace=False))
    t0 = time.perf_counter()
    fb, _, _, sb = O.cut(case.p, case.nodes, case.q, case.faces, ids=ids, brute=True)
    t_brute = time.perf_counter() - t0
    return {"workload": "16^3 Q2 hexes cut by a sphere of 384 Q2 faces (4096 elements)",
            "pruned_ms_per_cut": t_pruned * 1e3, "pruned_tritri_tests": int(st["tritri_tests"]),
            "brute_ms_per_cut": t_brute * case.n_elem / n_sample * 1e3,
            "brute_tritri_tests_per_s": sb["tritri_tests"] / t_brute,
            "brute_sample": f"{n_sample} seeded elements ({t_brute:.1f} s), scaled to all {case.n_elem}",
            "brute_same_flags": bool(np.array_equal(fb, flags[ids])), "threads": os.cpu_count()}


def run_reference(args, world, rank):
    if rank != 0:
        return
    case = WORKLOADS[args.workload]()
    s_star = necessary(args.workload)["s_star_pairs"]
    # the whole run stays within about --cpu-seconds, however many steps
    per_step = max(0.02, args.cpu_seconds / max(1, args.steps))
    cut_s = []
    n_el = 0
    for _ in range(args.warmup if args.warmup < 2 else 1):
        cpu_oracle_sample(case, 0.5, seed=99)
    for k in range(args.steps):
        done, dt, ncpu = cpu_oracle_sample(case, per_step, seed=k)
        cut_s.append(dt * case.n_elem / done)
        n_el += done
    ms = float(np.mean(cut_s)) * 1e3
    value = s_star / (ms * 1e-3)
    sample = (f"{n_el} random elements of the workload (of {case.n_elem}), {args.steps} steps of ~{per_step:.1f} s; "
              f"one cut = the sampled time scaled to all elements")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": bench_config(args.workload, case.n_elem, case.n_faces),
        "effective_rate": case.n_elem * case.n_faces / (ms * 1e-3),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ----------------------------------------------------------------- serving
def serving_measure(dc, W, dev, seconds, rate=200.0, seed=77):
    """Open-loop serving: requests arrive as a Poisson stream (mean `rate`
    per second) for `seconds` after a 1 s warm-up, each a cut of one of the
    resident 32^3 / 64^3 / 96^3 Q2 grids (probabilities 0.5 / 0.3 / 0.2) by the
    dimpled sphere turned 0.5 degrees per request.  A request is submitted at
    its arrival (dc_submit, host face nodes copied by the call; up to 3 in
    flight share the GPU, admitted as slots free up) and its latency is its
    completion (dc_poll) minus its arrival.  The plain path serves the same
    arrival stream one request at a time in arrival order (FIFO) with the
    FP64 exact stage, each a synchronous dc_cut; its latency is measured the
    same way.  Also: both paths' saturated rates (every request offered at
    once)."""
    import torch
    sizes = (32, 64, 96)
    meshes = [torch.from_numpy(W.background(n, 2, sinusoid=0.1)).to(dev) for n in sizes]
    faces_h = np.ascontiguousarray(W.dimpled_sphere_case(n=8, m=32, q=2).faces)
    g = np.random.default_rng(seed)
    axis = g.normal(size=3)
    warm = 1.0
    t_arr = np.cumsum(g.exponential(1.0 / rate, size=int((seconds + warm) * rate * 2) + 16))
    t_arr = t_arr[t_arr < seconds + warm]
    n_req = t_arr.size
    which = g.choice(3, size=n_req, p=[0.5, 0.3, 0.2])
    poses = [np.concatenate([W.axis_rotation(axis, np.deg2rad(0.5 * k)), np.zeros((3, 1))], axis=1)
             for k in range(n_req)]
    ring = 8
    outs = [[np.empty(n ** 3, dtype=np.int8) for _ in range(ring)] for n in sizes]
    keep = t_arr >= warm

    def open_loop(submit, poll):
        lat = np.full(n_req, np.nan)
        done_t = np.full(n_req, np.nan)
        pending = {}
        k = 0
        t0 = time.perf_counter()
        while k < n_req or pending:
            now = time.perf_counter() - t0
            while k < n_req and t_arr[k] <= now:
                tk = submit(k)
                if tk is None:
                    break
                pending[tk] = k
                k += 1
            for tk in list(pending):
                if poll(tk):
                    j = pending.pop(tk)
                    done_t[j] = time.perf_counter() - t0
                    lat[j] = done_t[j] - t_arr[j]
        return lat, done_t

    def summary(lat, done_t):
        L = lat[keep] * 1e3
        return {"requests": int(keep.sum()), "p50_ms": float(np.percentile(L, 50)),
                "p99_ms": float(np.percentile(L, 99)),
                "req_per_s": float(keep.sum() / (done_t[keep].max() - t_arr[keep].min()))}

    res = {"arrival_rate_per_s": rate, "seconds": seconds, "warmup_s": warm}
    with dc.Context([(2, m) for m in meshes], max_inflight=4) as ctx:
        # every serving slot warmed with every grid (arenas are reserved at
        # creation; this captures each slot's launch graphs)
        for w in range(3):
            tks = [ctx.submit(w, 2, faces_h, outs[w][j], pose=poses[0]) for j in range(3)]
            for tk in tks:
                ctx.poll(tk, timeout_us=-1)

        def submit(k):
            try:
                return ctx.submit(int(which[k]), 2, faces_h, outs[which[k]][k % ring], pose=poses[k])
            except dc.DirectCutError as e:
                if e.status != dc.DC_EBUSY:
                    raise
                return None

        lat, done_t = open_loop(submit, lambda tk: ctx.poll(tk, timeout_us=0) == 0)
        res.update(summary(lat, done_t))
        # saturated: every request offered at once
        pending = {}
        k = 0
        t1 = time.perf_counter()
        while k < n_req or pending:
            while k < n_req:
                tk = submit(k)
                if tk is None:
                    break
                pending[tk] = k
                k += 1
            for tk in list(pending):
                if ctx.poll(tk, timeout_us=0) == 0:
                    pending.pop(tk)
        res["saturated_req_per_s"] = float(n_req / (time.perf_counter() - t1))
    # the plain path: FP64 exact stage, one request on the GPU at a time,
    # served in arrival order
    with dc.Context([(2, m) for m in meshes], precision=dc.DC_FP64, max_inflight=1) as pctx:
        for w in range(3):
            pctx.cut(w, 2, faces_h, outs[w][0], pose=poses[0])
        lat = np.full(n_req, np.nan)
        done_t = np.full(n_req, np.nan)
        t0 = time.perf_counter()
        for k in range(n_req):
            while time.perf_counter() - t0 < t_arr[k]:
                pass
            pctx.cut(int(which[k]), 2, faces_h, outs[which[k]][k % ring], pose=poses[k])
            done_t[k] = time.perf_counter() - t0
            lat[k] = done_t[k] - t_arr[k]
        plain = summary(lat, done_t)
        t1 = time.perf_counter()
        for k in range(n_req):
            pctx.cut(int(which[k]), 2, faces_h, outs[which[k]][k % ring], pose=poses[k])
        plain["saturated_req_per_s"] = float(n_req / (time.perf_counter() - t1))
    res["plain_fp64_fifo"] = plain
    res["how"] = ("host face nodes and host flags through dc_submit / dc_poll (3 serving slots) against a "
                  "DC_FP64 context serving the same arrivals one synchronous dc_cut at a time")
    return res


# ----------------------------------------------------------------- batching
def batch_measure(dc, W, dev, stream, flush, steps=5):
    """The 256-instance batch (8^3 to 40^3 Q2 grids, cubed spheres of 6 m^2
    Q2 faces, random rotation and offset each) as one dc_cut_batch with the
    autotuned launch shapes, against the plain path: the same 256 requests as
    single synchronous FP64 cuts one after another.  Requests per second of
    each (host wall time of the whole batch, inputs resident on the device,
    L2 flushed before each), device time of the batch by CUDA events, and
    whether the flags agree."""
    import torch
    t0 = time.perf_counter()
    cases = W.batch_cases()
    gen_s = time.perf_counter() - t0
    meshes = [(cs.p, torch.from_numpy(cs.nodes).to(dev)) for cs in cases]
    fdev = {}
    for cs in cases:
        key = id(cs.faces)
        if key not in fdev:
            fdev[key] = torch.from_numpy(cs.faces).to(dev)
    outs = [torch.empty(cs.n_elem, dtype=torch.int8, device=dev) for cs in cases]
    reqs = [dict(q=cs.q, faces=fdev[id(cs.faces)], flags_out=o, pose=cs.pose, stream=stream.cuda_stream)
            for cs, o in zip(cases, outs)]
    idx = list(range(len(cases)))
    res = {"instances": len(cases), "elements": int(sum(cs.n_elem for cs in cases)),
           "faces": int(sum(cs.n_faces for cs in cases)), "generate_s": gen_s}
    with dc.Context(meshes, precision=dc.DC_FP32_RECHECK) as ctx:
        tuning, trials = ctx.autotune(idx, reqs, repeats=3)
        for _ in range(2):
            ctx.cut_batch(idx, reqs)
        wall, dev_ms = [], []
        for k in range(steps):
            flush.fill_(k & 0xff)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            t1 = time.perf_counter()
            ctx.cut_batch(idx, reqs)
            wall.append(time.perf_counter() - t1)
            b.record(stream)
            torch.cuda.synchronize()
            dev_ms.append(a.elapsed_time(b))
        st = ctx.stats()
    fl32 = [o.clone() for o in outs]
    with dc.Context(meshes, precision=dc.DC_FP64, max_inflight=1, reserve_faces=-1) as pctx:
        for i in idx[:8]:
            pctx.cut(i, reqs[i]["q"], reqs[i]["faces"], outs[i], pose=reqs[i]["pose"], stream=stream.cuda_stream)
        flush.fill_(0)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for i in idx:
            pctx.cut(i, reqs[i]["q"], reqs[i]["faces"], outs[i], pose=reqs[i]["pose"], stream=stream.cuda_stream)
        plain_s = time.perf_counter() - t1
    same = all(bool(torch.equal(a, b)) for a, b in zip(fl32, outs))
    bw = float(np.median(wall))
    res.update({"tuning": dict(tuning, trials=trials), "batch_ms": bw * 1e3,
                "batch_device_ms": float(np.median(dev_ms)), "req_per_s": len(cases) / bw,
                "candidates": st["n_candidates"],
                "plain_fp64_sequential": {"ms": plain_s * 1e3, "req_per_s": len(cases) / plain_s},
                "speedup_req_per_s": (len(cases) / bw) / (len(cases) / plain_s), "same_flags": same,
                "how": "dc_cut_batch of all 256 (FP32 bulk + FP64 re-solve, autotuned) vs 256 synchronous "
                       "DC_FP64 dc_cut calls; wall time, inputs resident, L2 flushed before each timing"})
    return res


# ----------------------------------------------------------------- precision stress
def precision_measure(dc, W, dev, stream, flush, steps=3):
    """The precision-stress workload: 128^3 Q3 hexes (2,097,152 elements,
    3.2 GB FP64) against a Q3 sphere of 6*32*32 faces, with the lattice
    vertices the oracle-side script placed within 1e-4 h of the linearised
    surface (tests/golden/precision_stress.npz; the grazing fraction of the
    necessary pair set is the oracle's count).  The FP32 bulk with FP64
    re-solve against all-FP64: cut times, flag agreement (distance and flags-
    only forms), re-solve counts, and the distribution of the FP32 stage's own
    distance error |d32 - d64| / h over the exact-test elements."""
    import torch
    G = np.load(os.path.join(ROOT, "tests", "golden", "precision_stress.npz"))
    n, p, m, q = int(G["n"]), int(G["p"]), int(G["m"]), int(G["q"])
    h = 4.0 / n
    t0 = time.perf_counter()
    lat = W.hex_lattice(n, p)
    lat.reshape(-1, 3)[G["idx"]] = G["coords"]
    lat_d = torch.from_numpy(lat).to(dev).reshape(-1, 3)
    del lat
    gi = torch.from_numpy(W.gather_index(n, p)).to(dev)
    nodes = lat_d[gi.reshape(-1)].reshape(n ** 3, (p + 1) ** 3, 3).contiguous()
    del gi, lat_d
    faces = torch.from_numpy(W.cubed_sphere(m, q, radius=1.0)).to(dev)
    gen_s = time.perf_counter() - t0
    NE = n ** 3
    res = {"elements": NE, "faces": int(faces.shape[0]), "p": p, "q": q, "pi_g": float(G["pi_g"]),
           "moved_vertices": int(G["idx"].size), "s_star_pairs": int(G["s_star_pairs"]),
           "grazing_pairs": int(G["grazing_pairs"]), "crossing_pairs": int(G["crossing_pairs"]),
           "grazing_fraction": int(G["grazing_pairs"]) / int(G["s_star_pairs"]),
           "grazing_definition": "S* pairs with 0 < d(E,F) < 1e-4 h (oracle count)", "generate_s": gen_s}
    out = {}
    for name, prec in (("fp32_recheck", dc.DC_FP32_RECHECK), ("fp64", dc.DC_FP64)):
        f = torch.empty(NE, dtype=torch.int8, device=dev)
        d = torch.empty(NE, dtype=torch.float64, device=dev)
        d32 = torch.empty(NE, dtype=torch.float32, device=dev) if prec == dc.DC_FP32_RECHECK else None
        g = torch.empty(NE, dtype=torch.int8, device=dev)
        with dc.Context([(p, nodes)], precision=prec) as ctx:
            ctx.cut(0, q, faces, f, d, stream=stream.cuda_stream, fp32_dist_out=d32)
            st = ctx.stats()
            ctx.cut(0, q, faces, g, stream=stream.cuda_stream)
            ms, ms_f = [], []
            for k in range(steps):
                for form, lst in ((d, ms), (None, ms_f)):
                    flush.fill_(k & 0xff)
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    ctx.cut(0, q, faces, f if form is not None else g, form, stream=stream.cuda_stream)
                    b.record(stream)
                    torch.cuda.synchronize()
                    lst.append(a.elapsed_time(b))
        out[name] = (f.cpu().numpy(), d.cpu().numpy(), None if d32 is None else d32.cpu().numpy(), g.cpu().numpy(),
                     st, float(np.median(ms)), float(np.median(ms_f)))
    del nodes
    f32, dd32, e32, g32, s32, ms32, msf32 = out["fp32_recheck"]
    f64, dd64, _, g64, s64, ms64, msf64 = out["fp64"]
    fin = np.isfinite(dd64) & np.isfinite(e32) & ~np.isnan(e32)
    err = np.abs(e32[fin].astype(np.float64) - dd64[fin]) / h
    edges = [0.0] + [10.0 ** k for k in range(-14, -3)] + [np.inf]
    hist, _ = np.histogram(err, bins=edges)
    zero = int((err == 0).sum())
    res.update({
        "fp32_recheck": {"dist_ms": ms32, "flags_only_ms": msf32, "pairs_fp32": s32["pairs_bulk"],
                         "pairs_fp64_resolved": s32["pairs_recheck"], "fp64_redo_elements": s32["fallbacks"],
                         "candidates": s32["n_candidates"]},
        "fp64": {"dist_ms": ms64, "flags_only_ms": msf64, "pairs_fp64": s64["pairs_bulk"]},
        "speedup_dist": ms64 / ms32, "speedup_flags_only": msf64 / msf32,
        "same_flags": bool(np.array_equal(f32, f64) and np.array_equal(g32, g64) and np.array_equal(f32, g32)),
        "fp32_error_over_h": {"elements": int(fin.sum()), "exactly_zero": zero,
                              "bins_upper_edges": [float(x) for x in edges[1:]],
                              "counts": [int(c) - (zero if i == 0 else 0) for i, c in enumerate(hist)],
                              "max": float(err.max()) if err.size else None,
                              "median": float(np.median(err)) if err.size else None,
                              "note": "counts per bin (edges[i], edges[i+1]]; elements with error exactly 0 "
                                      "listed apart"},
    })
    return res


# ----------------------------------------------------------------- our arm
def run_ours(args, world, rank, local):
    import torch
    if world > 1:
        import torch.distributed as D
        D.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1711_07663_gb300 as dc
    from paper_1711_07663_gb300 import build as B
    import workloads as W

    if rank == 0 or not os.path.exists(dc.lib_path()):
        B.build()
        B.build_peaks()
    barrier(world)
    dc.load()
    # the ALU rooflines' denominators, measured on this GPU before anything else
    peaks = None if args.no_peaks else alu_peaks(local)
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count

    def fp32_peak(sm_max):
        if peaks:
            return peaks["fp32_tflops"], "measured (bench_peaks.cu)"
        return n_sm * 128 * 2 * sm_max * 1e6 / 1e12, f"{n_sm} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz"

    case = WORKLOADS[args.workload]()
    NE, NF = case.n_elem, case.n_faces
    nodes = torch.from_numpy(case.nodes).to(dev)
    faces = torch.from_numpy(case.faces).to(dev)
    flags = torch.empty(NE, dtype=torch.int8, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2

    ctx = dc.Context([(case.p, nodes)], precision=dc.DC_FP32_RECHECK, device=local)
    tuning, tune_trials = None, 0
    if args.tuning:
        v = args.tuning.split(",")
        tuning = {"cubes_per_edge": float(v[0]), "bin_cubes": int(v[1]), "warps_per_cta": int(v[2]),
                  "cands_per_warp": int(v[3]), "ms": 0.0}
        ctx.set_tuning(**{k: x for k, x in tuning.items() if k != "ms"})
    elif not args.no_autotune:
        # the autotuner's sweep of launch shapes on this workload (untimed)
        tuning, tune_trials = ctx.autotune([0], [dict(q=case.q, faces=faces, flags_out=flags)], repeats=3)
    for _ in range(args.warmup):
        ctx.cut(0, case.q, faces, flags, stream=stream.cuda_stream)
    torch.cuda.synchronize()

    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    exact_ms, redo_ms, bulk, rech, ncand, total_ms, full = [], [], [], [], [], [], []
    surf_ms, hm_ms, cls_ms = [], [], []
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.6)
    barrier(world)
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(k & 0xff)  # evict the previous step's data from L2 (untimed)
        ev0[k].record(stream)
        ctx.cut(0, case.q, faces, flags, stream=stream.cuda_stream)
        ev1[k].record(stream)
        st = ctx.stats()
        bulk.append(st["pairs_bulk"])
        full.append(st["near_pairs_full"])
        rech.append(st["pairs_recheck"])
        ncand.append(st["n_candidates"])
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop()
    # phase times from a separate context that records events between the
    # phases (outside the timed loop: the events cost time and split the
    # kernels' programmatic launch chain)
    with dc.Context([(case.p, nodes)], precision=dc.DC_FP32_RECHECK, profile=1, device=local) as pctx:
        if tuning is not None:
            pctx.set_tuning(**{k: v for k, v in tuning.items() if k != "ms"})
        for k in range(max(args.warmup, 3) + 20):
            flush.fill_(k & 0xff)
            pctx.cut(0, case.q, faces, flags, stream=stream.cuda_stream)
            if k < max(args.warmup, 3):
                continue
            st = pctx.stats()
            exact_ms.append(st["ms_exact"])
            redo_ms.append(st["ms_redo"])
            total_ms.append(st["ms_total"])
            surf_ms.append(st["ms_surface"])
            hm_ms.append(st["ms_holemap"])
            cls_ms.append(st["ms_classify"])
    step_ms = np.array([a.elapsed_time(b) for a, b in zip(ev0, ev1)])
    t_sum = max_over_ranks(float(step_ms.sum()), world)
    ms_per_step = t_sum / args.steps
    nec = necessary(args.workload)
    S_STAR = nec["s_star_pairs"]
    value = world * S_STAR / (ms_per_step * 1e-3)

    # plain single-instance FP64 path (same flags): "vs plain"
    plain_ms = None
    same_flags = None
    f_plain = torch.empty_like(flags)
    if args.plain_steps > 0:
      with dc.Context([(case.p, nodes)], precision=dc.DC_FP64, device=local) as pctx:
        pctx.cut(0, case.q, faces, f_plain, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        same_flags = bool(torch.equal(f_plain, flags))
        pe = []
        for k in range(args.plain_steps):
            flush.fill_(k & 0xff)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pctx.cut(0, case.q, faces, f_plain, stream=stream.cuda_stream)
            b.record(stream)
            torch.cuda.synchronize()
            pe.append(a.elapsed_time(b))
        plain_ms = float(np.median(pe))

    # end to end through the public API with host buffers
    faces_h = torch.from_numpy(case.faces).pin_memory()
    flags_h = torch.empty(NE, dtype=torch.int8).pin_memory()
    for _ in range(3):
        ctx.cut(0, case.q, faces_h, flags_h)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        ctx.cut(0, case.q, faces_h, flags_h)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, world)
    e2e_same = bool(torch.equal(flags_h, flags.cpu()))

    # the unblank step of a moving grid (two cuts of the resident grid, at t and
    # t + dt, in one batched call, then the set logic), overset kind
    ft = torch.empty_like(flags)
    ftp = torch.empty_like(flags)
    ib_prev = torch.ones_like(flags)
    ib = torch.empty_like(flags)
    unb = torch.empty(NE, dtype=torch.uint8, device=dev)
    import workloads as Wl
    def step_poses(k):
        return [np.concatenate([Wl.axis_rotation([0.2, 0.9, 0.4], np.deg2rad(0.5 * (k + j))), np.zeros((3, 1))], axis=1)
                for j in (0, 1)]
    ub_ms = []
    for k in range(8 + args.warmup):
        pt, ptp = step_poses(k)
        flush.fill_(k & 0xff)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.cut_batch([0, 0], [dict(q=case.q, faces=faces, flags_out=ft, pose=pt),
                               dict(q=case.q, faces=faces, flags_out=ftp, pose=ptp)])
        dc.dc_unblank(dc.DC_OVERSET, ib_prev, ft, ftp, ib, unb, stream=stream.cuda_stream)
        b.record(stream)
        torch.cuda.synchronize()
        ib_prev, ib = ib, ib_prev
        if k >= args.warmup:
            ub_ms.append(a.elapsed_time(b))

    # the paper's truncating variant on the same workload: its time and how
    # many flags differ from the exact cut (flags of the timed loop above)
    heur = None
    if args.heuristic_steps > 0:
        hflags = torch.empty_like(flags)
        with dc.Context([(case.p, nodes)], precision=dc.DC_HEURISTIC, device=local) as hctx:
            for _ in range(2):
                hctx.cut(0, case.q, faces, hflags, stream=stream.cuda_stream)
            hms = []
            for k in range(args.heuristic_steps):
                flush.fill_(k & 0xff)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                hctx.cut(0, case.q, faces, hflags, stream=stream.cuda_stream)
                b.record(stream)
                torch.cuda.synchronize()
                hms.append(a.elapsed_time(b))
            hst = hctx.stats()
        ex, hv = flags.cpu().numpy(), hflags.cpu().numpy()
        ncand_h = float(np.mean(ncand))
        # the paper's variant per candidate: every face's key, 16 faces x 12
        # corner-triangle pairs, 4 faces x 3 element faces x 2p^2 x 2q^2 pairs
        hflops = ncand_h * (NF * FLOPS_PER_KEY + (16 * 12 + 4 * 3 * 2 * case.p ** 2 * 2 * case.q ** 2) * FLOPS_PER_PAIR)
        hpeak = fp32_peak(clocks.get("sm_max_mhz") or 2070.0)[0]
        heur = {"ms": float(np.median(hms)), "disagree": int((ex != hv).sum()),
                "roofline": {"bound": "alu", "achieved": hflops / (float(np.median(hms)) * 1e-3) / 1e12, "peak": hpeak,
                             "unit": "TFLOP/s", "frac": hflops / (float(np.median(hms)) * 1e-3) / 1e12 / hpeak,
                             "flops_per_cut": hflops, "scope": "whole variant cut (keys, pass 1, pass 2)"},
                "missed_fringe": int(((ex == dc.DC_FRINGE) & (hv != dc.DC_FRINGE)).sum()),
                "false_fringe": int(((ex != dc.DC_FRINGE) & (hv == dc.DC_FRINGE)).sum()),
                "side_differs": int(((ex != dc.DC_FRINGE) & (hv != dc.DC_FRINGE) & (ex != hv)).sum()),
                "fp64_key_rescans": hst["heur_rescans"], "fp64_pass1_resolves": hst["heur_resolves"]}

    # donor search after the cut: flux points of a near-body grid's overset
    # region (a body-fitted Q2 shell, 6*32*32*8 elements between radii 1 and
    # 1.6) located in it, the grid turned by a rigid pose; points, donors and
    # reference coordinates resident on the device
    pconn = None
    if args.locate_points > 0:
        shell = W.sphere_shell(32, 8, 2, 1.0, 1.6)
        qpts = torch.from_numpy(W.shell_points(args.locate_points, 1.0, 1.6, seed=17, order="morton")).to(dev)
        ppose = np.concatenate([W.axis_rotation([0.1, 0.7, 0.7], 0.3), np.array([[0.05], [-0.02], [0.01]])], axis=1)
        moved = (qpts @ torch.from_numpy(ppose[:, :3].T.copy()).to(dev) + torch.from_numpy(ppose[:, 3].copy()).to(dev))
        moved = moved.contiguous()
        pdon = torch.empty(args.locate_points, dtype=torch.int64, device=dev)
        pref = torch.empty((args.locate_points, 3), dtype=torch.float64, device=dev)
        with dc.PointLocator(2, torch.from_numpy(shell).to(dev), device=local) as pl:
            for _ in range(2):
                pl.locate(moved, pose=ppose, donor_out=pdon, ref_out=pref, stream=stream.cuda_stream)
            lms = []
            for k in range(5):
                flush.fill_(k & 0xff)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                pl.locate(moved, pose=ppose, donor_out=pdon, ref_out=pref, stream=stream.cuda_stream)
                b.record(stream)
                torch.cuda.synchronize()
                lms.append(a.elapsed_time(b))
            pst = pl.stats()
            # the same points in random order (the scattered case)
            perm = torch.from_numpy(np.random.default_rng(18).permutation(args.locate_points)).to(dev)
            moved_r = moved[perm].contiguous()
            pl.locate(moved_r, pose=ppose, donor_out=pdon, ref_out=pref, stream=stream.cuda_stream)
            rms = []
            for k in range(3):
                flush.fill_(k & 0xff)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                pl.locate(moved_r, pose=ppose, donor_out=pdon, ref_out=pref, stream=stream.cuda_stream)
                b.record(stream)
                torch.cuda.synchronize()
                rms.append(a.elapsed_time(b))
        lm = float(np.median(lms))
        # algorithmic: Newton to convergence on every candidate box (4 steps
        # each) -- the containment checks the paper's search leaves
        pflops = pst["candidates"] * 4 * FLOPS_PER_NEWTON_STEP_Q2
        ppeak = fp32_peak(clocks.get("sm_max_mhz") or 2070.0)[0]
        pconn = {"elements": int(shell.shape[0]), "points": args.locate_points, "ms": lm,
                 "roofline": {"bound": "alu", "achieved": pflops / (lm * 1e-3) / 1e12, "peak": ppeak, "unit": "TFLOP/s",
                              "frac": pflops / (lm * 1e-3) / 1e12 / ppeak, "flops": pflops,
                              "scope": "search + Newton (k_pc_search, k_pc_newton)"},
                 "points_per_s": args.locate_points / (lm * 1e-3), "found": pst["n_found"],
                 "order": "Morton curve (receptor points come face by face)",
                 "random_order_ms": float(np.median(rms)),
                 "candidates": pst["candidates"], "fp64_steps": pst["fp64_steps"], "tree_depth": pst["tree_depth"]}

    serving = serving_measure(dc, W, dev, args.serving_seconds) if args.serving_seconds > 0 else None
    batch = batch_measure(dc, W, dev, stream, flush, args.batch_steps) if args.batch_steps > 0 else None
    precision = (precision_measure(dc, W, dev, stream, flush, args.precision_steps)
                 if args.precision_steps > 0 else None)

    # cold: the grid is not resident -- create the context from pinned host
    # nodes (upload, element boxes and frames), cut once, destroy it
    cold = []
    nodes_h = torch.from_numpy(case.nodes).pin_memory()
    for _ in range(3):
        torch.cuda.synchronize()
        a = time.perf_counter()
        with dc.Context([(case.p, nodes_h)], precision=dc.DC_FP32_RECHECK, device=local) as cctx:
            cctx.cut(0, case.q, faces, flags, stream=stream.cuda_stream)
            torch.cuda.synchronize()
        cold.append((time.perf_counter() - a) * 1e3)

    # roofline of the dominant kernel (the flags-only exact stage): ALU bound.
    # Algorithmic arithmetic = the exact test on the necessary pair set S*:
    # |S*| x n_Tc x n_T(F) triangle pairs x C_tt (the oracle's triangle-pair
    # routine), with n_Tc = the 3 element faces at the nearest corner (lower
    # count) or all 6 (upper).  Executed arithmetic (what this kernel runs):
    # every listed triangle pair takes the separation test, the undecided ones
    # the kernels' full test.
    ex_ms = float(np.mean(exact_ms))
    pairs = float(np.mean(bulk))
    pairs_full = float(np.mean(full))
    flops_exec = pairs * FLOPS_PER_SEP + pairs_full * FLOPS_PER_PAIR_KERNEL
    flops_alg = S_STAR * nec["n_tc_lower"] * nec["n_tf"] * FLOPS_PER_PAIR
    flops_alg_upper = S_STAR * nec["n_tc_upper"] * nec["n_tf"] * FLOPS_PER_PAIR
    achieved = flops_alg / (ex_ms * 1e-3) / 1e12
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    peak, peak_basis = fp32_peak(sm_max)
    fp64_peak = peaks["fp64_tflops"] if peaks else None
    # the whole cut: T* = max(bytes / HBM peak, flops / FP32 peak)
    hbm = measured_peaks().get("hbm_gbs")
    cut_bytes = NE * BYTES_PER_ELEM + nec["exact_test_elements"] * BYTES_PER_EXACT_ELEM + NF * BYTES_PER_FACE
    t_bytes_us = cut_bytes / (hbm * 1e9) * 1e6 if hbm else None
    t_flops_us = flops_alg / (peak * 1e12) * 1e6
    t_star_us = max(t_flops_us, t_bytes_us or 0.0)
    # the plain FP64 path against the FP64 peak (the same algorithmic count)
    plain_roofline = None
    if plain_ms and fp64_peak:
        plain_roofline = {"bound": "alu", "achieved": flops_alg / (plain_ms * 1e-3) / 1e12, "peak": fp64_peak,
                          "unit": "TFLOP/s", "frac": flops_alg / (plain_ms * 1e-3) / 1e12 / fp64_peak,
                          "scope": "whole plain DC_FP64 cut, S* algorithmic flops", "peak_basis": "measured FP64 FMA"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        done, dt, ncpu = cpu_oracle_sample(case, args.cpu_seconds)
        d1, t1, _ = cpu_oracle_sample(case, max(2.0, args.cpu_seconds / 3), seed=5, threads=1)
        cpu = {"value": S_STAR * done / NE / dt, "unit": UNIT, "cores": ncpu, "kind": "oracle",
               "sample": f"{done} random elements of the workload ({dt:.1f} s, all {ncpu} host threads); "
                         f"one cut = the sampled time scaled to all {NE} elements",
               "single_thread_value": S_STAR * d1 / NE / t1, "cpu_model": cpu_model(),
               "config1": config1_oracle()}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "effective_rate": world * NE * NF / (ms_per_step * 1e-3), "s_star_pairs": S_STAR,
            "config": bench_config(args.workload, NE, NF),
            "precision": "fp32 bulk + fp64 re-solve", "mesh": "resident", "parallelism": f"replicas x{world}",
            "cut_ms_p50": float(np.percentile(step_ms, 50)), "cut_ms_p99": float(np.percentile(step_ms, 99)),
            "plain_fp64_ms": plain_ms, "speedup_vs_plain": (plain_ms / float(np.median(step_ms))) if plain_ms else None,
            "plain_same_flags": same_flags,
            "unblank_step_ms": float(np.median(ub_ms)),
            "cold_create_and_cut_ms": float(np.median(cold)),
            "tuning": None if tuning is None else dict(tuning, trials=tune_trials),
            "paper_truncating_variant": heur,
            "point_connectivity": pconn,
            "serving": serving,
            "phases_ms": {"prep": float(np.mean(surf_ms)) + float(np.mean(hm_ms)) + float(np.mean(cls_ms)),
                          "exact_fp32": ex_ms, "redo_fp64": float(np.mean(redo_ms)),
                          "library_total": float(np.mean(total_ms)),
                          "note": "separate profiled context (events between phases); prep = the fused kernel "
                                  "(pose, hole map, bins, classification)"},
            "candidates": int(np.mean(ncand)), "pairs_fp32": int(pairs), "pairs_fp64": int(np.mean(rech)),
            "e2e": {"value": world * S_STAR / e2e_s, "unit": UNIT, "ms_per_step": e2e_s * 1e3,
                    "h2d_bytes_per_step": int(case.faces.nbytes), "d2h_bytes_per_step": int(NE), "same_flags": e2e_same},
            "gpu_launches": LAUNCHES_PER_CUT * args.steps,
            "roofline": {"bound": "alu", "kernel": "k_near_main (flags-only exact stage)", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         # dram__bytes_read.sum + dram__bytes_write.sum of one launch of
                         # the current kernel (ncu, profiles/k_near_main_scale64.md)
                         "traffic": K_NEAR_MAIN_TRAFFIC,
                         "flops_per_launch": flops_alg, "flops_upper_count": flops_alg_upper,
                         "units": f"|S*| = {S_STAR} element-face pairs x {nec['n_tc_lower']} x {nec['n_tf']} "
                                  f"triangle pairs x C_tt = {FLOPS_PER_PAIR} flops (the oracle's triangle routine)",
                         "note": "frac above 1: the kernel settles the flags with less arithmetic than the "
                                 "method's exact test on S* (certified plane separation and crossings); its "
                                 "own limit is latency, see executed",
                         "executed": {"flops": flops_exec, "tflops": flops_exec / (ex_ms * 1e-3) / 1e12,
                                      "frac_fp32_peak": flops_exec / (ex_ms * 1e-3) / 1e12 / peak,
                                      "dram_bytes": K_NEAR_MAIN_TRAFFIC,
                                      "frac_hbm": (K_NEAR_MAIN_TRAFFIC / (ex_ms * 1e-3) / (hbm * 1e9)
                                                   if (K_NEAR_MAIN_TRAFFIC and hbm) else None),
                                      "pairs": pairs, "pairs_full_test": pairs_full,
                                      "flops_per_pair": {"separation": FLOPS_PER_SEP, "full": FLOPS_PER_PAIR_KERNEL}},
                         "duration_ms": ex_ms, "peak_basis": peak_basis},
            "cut_roofline": {"t_star_us": t_star_us, "t_flops_us": t_flops_us, "t_bytes_us": t_bytes_us,
                             "bytes": cut_bytes, "hbm_gbs": hbm, "frac": t_star_us / (ms_per_step * 1e3),
                             "bound": "alu" if t_flops_us >= (t_bytes_us or 0.0) else "hbm",
                             "peak_tflops": peak},
            "plain_fp64_roofline": plain_roofline,
            "alu_peaks": peaks,
            "batch256": batch,
            "precision_stress": precision,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        import torch.distributed as D
        D.destroy_process_group()


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
