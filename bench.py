#!/usr/bin/env python3
"""Benchmark: one-shot GWN queries/s on one GPU.

Default workload (one step), the largest single-GPU configuration: the
generalized winding number of a heightfield disk (2049^2 vertex grid mapped to
the unit disk, 16 sinusoids of amplitude 0.05; 32 circular holes remove
triangles, leaving 8,102,716 triangles and 33 boundary loops of 17,478 edges)
at every point of a 512^3 grid on [-1.1, 1.1]^3 (134,217,728 queries), for one
seeded ray direction: exact crossing counts + float32 boundary term +
epilogue, with the mesh, its boundary loops and its crossing index resident on
the device.  ``--workload icosphere_cap`` runs the same measurement on the
capped icosphere (73,724 triangles, 252 boundary edges, 256^3 grid).

JSON keys beyond the common contract:
  roofline      dominant kernel (boundary term) vs the FP32 issue roofline
  kernels       per-kernel average time from CUDA events on the launch stream
  prep_ms       per-geometry preparation (mesh upload with device boundary
                extraction, LBVH build, crossing-bin build), outside `value`
  bruteforce_gpu  the brute-force per-triangle solid-angle sum on the same GPU
  cpu_baseline  the FP64 oracle on this host's cores (bounded sample)
  e2e           through the C ABI from host buffers: mesh creation from host
                V/F, LBVH and bin builds, evaluation, w into a pinned host
                buffer, per step

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                       [--workload NAME]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "GWN queries/sec, one-shot vs brute-force solid-angle sum on 1 GB300 at |Δw|≤1e-6"
UNIT = "queries/s"
# The two workloads of the main measurement: each one mesh on a full 3D grid.
#   grid      default grid resolution per axis
#   traffic   DRAM bytes of one bterm3d_kernel launch at that grid, from ncu
#             (dram__bytes_read.sum + dram__bytes_write.sum), valid only
#             while the boundary-term sources (csrc/bterm.cu, bterm.cuh,
#             bterm_main_pass.inc) hash to `bterm_cu_sha256`
#   bf_planes grid planes (of z) timed for the brute-force comparator
#   cpu/ref   oracle queries for the CPU baseline and per reference-arm step
MAIN = {
    "holey_heightfield": {
        "label": "holey_heightfield_8102716tris_512^3grid", "grid": 512,
        "desc": "heightfield disk, 8,102,716 triangles, 33 boundary loops (17,478 edges), 512^3 grid on [-1.1,1.1]^3",
        # read 582.47 MB, write 503.97 MB: the 8 algorithmic bytes per query
        # (chi in, w out: 1073.7 MB) and nothing re-read
        "traffic": {"bytes": 1086.44e6, "bterm_cu_sha256": "994550d7d44c7a8bf1e72d1e66e500b7ac993c1c2f0a991fa72a48f01f78912f"},
        "bf_rows": 16, "cpu_sample": 192, "ref_sample": 48, "steps": 10,
    },
    "icosphere_cap": {
        "label": "icosphere_cap_s6_73724tris_256^3grid", "grid": 256,
        "desc": "icosphere s6 with the cap z>0.8 removed, 73,724 triangles, 252 boundary edges, 256^3 grid on "
                "[-1.2,1.2]^3",
        # read 67.31 MB, write 21.43 MB: DRAM writes fall below the 8 algorithmic
        # bytes per query because L2 still holds part of w when the kernel ends
        "traffic": {"bytes": 89.74e6,
                    "bterm_cu_sha256": "994550d7d44c7a8bf1e72d1e66e500b7ac993c1c2f0a991fa72a48f01f78912f"},
        "bf_rows": 1024, "cpu_sample": 4096, "ref_sample": 1024, "steps": 100,
    },
}

# FP32 lane operations per boundary record (vertex) and per boundary edge of
# the boundary-term kernel, counted from its formulation (an FMA counts as
# one operation):
#   vertex: a = A - p (3), projection on e1, e2, n (9), |a_perp|^2, |a|^2 (3),
#           rsqrt + scale + clamp (3), s = |a|+a_n or |a_perp|^2/(|a|-a_n) (6),
#           q = s |a| and the near-ray test (2)                               -> 26
#   edge:   num (2), den (3), atan2 (20: min/max 2, reciprocal + product 2,
#           degree-8 polynomial 10, reduction/quadrant fix-ups 6),
#           cut and spindle tests (2), compensated accumulation (4)             -> 31
W_VERTEX = 26
W_EDGE = 31
# FP32 lane operations per (query, boundary edge) pair of the fused backward
# pass (both gradients), on the path of the pairs with a.b >= 0 (every pair of
# the timed workloads but those whose query lies inside the sphere on the
# edge as diameter): a = A - p, b = B - p (6); c = a x E (6); |a|^2, |b|^2 with
# the clamp constant in the first FMA (6); rsqrt x 2 (2); 1/|a||b| (1); a.b
# (3); 1 + a.b/|a||b| (1); the sign test of a.b (1); reciprocal (1);
# 1/Q x dL/dw (2); J_A g, J_B g and their sum (3); per-edge and per-query
# accumulation (9)                                                        -> 41
W_GRAD_PAIR = 41
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        # nvidia-smi numbers GPUs by PCI order and ignores CUDA_VISIBLE_DEVICES,
        # so the device is named by its UUID (a read-only query either way)
        self.uuid = _gpu_uuid(gpu_index)
        self.gpu = str(gpu_index)
        if self.uuid:
            try:
                r = subprocess.run(["nvidia-smi", f"--id={self.uuid}", "--query-gpu=uuid", "--format=csv,noheader"],
                                   capture_output=True, text=True, timeout=20)
                if r.returncode == 0 and self.uuid in r.stdout:
                    self.gpu = self.uuid
            except Exception:
                pass
        self.proc = None
        self.path = os.path.join("/tmp", f"gwn_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "gpu_uuid": self.uuid,
                "smi_id": self.gpu}


def _gpu_uuid(index: int):
    """UUID string of torch's CUDA device `index` ("GPU-xxxxxxxx-..."), or None."""
    try:
        import torch
        u = torch.cuda.get_device_properties(index).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        return None


def make_mesh(name: str, grid_n: int | None = None):
    import gen
    grid_n = grid_n or MAIN[name]["grid"]
    if name == "holey_heightfield":
        return gen.holey_heightfield(grid_n=grid_n)
    return gen.icosphere_cap(grid_n=grid_n)


def workload(name: str = "holey_heightfield", rank: int = 0, world: int = 1, grid_n: int | None = None):
    from paper_2408_04466_gb300.shard import shard_grid
    m = make_mesh(name, grid_n)
    lo, hi, dims, span = shard_grid(m.grid.lo, m.grid.hi, m.grid.dims, rank, world, weak=True)
    return m, (lo, hi, dims)


# ----------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ----------------------------------------------------------------------------
def oracle_rate(m, n_sample: int, seed: int, want=False):
    import gen
    import oracle
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(m.grid.n, n_sample, replace=False))
    P = gen.grid_points(m.grid, index=idx)
    edges = oracle.boundary_edges(m.F)
    t0 = time.perf_counter()
    wo, chio, _ = oracle.w3d_oneshot(m.V, m.F, P, m.d, edges=edges)
    dt = time.perf_counter() - t0
    if want:
        return n_sample / dt, dt, (idx, P, wo, chio)
    return n_sample / dt, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    spec = MAIN[args.workload]
    m, _ = workload(args.workload, grid_n=args.grid)
    cores = oracle.default_threads()
    n = args.ref_sample or spec["ref_sample"]
    for w in range(args.warmup):
        oracle_rate(m, n, 1000 + w)
    times = []
    for s in range(args.steps):
        r, dt = oracle_rate(m, n, 2000 + s)
        times.append(dt)
    tot = sum(times)
    value = n * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": spec["label"], "queries_per_step": n, "l2": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n} seeded queries of the {m.grid.dims[0]}^3 grid per step; FP64 one-shot "
                                   f"(exact crossing count by brute force over all {len(m.F):,} triangles + "
                                   f"boundary term)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def run_gpu(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2408_04466_gb300 import build as gbuild
    if rank == 0 or world == 1:
        gbuild.build()
    if world > 1:
        dist.barrier()
    import paper_2408_04466_gb300 as gwn

    spec = MAIN[args.workload]
    m, (lo, hi, dims) = workload(args.workload, rank, world, args.grid)
    nq = int(np.prod(dims))
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    ctx = gwn.Context(local, stream)
    t0 = time.perf_counter()
    mesh = gwn.Mesh(ctx, m.V, m.F)
    t1 = time.perf_counter()
    mesh.prepare(m.d)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    prep = {"mesh_create_ms": 1e3 * (t1 - t0), "lbvh_build_ms": 1e3 * (t2 - t1)}
    info = mesh.info()
    E, L = info["n_boundary_edges"], info["n_loops"]
    grid = gwn.Grid(lo, hi, dims)
    w = torch.empty(nq, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # stats run (also a warm-up): per-kernel times and counters; on this first
    # evaluation the crossing bins are built (timed as its ms_prepare)
    st = mesh.eval(grid, m.d, stats=True, out=w)["stats"]
    prep["bins_build_ms"] = st["ms_prepare"]
    prep["bins"] = {k: mesh.info()[k] for k in ("n_bins", "n_bin_entries", "bin_maxlen")}
    for _ in range(args.warmup):
        mesh.eval(grid, m.d, out=w)
    torch.cuda.synchronize()

    # timed region: per step, flush L2 (256 MiB write), then time the step with
    # events on the launch stream; a second pair of events splits the kernels
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    for s in range(args.steps):
        flush.fill_(float(s))
        ev[s][0].record(stream)
        mesh.eval(grid, m.d, out=w)
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([tot_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
        tot_ms = float(t.item())
    value = world * nq * args.steps / (tot_ms * 1e-3)

    # per-kernel split: a stats call times traverse and boundary separately
    ks = []
    for _ in range(5 if nq <= (1 << 25) else 2):
        ks.append(mesh.eval(grid, m.d, stats=True, out=w)["stats"])
    ms_trav = statistics.median(k["ms_traverse"] for k in ks)
    ms_bterm = statistics.median(k["ms_boundary"] for k in ks)

    line = None
    if rank == 0 and args.no_extras:
        print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                          "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "grid": args.grid,
                          "kernels": {"traverse_ms": ms_trav, "bterm3d_ms": ms_bterm}}))
    elif rank == 0:
        peaks, peak_kind = _peaks()
        clk_hz = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
        alu_peak = SM_COUNT * FP32_LANES_PER_SM * clk_hz / 1e12          # Tops/s
        ops = nq * ((E + L) * W_VERTEX + E * W_EDGE)
        achieved = ops / (ms_bterm * 1e-3) / 1e12
        import hashlib
        hsh = hashlib.sha256()
        for fn in ("bterm.cu", "bterm.cuh", "bterm_main_pass.inc"):
            with open(os.path.join(ROOT, "paper_2408_04466_gb300", "csrc", fn), "rb") as f:
                hsh.update(f.read())
        src_hash = hsh.hexdigest()
        tr = spec["traffic"]
        same_src = tr is not None and src_hash == tr["bterm_cu_sha256"] and nq == MAIN[args.workload]["grid"] ** 3
        roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s (FP32 lane ops)",
                "frac": achieved / alu_peak, "traffic": tr["bytes"] if same_src else None,
                "traffic_unit": "bytes per launch (DRAM, ncu)", "kernel": "bterm3d_kernel",
                "peak_source": f"{SM_COUNT} SMs x {FP32_LANES_PER_SM} FP32 lanes x sm_max_mhz "
                               f"({peak_kind} MEASURED_PEAKS)" if peak_kind == "measured" else "fallback clock"}
        # brute-force comparator on a sub-grid: the first bf_rows rows (of x)
        # of the grid's middle z-plane
        nr = min(spec["bf_rows"], dims[1] * dims[2])
        zc = lo[2] + (hi[2] - lo[2]) * (dims[2] // 2) / (dims[2] - 1)
        if nr >= dims[1]:
            nz = nr // dims[1]
            sub = gwn.Grid(lo, (hi[0], hi[1], lo[2] + (hi[2] - lo[2]) * (nz - 1) / (dims[2] - 1)),
                           (dims[0], dims[1], nz))
        else:
            sub = gwn.Grid((lo[0], lo[1], zc), (hi[0], lo[1] + (hi[1] - lo[1]) * (nr - 1) / (dims[1] - 1), zc),
                           (dims[0], nr, 1))
        bw = torch.empty(sub.n, dtype=torch.float32, device=dev)
        mesh.bruteforce(sub)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            bw = mesh.bruteforce(sub)
        e1.record(stream)
        torch.cuda.synchronize()
        bf_rate = 3 * sub.n / (e0.elapsed_time(e1) * 1e-3)

        # end to end: host V/F (pinned) -> mesh, LBVH, eval, w -> pinned host
        Vh = torch.as_tensor(m.V).pin_memory()
        Fh = torch.as_tensor(m.F).pin_memory()
        wh = torch.empty(nq, dtype=torch.float32).pin_memory()
        import ctypes as C
        from paper_2408_04466_gb300 import _capi
        e2e_steps = max(3, min(args.steps, 10 if nq <= (1 << 25) else 3))
        times = []
        for s in range(e2e_steps + 1):
            torch.cuda.synchronize()
            a = time.perf_counter()
            mh = gwn.Mesh(ctx, Vh, Fh)
            qc = grid.to_c()
            _capi.check(ctx.lib.gwn_eval_host(mh.h, C.byref(qc), np.ascontiguousarray(m.d).ctypes.data_as(C.c_void_p),
                                              C.c_void_p(wh.data_ptr())), "gwn_eval_host")
            b = time.perf_counter()
            mh.close()
            if s > 0:
                times.append(b - a)
        e2e = {"value": nq / statistics.median(times), "unit": UNIT,
               "h2d_bytes_per_step": int(m.V.nbytes + m.F.nbytes), "d2h_bytes_per_step": int(nq * 4),
               "includes": "upload of V and F, mesh checks and boundary extraction, LBVH build, traversal, "
                           "boundary term writing w into the pinned host buffer"}

        # CPU baseline: the oracle on this host's cores, bounded sample
        import oracle
        oracle.build()
        n_cpu = args.cpu_sample or spec["cpu_sample"]
        rate, dt, (sidx, sP, wo, chio) = oracle_rate(m, n_cpu, 7, want=True)
        # parity on the same sample: crossing counts exactly, |dw| beyond 1e-4 x diagonal
        r = mesh.eval(grid, m.d, want_chi=True)
        torch.cuda.synchronize()
        ti = torch.as_tensor(sidx, device=dev)
        wg = r["w"][ti].double().cpu().numpy()
        chig = r["chi"][ti].cpu().numpy()
        diag = float(np.linalg.norm(m.V.max(0).astype(np.float64) - m.V.min(0)))
        far = oracle.dist3d(m.V, m.F, sP) > 1e-4 * diag
        parity = {"n": int(n_cpu), "chi_mismatch": int((chig != chio).sum()),
                  "max_abs_dw": float(np.abs(wg - wo)[far].max()) if far.any() else None,
                  "n_within_1e-4_diag": int((~far).sum()), "reference": "FP64 oracle on the cpu_baseline sample"}
        cpu = {"value": rate, "unit": UNIT, "cores": oracle.default_threads(), "kind": "oracle",
               "sample": f"{n_cpu} seeded queries of the {dims[0]}^3 grid; FP64 one-shot (brute-force exact crossing "
                         f"count over all triangles + boundary term); {dt:.1f} s"}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": spec["label"], "description": spec["desc"], "queries_per_gpu": nq, "boundary_edges": E, "boundary_loops": L,
                       "triangles": int(len(m.F)), "l2": "flushed (256 MiB write before every step)",
                       "parallelism": f"queries sharded in z-slabs over {world} GPU(s), geometry replicated"},
            "roofline": roof,
            "kernels": {"traverse_ms": ms_trav, "bterm3d_ms": ms_bterm,
                        "n_tri_tests_per_query": st["n_tri_tests"] / nq,
                        "n_cut_sign_per_query": st["n_cut_sign"] / nq,
                        "n_fp64_filter": st["n_fp64_filter"], "n_exact": st["n_exact"],
                        "deferred_traverse_per_query": st["n_deferred_traverse"] / nq,
                        "deferred_boundary_per_query": st["n_deferred_boundary"] / nq},
            "prep_ms": prep,
            "bruteforce_gpu": {"value": bf_rate, "unit": UNIT,
                               "sample": f"{sub.n} grid queries x {len(m.F):,} triangles"},
            "speedup_vs_bruteforce_gpu": value / world / bf_rate,
            "cpu_baseline": cpu,
            "parity_sample": parity,
            "e2e": e2e,
            # per step: packet traversal, deferred-pair settlement, whole-query
            # recount, boundary term, careful boundary pass (the list-length
            # memsets are not kernels)
            "gpu_launches": 5 * args.steps,
            "clocks": clk,
            "wall_s_timed": wall,
        }
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------
# other workloads (parity-test configurations), measured with --workload
# ----------------------------------------------------------------------------
def _alu_roofline(nq, info, ms):
    """Boundary-term FP32 roofline for nq queries against a mesh boundary."""
    peaks, kind = _peaks()
    peak = SM_COUNT * FP32_LANES_PER_SM * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    E, L = info["n_boundary_edges"], info["n_loops"]
    achieved = nq * ((E + L) * W_VERTEX + E * W_EDGE) / (ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s (FP32 lane ops)",
            "frac": achieved / peak, "peak_source": kind}


_TIMED_CLOCKS = []     # clock samples of each _timed region, for the workload's JSON line


def _timed(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for a, b in ev:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    _TIMED_CLOCKS.append(clocks.stop())
    return [a.elapsed_time(b) for a, b in ev]


def run_other(args):
    import torch
    import gen
    import oracle
    from paper_2408_04466_gb300 import build as gbuild
    gbuild.build()
    oracle.build()
    import paper_2408_04466_gb300 as gwn
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    ctx = gwn.Context(0, stream)
    name = args.workload
    out = {"workload": name, "unit": UNIT, "higher_is_better": True, "data": "synthetic", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup}
    if name in ("circle_chain_fp64", "star_chains"):
        ch = gen.bezier_circle_chain() if name == "circle_chain_fp64" else gen.star_chains()
        geo = gwn.Bezier2D(ctx, ch.ctrl, ch.offsets)
        grids = [gwn.Grid(g.lo, g.hi, g.dims) for g in ch.grids]
        nq = sum(g.n for g in grids)
        if name == "circle_chain_fp64":
            # latency-bound (16,384 queries): the graph-replayed launch, with the
            # plain gwn_eval call timed beside it
            w = torch.empty(nq, dtype=torch.float64, device=dev)
            bq = geo.batch_queries(grids)
            fn = lambda: geo.eval_batch(bq, out=w)
            out["gwn_eval_ms"] = statistics.median(_timed(lambda: geo.eval(grids[0]), args.steps, args.warmup,
                                                          stream))
            out["dtype"] = "f64"
        else:
            w = torch.empty(nq, dtype=torch.float32, device=dev)
            bq = geo.batch_queries(grids)          # marshalled once, as a serving loop would
            fn = lambda: geo.eval_batch(bq, out=w)
            out["dtype"] = "f32"
        ms = _timed(fn, args.steps, args.warmup, stream)
        out["ms_per_step"] = statistics.median(ms)
        out["value"] = nq / (out["ms_per_step"] * 1e-3)
        out["queries_per_step"] = nq
        if name == "star_chains":
            out["plan"] = dict(zip(("threads", "rows_per_item"), geo.batch_plan()))
            _, _, bst = geo.eval_batch(bq, out=w, stats=True)
            out["graph_launch_ms"] = bst["ms_total"]        # events around the graph launch alone
            out["autotuned_ms"] = bst["ms_prepare"]         # best candidate during autotuning
            out["roots"] = bst["n_tri_tests"]               # row crossings found, all chains
            out["newton_iters_per_root"] = bst["n_root_iters"] / max(1, bst["n_tri_tests"])
        # brute-force comparator (per-segment quadrature) on one chain's grid
        c0 = int(np.argmax(np.diff(ch.offsets))) if name == "star_chains" else 0
        ctrl0 = ch.ctrl[ch.offsets[c0]:ch.offsets[c0 + 1]]
        g0 = ch.grids[c0]
        one = gwn.Bezier2D(ctx, ctrl0, [0, len(ctrl0)])
        gq = gwn.Grid(g0.lo, g0.hi, g0.dims)
        bms = _timed(lambda: one.bruteforce(gq), 3, 1, stream)
        out["bruteforce_gpu"] = {"value": gq.n / (statistics.median(bms) * 1e-3), "unit": UNIT,
                                 "sample": f"chain {c0} ({(len(ctrl0) - 1) // 3} segments) on its {g0.dims} grid"}
        P = gen.grid_points(g0, np.float64)[:4096]
        t0 = time.perf_counter()
        oracle.w2d_closed_x(ctrl0.astype(np.float64), P)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": len(P) / dt, "unit": UNIT, "cores": oracle.default_threads(), "kind": "oracle",
                               "sample": f"{len(P)} queries of chain {c0}, FP64 closed form (+x ray per query)"}
    elif name == "slit_torus":
        m = gen.slit_torus(n_queries=args.queries)
        mesh = gwn.Mesh(ctx, m.V, m.F)
        mesh.prepare(m.d)
        Pt = torch.as_tensor(m.points).to(dev)
        gw = torch.ones(len(Pt), device=dev)
        w = torch.empty(len(Pt), dtype=torch.float32, device=dev)
        # the crossing index settles before anything is timed: the 2D bins are
        # built once the evaluations of this (mesh, d) reach 4 queries per
        # triangle (8 calls of 1M queries here); until then the tree serves
        for _ in range(-(-4 * len(m.F) // len(Pt)) + 1):
            mesh.eval(gwn.Points(Pt), m.d, out=w)
        torch.cuda.synchronize()

        def step():
            mesh.eval(gwn.Points(Pt), m.d, out=w)
            mesh.backward(Pt, gw)
        ms = _timed(step, args.steps, args.warmup, stream)
        fms = _timed(lambda: mesh.eval(gwn.Points(Pt), m.d, out=w), args.steps, args.warmup, stream)
        info = mesh.info()
        st = mesh.eval(gwn.Points(Pt), m.d, stats=True, out=w)["stats"]
        out.update({"metric": "queries/s, forward + backward (dw/dp, dw/dV)", "dtype": "f32",
                    "ms_per_step": statistics.median(ms), "forward_ms": statistics.median(fms),
                    "value": len(Pt) / (statistics.median(ms) * 1e-3), "queries_per_step": len(Pt),
                    "boundary_edges": info["n_boundary_edges"], "triangles": int(len(m.F)),
                    "kernels": {"traverse_ms": st["ms_traverse"], "bterm3d_ms": st["ms_boundary"]},
                    "roofline_bterm": _alu_roofline(len(Pt), info, st["ms_boundary"])})
        bwd = statistics.median(ms) - statistics.median(fms)
        peaks, kind = _peaks()
        peak = SM_COUNT * FP32_LANES_PER_SM * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
        ach = len(Pt) * info["n_boundary_edges"] * W_GRAD_PAIR / (bwd * 1e-3) / 1e12
        out["backward_ms"] = bwd
        out["roofline_backward"] = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Tops/s (FP32 lane ops)",
                                    "frac": ach / peak, "peak_source": kind,
                                    "note": "step minus forward; W_GRAD_PAIR lane-ops per (query, edge) pair"}
    elif name == "patch_spheroid":
        # parametric surface: 320 bicubic Bezier patches (8 x 8 per cube face,
        # one face left open: one boundary loop of 32 curves x 64 segments),
        # 256^3 grid on [-1.3, 1.3]^3, seeded random d
        pc = gen.patch_spheroid(n=8, amp=0.08, open_faces=(4,), grid_n=args.grid or 256, seed=0)
        ps = gwn.Patches(ctx, pc.ctrl, segments=64)
        g = gwn.Grid(pc.grid.lo, pc.grid.hi, pc.grid.dims)
        w = torch.empty(g.n, dtype=torch.float32, device=dev)
        st = ps.eval(g, pc.d, stats=True, out=w)["stats"]
        ms = _timed(lambda: ps.eval(g, pc.d, out=w), args.steps, args.warmup, stream)
        st = ps.eval(g, pc.d, stats=True, out=w)["stats"]
        info = ps.info()
        Pq = gen.grid_points(pc.grid)[::max(1, g.n // 64)][:64]
        t0 = time.perf_counter()
        oracle.w3d_patches_quad(pc.ctrl, Pq)
        dto = time.perf_counter() - t0
        out.update({"metric": "GWN queries/s, bicubic patch surface (crossings by projection degree)", "dtype": "f32",
                    "ms_per_step": statistics.median(ms), "value": g.n / (statistics.median(ms) * 1e-3),
                    "queries_per_step": g.n, "patches": int(len(pc.ctrl)),
                    "boundary_edges": info["n_boundary_edges"], "boundary_loops": info["n_loops"],
                    "kernels": {"chi_patches_ms": st["ms_traverse"], "bterm3d_ms": st["ms_boundary"],
                                "patch_tests_per_query": st["n_tri_tests"] / g.n,
                                "near_surface_queries": st["n_stack_overflow"]},
                    "roofline_bterm": _alu_roofline(g.n, info, st["ms_boundary"]),
                    "cpu_baseline": {"value": len(Pq) / dto, "unit": UNIT, "cores": oracle.default_threads(),
                                     "kind": "oracle", "sample": f"{len(Pq)} grid queries, FP64 adaptive quadrature "
                                                                 "of the patch definition"}})
    elif name == "chain_points":
        # 2D point queries (one +x ray per point, no ray reuse): the largest
        # star chain (float32, 4,194,304 uniform points in its grid's box) and
        # the circle chain (float64, 1,048,576 points)
        res = {}
        cs = gen.star_chains()
        c = int(np.argmax(np.diff(cs.offsets)))
        cases = [("star_chain_f32", cs.ctrl[cs.offsets[c]:cs.offsets[c + 1]], cs.grids[c], 1 << 22, np.float32),
                 ("circle_chain_f64", gen.bezier_circle_chain().ctrl, gen.bezier_circle_chain().grids[0], 1 << 20,
                  np.float64)]
        for label, ctrl, g, npts, dt in cases:
            geo = gwn.Bezier2D(ctx, np.ascontiguousarray(ctrl, dt), [0, len(ctrl)])
            rng = np.random.default_rng(5)
            P = np.stack([rng.uniform(g.lo[0], g.hi[0], npts), rng.uniform(g.lo[1], g.hi[1], npts)], 1).astype(dt)
            Pt = gwn.Points(torch.as_tensor(P).to(dev))
            ms = _timed(lambda: geo.eval(Pt), args.steps, args.warmup, stream)
            sub = P[:4096].astype(np.float64)
            t0 = time.perf_counter()
            oracle.w2d_closed_x(np.asarray(ctrl, np.float64), sub)
            dto = time.perf_counter() - t0
            res[label] = {"segments": (len(ctrl) - 1) // 3, "points": npts, "ms": statistics.median(ms),
                          "queries_per_s": npts / (statistics.median(ms) * 1e-3),
                          "cpu_baseline_queries_per_s": len(sub) / dto}
        out.update({"metric": "2D point queries/s (one +x ray per point)", "dtype": "f32/f64", "cases": res,
                    "value": res["star_chain_f32"]["queries_per_s"],
                    "ms_per_step": res["star_chain_f32"]["ms"]})
    elif name == "icosphere_cap_axis":
        # the benchmark mesh and grid with d = +z: one ray per grid line
        m, (lo, hi, dims) = workload("icosphere_cap", 0, 1, args.grid)
        mesh = gwn.Mesh(ctx, m.V, m.F)
        g = gwn.Grid(lo, hi, dims)
        w = torch.empty(g.n, dtype=torch.float32, device=dev)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        out_k = {}
        for label, d in (("axis_z", np.array([0, 0, 1], np.float32)), ("random", m.d)):
            mesh.prepare(d)
            times = []
            for it in range(args.warmup + args.steps):
                flush.fill_(1.0)                               # L2 flushed before every step
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                mesh.eval(g, d, out=w)
                e1.record(stream)
                torch.cuda.synchronize()
                if it >= args.warmup:
                    times.append(e0.elapsed_time(e1))
            ks = [mesh.eval(g, d, stats=True, out=w)["stats"] for _ in range(5)]   # after warm-up
            out_k[label] = {"ms_per_step": statistics.median(times),
                            "traverse_ms": statistics.median(k["ms_traverse"] for k in ks),
                            "bterm3d_ms": statistics.median(k["ms_boundary"] for k in ks),
                            "n_tri_tests_per_query": ks[0]["n_tri_tests"] / g.n}
        out.update({"metric": METRIC, "dtype": "f32", "queries_per_step": g.n,
                    "ms_per_step": out_k["axis_z"]["ms_per_step"],
                    "value": g.n / (out_k["axis_z"]["ms_per_step"] * 1e-3),
                    "directions": out_k,
                    "note": "d = +z reuses one ray per grid line; the random-d run of the same mesh and grid is "
                            "beside it"})
    elif name == "mesh_batch":
        # nine meshes of 1,148 to 1,035,360 triangles (icosphere caps, slit tori,
        # holey heightfields), each with its own grid or point list, in one
        # persistent launch replayed from a CUDA graph; the same meshes and
        # queries as nine gwn_eval calls beside it
        d = gen.random_direction(31)
        specs = []
        for sd in (3, 4, 5, 6):
            m = gen.icosphere_cap(subdiv=sd, seed=sd)
            specs.append((m.V, m.F, gwn.Grid((-1.2, -1.15, -1.25), (1.2, 1.3, 1.1), (24 + 8 * sd, 20 + 8 * sd, 28))))
        for nu, nv, nq in ((96, 64, 20000), (512, 512, 300000), (720, 720, 1 << 20)):
            m = gen.slit_torus(n_u=nu, n_v=nv, n_queries=nq, seed=nu)
            specs.append((m.V, m.F, gwn.Points(torch.as_tensor(m.points).to(dev))))
        for nn, holes in ((128, 6), (256, 10)):
            m = gen.holey_heightfield(n=nn, n_holes=holes, grid_n=40, seed=nn)
            specs.append((m.V, m.F, gwn.Grid(m.grid.lo, m.grid.hi, (48, 40, 36))))
        meshes = [gwn.Mesh(ctx, V, F) for V, F, _ in specs]
        for mh in meshes:
            mh.prepare(d)
        qs = [q for _, _, q in specs]
        outs = [torch.empty(q.n, dtype=torch.float32, device=dev) for q in qs]
        nq = sum(q.n for q in qs)
        gwn.eval_meshes(ctx, meshes, qs, d, outs=outs)              # plan, autotune, capture
        ms = _timed(lambda: gwn.eval_meshes(ctx, meshes, qs, d, outs=outs), args.steps, args.warmup, stream)

        def seq():
            for mh, q, o in zip(meshes, qs, outs):
                mh.eval(q, d, out=o)
        sms = _timed(seq, args.steps, args.warmup, stream)
        out.update({"metric": "GWN queries/s, many meshes of uneven sizes in one persistent launch (CUDA graph)",
                    "dtype": "f32", "ms_per_step": statistics.median(ms), "queries_per_step": nq,
                    "value": nq / (statistics.median(ms) * 1e-3), "meshes": len(meshes),
                    "triangles": [int(len(F)) for _, F, _ in specs], "plan": dict(zip(("tiles_per_item",
                                                                                         "blocks_per_sm"),
                                                                                        gwn.meshes_plan(ctx))),
                    "sequential_gwn_eval_ms": statistics.median(sms),
                    "speedup_vs_sequential": statistics.median(sms) / statistics.median(ms)})
    else:
        raise SystemExit(f"unknown workload {name}")
    if _TIMED_CLOCKS:      # SM clocks sampled (every 100 ms) during the first timed region
        out["clocks"] = _TIMED_CLOCKS[0]
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0, help="timed steps (0: 10 for the heightfield, 100 for the "
                                                          "icosphere, 20 for the other workloads)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=0, help="oracle queries of the CPU baseline (0: the "
                                                                "workload's default)")
    ap.add_argument("--ref-sample", type=int, default=0, help="oracle queries per reference-arm step (0: the "
                                                                "workload's default)")
    ap.add_argument("--grid", type=int, default=0, help="grid resolution per axis (0: the workload's own, 512 for "
                                                          "the heightfield, 256 for the icosphere; smaller values "
                                                          "only for profiling captures)")
    ap.add_argument("--queries", type=int, default=1 << 20, help="slit_torus point queries (1,048,576 = the "
                                                                   "measured configuration; fewer only for profiling)")
    ap.add_argument("--no-extras", action="store_true", help="skip comparator, e2e and CPU baseline legs")
    ap.add_argument("--workload", default="holey_heightfield",
                    choices=["holey_heightfield", "icosphere_cap", "circle_chain_fp64", "star_chains", "slit_torus",
                             "icosphere_cap_axis", "chain_points", "patch_spheroid", "mesh_batch"],
                    help="holey_heightfield (default, the largest single-GPU configuration) and icosphere_cap are "
                         "the main measurement; the others print their own measurement line")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.steps <= 0:
        args.steps = MAIN[args.workload]["steps"] if args.workload in MAIN else 20
    if args.impl == "reference":
        if args.workload not in MAIN:
            raise SystemExit("--impl reference measures the main workloads only")
        return run_reference(args)
    if args.workload not in MAIN:
        return run_other(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
