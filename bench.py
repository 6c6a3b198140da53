#!/usr/bin/env python3
"""Throughput of the TTIE hot path on one GB300 (or N independent replicas).

A step is one full inexact-Newton iteration of the library on the workload's
initial state: LBVH candidates, certified narrow phase, energy / gradient /
PSD Hessian of every intersecting pair, block-CSR assembly, PCG, and the
line search with its swept-box candidates.  ``value`` is candidate pairs
through that step per second (whole job), inputs resident in HBM.  ``e2e`` is
the same metric through the public API with the positions copied host->device
before and device->host after every step.

The default workload is the largest single-GPU configuration: the 2,097,152-
triangle noisy sphere.  The other configurations (two icospheres in FP64 with
brute-force pairs, the crossing cloth, the interlocked tori with the Adam loop,
the batch of 512 ellipsoid pairs) are reported under ``configs`` in the same
line, each with its time per step, rooflines and the outcome of the solve to
intersection-free in the FP32 form and the plain FP64 form.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the CPU oracle (the program the CUDA path is
checked against) on a bounded sample of the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TTIE pair evals/s (E+grad+PSD Hess+assembly); seconds to intersection-free"
UNIT = "pair evals/s"
L2_FLUSH_BYTES = 256 << 20   # larger than the 129 MB L2
# dram__bytes_read.sum + dram__bytes_write.sum per launch of the dominant kernel, from one ncu
# capture of the kernels as they are now (None until one is taken)
NCU_TRAFFIC = {
    # k_pcg_resident<float, Chebyshev, 1024 threads>, first Newton step of the noisy sphere,
    # one launch (68 iterations, 204 products): dram__bytes_read.sum + dram__bytes_write.sum
    ("noisy_sphere", "pcg"): 35991111000,
}

# Algorithmic bytes (the minimum an implementation moves, FP32):
B_CANDIDATE = 104.0      # pair ids 8 + 2 x (indices 12 + coordinates 36)
B_ACTIVE_EVAL = 228.0    # T 4 + gradient 72 + t_c and their gradients 152
B_ASM_PAIR = 36 * 36 * 2 + 36 * 8   # 36 block values written and read, 36 keys
B_ASM_BLOCK = 36.0       # assembled 3x3 block
B_PCG_BLOCK = 40.0       # per product: 3x3 block 36 + column index 4
B_PCG_ROW = 72.0         # per product: 3 floats x 6 vectors per row


def workload(name):
    """(mesh, precision, description, pair mode: 0 self, 1 inter-group, 2 intra-group; brute)."""
    import ttie_inputs as ti
    if name == "noisy_sphere":
        return ti.noisy_sphere(9, seed=5).as_f32(), 0, (
            "octahedral sphere level 9 (2,097,152 triangles, radius 1) displaced by 0.15*(N1,N2,N3), three "
            "seeded 5-octave value-noise fields of base frequency 8 (folds through itself); self pairs, "
            "LBVH; float32"), 0, False
    if name == "noisy_sphere_literal":
        return ti.noisy_sphere(9, seed=5, vector=False).as_f32(), 0, (
            "octahedral sphere level 9 displaced radially by 0.15*N (intersection-free by construction); "
            "float32"), 0, False
    if name == "cloth256":
        return ti.cloth(256, seed=2).as_f32(), 0, (
            "cloth 256x256 vertices (130,050 triangles) on [0,1]^2, z = 8 seeded sinusoids "
            "(A~U[0.05,0.3], k~U[2,12]), x += 0.4*g(x,y) with g an independent 8-sinusoid field "
            "(folds that cross themselves); self pairs, LBVH; float32"), 0, False
    if name == "cloth256_literal":
        return ti.cloth(256, seed=2, crossing=False).as_f32(), 0, (
            "cloth 256x256 (130,050 triangles), x += 0.4*z shear (intersection-free by construction)"), 0, False
    if name == "ellipsoids512":
        m, _, _ = ti.ellipsoid_batch(512, seed=4)
        return m.as_f32(), 0, (
            "512 independent pairs of lat-long ellipsoids, triangles per mesh log-uniform in [100, 20000], "
            "semi-axes U[0.5,1.5], random relative rotation, centre offset U[0.3,1] x (sum of mean semi-axes); "
            "pairs within an instance, each instance solved on its own; float32"), 2, False
    if name == "icospheres":
        return ti.two_icospheres(), 1, (
            "two unit icospheres (2 subdivisions, 320 triangles each), the second rotated at random and "
            "centred at (1.2, 0, 0); all 102,400 inter-mesh pairs by brute force; float64"), 1, True
    if name == "tori":
        return ti.interlocked_tori(offset=(0.5, 0, 0)).as_f32(), 0, (
            "two tori R=1, r=0.3, 256x128 segments (65,536 triangles each), the second rotated 90 deg "
            "about x and offset by (0.5, 0, 0) so the tubes interpenetrate, Gaussian jitter 0.005; self "
            "pairs, LBVH; float32"), 0, False
    raise SystemExit("unknown workload %s" % name)


def oracle_sample(m, n_side, mode=0, part=0, parts=1):
    """The workload restricted to n_side x n_side grid vertices (cloth), to whole instances up to
    about 2 n_side^2 triangles (batched instances), or to the 2 n_side^2 triangles whose
    centroids lie nearest one triangle's (a connected patch, others): what the oracle can
    process in seconds.  part of parts: one of parts disjoint-start samples spread over the
    workload (part 0: the grid's corner, the first instances, the first triangle)."""
    import numpy as np
    import ttie_inputs as ti
    if m.V == 256 * 256:
        ij = np.arange(m.V)
        i0 = (part * (256 - n_side)) // max(parts - 1, 1) if parts > 1 else 0
        keep_v = ((ij % 256) >= i0) & ((ij % 256) < i0 + n_side) & ((ij // 256) < n_side)
        keep_t = keep_v[m.tri].all(axis=1)
    elif mode == 2:
        counts = np.bincount(m.group)
        cum = np.cumsum(counts)
        g0 = int(np.searchsorted(cum, cum[-1] * part // parts, side="right")) if parts > 1 else 0
        upto = max(g0 + 1, int(np.searchsorted(cum, (cum[g0 - 1] if g0 else 0) + 2 * n_side * n_side)))
        keep_t = (m.group >= g0) & (m.group < upto)
    else:
        cen = m.x[m.tri].mean(axis=1)
        a = (part * m.F) // parts
        near = np.argsort(np.linalg.norm(cen - cen[a], axis=1), kind="stable")[: n_side * n_side * 2]
        keep_t = np.zeros(m.F, bool)
        keep_t[near] = True
    tri = m.tri[keep_t]
    used = np.unique(tri)
    remap = -np.ones(m.V, np.int64)
    remap[used] = np.arange(len(used))
    return ti.Mesh(m.x[used], remap[tri].astype(np.int32), m.group[keep_t])


def oracle_step(sub, mode=0):
    """One pass of the oracle over the sample: brute-force candidates, per-pair evaluation
    (duals + exact test), gradient, PSD Hessian and assembly.  Returns candidate pairs."""
    import oracle as O
    pairs = O.candidate_pairs(sub.x, sub.tri, sub.group, ("self", "inter", "instance")[mode])
    ev = O.evaluate(sub.x, sub.tri, pairs)
    O.assemble(sub.tri, ev, sub.V)
    return len(pairs)


class Clocks:
    """nvidia-smi samples (every 50 ms) kept only inside the timed window."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def mark_begin(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        import datetime
        rows = []
        for line in out.strip().splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(f[2]), float(f[3]), f[6:10]))
            except ValueError:
                continue
        inside = [r for r in rows if self.t0 is not None and self.t0 <= r[0] <= self.t1]
        if not inside and rows and self.t0 is not None:   # window shorter than the sampling period
            mid = 0.5 * (self.t0 + self.t1)
            inside = [min(rows, key=lambda r: abs(r[0] - mid))]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in inside for n, v in zip(names, r[3]) if v.lower().startswith("active")})
        sm = sorted(r[1] for r in inside)
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": inside[0][2] if inside else None,
                "reasons": reasons, "samples": len(inside)}


def aggregate(total_ms, pairs, world, device):
    """Whole-job figures over N replica ranks: the slowest rank's time (MAX) and the pairs all
    ranks processed (SUM).  Returns (seconds, pairs)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    p = torch.tensor([float(pairs)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return t.item() / 1e3, p.item()


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def run_reference(args, rank, world):
    """CPU oracle arm: rank 0 only."""
    if rank != 0:
        return
    m, _, desc, mode, _ = workload(args.workload)
    sub = oracle_sample(m, 24, mode)
    for _ in range(args.warmup):
        oracle_step(sub, mode)
    t0 = time.perf_counter()
    n = 0
    for _ in range(args.steps):
        n += oracle_step(sub, mode)
    dt = time.perf_counter() - t0
    v = n / dt
    sample = "oracle on a %d-triangle patch of the workload (%d candidate pairs per step)" % (
        sub.F, n // max(args.steps, 1))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "sample": sample},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def cpu_baseline(m, mode=0, seconds_target=15.0):
    """Oracle throughput on a bounded sample (patch of the workload), single core."""
    sub = oracle_sample(m, 80, mode)
    t0 = time.perf_counter()
    n, reps = 0, 0
    while True:
        n += oracle_step(sub, mode)
        reps += 1
        if time.perf_counter() - t0 > seconds_target or reps >= 4:
            break
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "oracle on a sample of the workload (an 80x80-vertex patch of a grid, whole instances "
                      "up to ~12,800 triangles, or a patch of 12,800 triangles; %d triangles, %d candidate "
                      "pairs) x %d, %.1f s" % (sub.F, n // reps, reps, dt)}


def _oracle_worker(sub, mode, seconds_target):
    """One process of the all-cores baseline: the oracle over its sample until the target time."""
    t0 = time.perf_counter()
    n = 0
    while True:
        n += oracle_step(sub, mode)
        if time.perf_counter() - t0 > seconds_target:
            break
    return n, time.perf_counter() - t0


def cpu_baseline_all_cores(m, mode=0, seconds_target=10.0):
    """The oracle on every host core: one process per core (started by spawn, as the GPU is in
    use), each running the oracle as it stands over its own sample of the workload; throughput
    is all processes' candidate pairs over the wall time."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    subs = [oracle_sample(m, 80, mode, part=i, parts=cores) for i in range(cores)]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.starmap(_oracle_worker, [(sub, mode, seconds_target) for sub in subs])
    wall = time.perf_counter() - t0
    n = sum(r[0] for r in res)
    busy = max(r[1] for r in res)   # the processes run side by side; the longest one's compute time
    return {"value": n / busy, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "oracle, one process per host core, each on its own sample of the workload (an 80x80-vertex "
                      "patch of a grid, whole instances up to ~12,800 triangles, or a patch of 12,800 triangles "
                      "around a different triangle) for about %.0f s; %d candidate pairs over the longest "
                      "process's %.1f s (%.1f s of wall time with process start)" % (seconds_target, n, busy, wall)}


def rooflines(last, ms, peak, hbm):
    """Algorithmic bytes per launch (or stage) over its CUDA-event duration, against the peak.
    ms: per-step milliseconds of the PCG kernel, the classification kernel and the assembly
    and evaluation stages."""
    src = "measured" if hbm else "fallback"

    def line(name, nbytes, t_ms, kind="kernel"):
        ach = nbytes / (t_ms * 1e-3) / 1e9 if t_ms > 0 else None
        return {kind: name, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "peak_source": src,
                "frac": ach / peak if ach else None, "ms": t_ms, "algorithmic_bytes": nbytes}
    pcg = line("k_pcg_resident", B_PCG_BLOCK * last["pcg_block_iters"] + B_PCG_ROW * last["pcg_row_iters"], ms["pcg"])
    cls = line("k_classify", B_CANDIDATE * last["n_candidates"], ms["classify"])
    asm = line("assemble", B_ASM_PAIR * last["n_active"] + B_ASM_BLOCK * last["nnzb"], ms["assemble"], "stage")
    ev = line("eval", B_CANDIDATE * last["n_candidates"] + B_ACTIVE_EVAL * last["n_active"], ms["eval"], "stage")
    return pcg, cls, asm, ev


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="noisy_sphere")
    ap.add_argument("--configs", default="icospheres,cloth256,tori,ellipsoids512",
                    help="further configurations reported under 'configs' ('' for none)")
    ap.add_argument("--no-solve", action="store_true", help="skip the solves to intersection-free")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-form", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-quasi-static", action="store_true", help="skip the quasi-static simulation run")
    ap.add_argument("--no-next-rows", action="store_true",
                    help="skip the timings of the PSD variants, the exact Hessian-vector product and the dual evaluator")
    ap.add_argument("--pcg-precond", choices=["auto", "block_jacobi", "chebyshev"], default="auto",
                    help="preconditioner of the shared-memory PCG")
    ap.add_argument("--pcg-cheb-degree", type=int, default=0, help="Chebyshev degree (0: the library's default)")
    ap.add_argument("--traversal", choices=["one_walk", "two_walks"], default="one_walk",
                    help="LBVH traversal")
    ap.add_argument("--pcg-kernel", choices=["auto", "resident", "streamed", "resident_uncached"], default="auto",
                    help="PCG kernel: block-resident (one launch; uncached: matrix rows from global memory on "
                         "every product) or streamed (two kernels per iteration)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch
    import torch.distributed as dist
    import ttie_inputs as ti
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_06511_gb300 import ttie

    solver = {"pcg_precond": {"auto": ttie.PCG_AUTO, "block_jacobi": ttie.PCG_BLOCK_JACOBI,
                              "chebyshev": ttie.PCG_CHEBYSHEV}[args.pcg_precond],
              "pcg_cheb_degree": args.pcg_cheb_degree,
              "traversal_mode": {"two_walks": ttie.TRAVERSAL_TWO_WALKS,
                                 "one_walk": ttie.TRAVERSAL_ONE_WALK}[args.traversal],
              "pcg_kernel": {"auto": ttie.PCG_KERNEL_AUTO, "resident": ttie.PCG_KERNEL_RESIDENT,
                             "streamed": ttie.PCG_KERNEL_STREAMED,
                             "resident_uncached": ttie.PCG_KERNEL_RESIDENT_UNCACHED}[args.pcg_kernel]}
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    peak = hbm if hbm else 6800.0

    def on_device(m, precision, mode):
        dt = torch.float32 if precision == 0 else torch.float64
        x0 = torch.tensor(m.x, dtype=dt, device="cuda")
        tri = torch.tensor(m.tri, dtype=torch.int32, device="cuda")
        grp = torch.tensor(m.group, dtype=torch.int32, device="cuda") if mode else None
        return x0, tri, grp

    def time_steps(ctx, x0, steps, warmup):
        """Newton steps from x0 (L2 flushed before each), timed with CUDA events on the stream."""
        x = x0.clone()
        for _ in range(warmup):
            x.copy_(x0)
            ctx.newton_step(x)
        torch.cuda.synchronize()
        tot, pairs, active = 0.0, 0, 0
        stage = {"build": 0.0, "eval": 0.0, "assemble": 0.0, "pcg": 0.0, "line_search": 0.0}
        kern = {"classify": 0.0, "pcg": 0.0}
        last = None
        for _ in range(steps):
            x.copy_(x0)
            flush.zero_()
            ev0.record(stream)
            info = ctx.newton_step(x)
            ev1.record(stream)
            ev1.synchronize()
            tot += ev0.elapsed_time(ev1)
            pairs += info["n_candidates"]
            active += info["n_active"]
            for k in stage:
                stage[k] += info["ms_" + k]
            kern["classify"] += info["ms_classify"]
            kern["pcg"] += info["ms_pcg_kernel"]
            last = info
        ms = {"pcg": kern["pcg"] / steps, "classify": kern["classify"] / steps,
              "assemble": stage["assemble"] / steps, "eval": stage["eval"] / steps}
        return {"total_ms": tot, "pairs": pairs, "active": active, "last": last,
                "stage_ms_per_step": {k: v / steps for k, v in stage.items()}, "kernel_ms": ms}

    def step_launches(info):
        """Kernels the step launched per stage; for batched instances also the PCG schedule."""
        out = {"launches_per_stage": dict(zip(["build", "eval", "assemble", "pcg", "line_search"],
                                              info["stage_launches"]))}
        if info.get("inst_threads"):
            out["pcg_schedule"] = {"threads": info["inst_threads"], "blocks_per_sm": info["inst_blocks_per_sm"],
                                   "order": "largest first" if info["inst_order"] == 0 else "as numbered"}
        return out

    def certify(m, x, mode):
        """The oracle's exact test on an end state (intersecting pairs; 0 = intersection-free),
        with its brute-force candidate list where that fits the bench's time."""
        import oracle as O
        if m.F > 20000:
            return None
        return O.certify(x.double().cpu().numpy(), m.tri, m.group, ("self", "inter", "instance")[mode])

    def c_active_tris(c, x, tri, grp):
        """First triangles of the intersecting pairs of the last evaluation (x given: evaluate at x)."""
        if x is not None:
            c.build_bvh(x, tri, grp)
            c.eval_pairs(x, ttie.EVAL_E)
        ap, _, _ = c.get_active(with_derivatives=False)
        return ap[:, 0].long().cpu().numpy()

    def solve_outcome(m, precision, mode, brute, max_it=100):
        """Seconds to intersection-free (ttie_solve's wall time, after one solve that allocates the
        context's buffers), with the end state certified by the oracle where its brute force fits."""
        x0, tri, grp = on_device(m, precision, mode)
        pm = mode | (ttie.PAIRS_BRUTE if brute else 0)
        c = ttie.Context(precision=precision, pair_mode=pm, newton_max_it=max_it, **solver)
        try:
            c.build_bvh(x0, tri, grp)
            c.newton_step(x0.clone())   # allocations
            xs = x0.clone()
            torch.cuda.synchronize()
            s = c.solve(xs)
            cert = certify(m, xs, mode) if s["converged"] else None
            out = {"dtype": "f32" if precision == 0 else "f64", "converged": bool(s["converged"]),
                   "iterations": s["iterations"], "seconds": s["seconds"],
                   "n_active_initial": s["n_active_initial"], "n_active_final": s["n_active_final"],
                   "energy_initial": s["energy_initial"], "energy_final": s["energy_final"],
                   "newton_max_it": max_it,
                   "oracle_certified_intersecting": cert}
            if mode == 2:   # independent instances: how many end without an intersecting pair
                n_inst = int(m.group.max()) + 1
                open0 = np.unique(m.group[c_active_tris(c, x0, tri, grp)])
                c.build_bvh(xs, tri, grp)
                c.eval_pairs(xs, ttie.EVAL_E)
                open1 = np.unique(m.group[c_active_tris(c, None, None, None)])
                out.update({"instances": n_inst, "instances_intersecting_initial": int(len(open0)),
                            "instances_intersecting_final": int(len(open1))})
            return out
        except ttie.TTIEError as e:   # reported, the line still prints
            return {"dtype": "f32" if precision == 0 else "f64", "error": str(e)[:200]}
        finally:
            c.close()

    # ---------------------------------------------------------------- main workload
    m, precision, desc, mode, brute = workload(args.workload)
    x0, tri, grp = on_device(m, precision, mode)
    ctx = ttie.Context(precision=precision, pair_mode=mode | (ttie.PAIRS_BRUTE if brute else 0), profile=1, **solver)
    ctx.build_bvh(x0, tri, grp)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = Clocks(local)
    clocks.start()
    x = x0.clone()
    for _ in range(args.warmup):
        x.copy_(x0)
        ctx.newton_step(x)
    barrier()
    clocks.mark_begin()
    launches0 = ctx.get_launch_count()
    main_t = time_steps(ctx, x0, args.steps, 0)
    launches = ctx.get_launch_count() - launches0
    barrier()
    clocks.mark_end()
    clk = clocks.stop()
    total_ms = main_t["total_ms"]
    total_s, all_pairs = aggregate(total_ms, main_t["pairs"], world, "cuda")
    value = all_pairs / total_s
    last = main_t["last"]

    # end to end through the public API with host buffers
    xh0 = x0.cpu().pin_memory()
    xh = torch.empty_like(xh0).pin_memory()
    e2e_ms, e2e_pairs = 0.0, 0
    for i in range(args.warmup + max(3, args.steps // 2)):
        flush.zero_()
        ev0.record(stream)
        x.copy_(xh0, non_blocking=True)
        info = ctx.newton_step(x)
        xh.copy_(x, non_blocking=True)
        ev1.record(stream)
        ev1.synchronize()
        if i >= args.warmup:
            e2e_ms += ev0.elapsed_time(ev1)
            e2e_pairs += info["n_candidates"]
    e2e_bytes = x0.numel() * x0.element_size()

    r_pcg, r_cls, r_asm, r_ev = rooflines(last, main_t["kernel_ms"], peak, hbm)
    r_pcg["kernel"] = ("k_pcg_instances" if mode == 2 else
                       "k_cg_spmv + k_cg_update" if last.get("pcg_kernel") == ttie.PCG_KERNEL_STREAMED else
                       "k_pcg_resident")
    r_pcg["traffic"] = NCU_TRAFFIC.get((args.workload, "pcg"))
    r_cls["traffic"] = NCU_TRAFFIC.get((args.workload, "classify"))
    r_pcg["share_of_step"] = r_pcg["ms"] / (total_ms / args.steps)
    roofline = r_pcg

    def fp64_form(mm, mode_, brute_, steps):
        """The plain FP64 form on the same GPU: every stage in double precision (same kernels
        instantiated for FP64), a few steps of the workload."""
        x64_0, tri64, grp64 = on_device(mm, 1, mode_)
        c64 = ttie.Context(precision=ttie.F64, pair_mode=mode_ | (ttie.PAIRS_BRUTE if brute_ else 0), profile=1,
                           **solver)
        c64.build_bvh(x64_0, tri64, grp64)
        t = time_steps(c64, x64_0, steps, args.warmup)
        c64.close()
        return {"value": t["pairs"] / (t["total_ms"] / 1e3), "unit": UNIT, "ms_per_step": t["total_ms"] / steps,
                "steps": steps, "dtype": "f64", "pcg_iters": t["last"]["pcg_iters"],
                "intersecting_per_step": t["last"]["n_active"], "stage_ms_per_step": t["stage_ms_per_step"]}

    fp64 = None
    if precision == 0 and not args.no_fp64_form and rank == 0:
        fp64 = fp64_form(m, mode, brute, max(3, min(args.steps, 10)))
        fp64["speedup_of_fp32_form"] = fp64["ms_per_step"] / (total_ms / args.steps)

    solve = None
    if not args.no_solve and rank == 0:
        solve = {"f32": solve_outcome(m, precision, mode, brute)}
        if precision == 0 and not args.no_fp64_form:
            solve["f64"] = solve_outcome(m, 1, mode, brute)

    # ---------------------------------------------------------------- the other configurations
    configs = {}
    if rank == 0:
        for name in [c for c in args.configs.split(",") if c and c != args.workload]:
            mc, pc, dc, mdc, bc = workload(name)
            entry = {"workload": dc, "triangles": mc.F, "vertices": mc.V}
            try:
                xc0, tc_, gc = on_device(mc, pc, mdc)
                cc = ttie.Context(precision=pc, pair_mode=mdc | (ttie.PAIRS_BRUTE if bc else 0), profile=1, **solver)
                cc.build_bvh(xc0, tc_, gc)
                ks = max(3, min(args.steps, 10))
                t = time_steps(cc, xc0, ks, args.warmup)
                cc.close()
                lc = t["last"]
                rp, rc, ra, re = rooflines(lc, t["kernel_ms"], peak, hbm)
                rp["kernel"] = ("k_pcg_instances" if mdc == 2 else
                                "k_cg_spmv + k_cg_update" if lc.get("pcg_kernel") == ttie.PCG_KERNEL_STREAMED else
                                "k_pcg_resident")
                entry.update({
                    "dtype": "f32" if pc == 0 else "f64", "steps": ks, "ms_per_step": t["total_ms"] / ks,
                    "value": t["pairs"] / (t["total_ms"] / 1e3), "unit": UNIT,
                    "active_pairs_per_s": t["active"] / (t["total_ms"] / 1e3),
                    "candidates_per_step": lc["n_candidates"], "intersecting_per_step": lc["n_active"],
                    "pcg_iters": lc["pcg_iters"], "bsr_rows": lc["n_rows"], "bsr_blocks": lc["nnzb"],
                    "stage_ms_per_step": t["stage_ms_per_step"],
                    "roofline_pcg": rp, "roofline_pair_eval": rc, "roofline_assembly": ra, "roofline_eval": re})
                entry.update(step_launches(lc))
                if pc == 0 and not args.no_fp64_form:
                    f = fp64_form(mc, mdc, bc, ks)
                    f["speedup_of_fp32_form"] = f["ms_per_step"] / entry["ms_per_step"]
                    entry["fp64_form"] = f
                if not args.no_solve:
                    entry["solve"] = {"f32" if pc == 0 else "f64": solve_outcome(mc, pc, mdc, bc)}
                    if pc == 0 and not args.no_fp64_form:
                        entry["solve"]["f64"] = solve_outcome(mc, 1, mdc, bc)
            except Exception as e:   # a failure here is reported, the line still prints
                entry["error"] = "%s: %s" % (type(e).__name__, str(e)[:200])
            configs[name] = entry

    # the tori configuration's use of the energy as a loss: Adam on sum T + lambda/2 |x - x0|^2
    # through the autograd Function (forward: the library's energy; backward: its gradient)
    if rank == 0 and "tori" in configs and "error" not in configs["tori"]:
        from paper_2606_06511_gb300.autograd import TTIEnergy
        mt, _, _, _, _ = workload("tori")
        xt0 = torch.tensor(mt.x, dtype=torch.float32, device="cuda")
        f = TTIEnergy(torch.tensor(mt.tri, dtype=torch.int32, device="cuda"), None, precision=ttie.F32, **solver)
        xa = xt0.clone().requires_grad_(True)
        opt = torch.optim.Adam([xa], lr=1e-3)
        lam, n_adam = 1.0, 200
        hist = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_adam):
            opt.zero_grad()
            E = f(xa)
            loss = E + 0.5 * lam * ((xa - xt0) ** 2).sum()
            loss.backward()
            opt.step()
            hist.append((E.item(), f.last))
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        E_end = f(xa.detach()).item()
        configs["tori"]["adam"] = {
            "loss": "sum T + lambda/2 |x - x0|^2, lambda 1, Adam lr 1e-3, through the autograd Function",
            "steps": n_adam, "seconds": sec, "ms_per_step": 1e3 * sec / n_adam,
            "energy_initial": hist[0][0], "n_active_initial": hist[0][1],
            "energy_final": E_end, "n_active_final": f.last,
            "energy_min": min(h[0] for h in hist)}
        f.ctx.close()

    # seconds to intersection-free where the method reaches it on small scenes: a shallow
    # overlap of two spheres and a mildly folded cloth (substitute workloads, not configs)
    reach = None
    if not args.no_solve and rank == 0:
        reach = []
        for name, mr, pm, d in (
                ("spheres_shallow", ti.two_icospheres(offset=(1.95, 0.0, 0.0)), 1,
                 "two unit icospheres (640 triangles), overlap 0.05, inter-mesh pairs"),
                ("cloth_mild", ti.cloth(16, seed=2, shear=0.05), 0,
                 "16x16-vertex cloth, the crossing fold field scaled to 0.05; self pairs")):
            row = {"workload": name, "description": d, "triangles": mr.F}
            for prec in (0, 1):   # the same float32-representable start for both forms
                row["f32" if prec == 0 else "f64"] = solve_outcome(mr.as_f32(), prec, pm, False, max_it=60)
            reach.append(row)

    # the quasi-static simulation (Fig. 2): from an intersecting state to a valid one with a
    # mass-spring term on every edge (rest = initial lengths); seconds to valid, median of 5
    qs = None
    if rank == 0 and not args.no_quasi_static:
        mq = ti.two_icospheres(offset=(1.95, 0.0, 0.0)).as_f32()
        eq = ti.edge_list(mq.tri)
        rest = np.linalg.norm(mq.x[eq[:, 0]] - mq.x[eq[:, 1]], axis=1)
        xq0 = torch.tensor(mq.x, dtype=torch.float32, device="cuda")
        tq = torch.tensor(mq.tri, dtype=torch.int32, device="cuda")
        gq = torch.tensor(mq.group, dtype=torch.int32, device="cuda")
        cq = ttie.Context(pair_mode=1, newton_max_it=40)
        cq.build_bvh(xq0, tq, gq)
        cq.set_elastic(torch.tensor(eq, device="cuda"), torch.tensor(rest, dtype=torch.float32, device="cuda"), 0.1)
        runs = []
        for _ in range(6):
            xq = xq0.clone()
            torch.cuda.synchronize()
            r = cq.solve(xq)
            runs.append((r["seconds"], r, xq))
        runs = runs[1:]   # the first run allocates the context's buffers
        runs.sort(key=lambda t: t[0])
        sec, r, xq = runs[len(runs) // 2]
        xf = xq.double().cpu().numpy()
        strain = float(np.abs(np.linalg.norm(xf[eq[:, 0]] - xf[eq[:, 1]], axis=1) / rest - 1).max())
        qs = {"workload": "two unit icospheres (2 subdivisions, 640 triangles), the second rotated at random "
                          "and offset by 1.95 (overlap 0.05); springs on all %d edges at rest, k = 0.1; "
                          "inter-mesh pairs; float32" % len(eq),
              "seconds_to_valid": sec, "iterations": r["iterations"], "converged": bool(r["converged"]),
              "n_active_initial": r["n_active_initial"], "n_active_final": r["n_active_final"],
              "max_edge_strain": strain, "runs": 5}
        cq.close()

    # the rows beyond the step: a Newton step under each PSD projection of §1.1, the exact
    # Hessian-vector product and the FP64 dual-number gradient pass, on this workload at x0
    nxt = None
    if rank == 0 and not args.no_next_rows and mode != 2:
        def med(fn, k=5):
            ts = []
            for _ in range(k):
                flush.zero_()
                ev0.record(stream)
                r = fn()
                ev1.record(stream)
                ev1.synchronize()
                ts.append(ev0.elapsed_time(ev1))
            return sorted(ts)[k // 2], r
        nxt = {"psd_modes": {}}
        for name, pm in (("per_part", ttie.PSD_PER_PART), ("drop_cross", ttie.PSD_DROP_CROSS),
                         ("whole", ttie.PSD_WHOLE)):
            cp = ttie.Context(precision=precision, pair_mode=mode, psd_mode=pm)
            cp.build_bvh(x0, tri, grp)
            xs = x0.clone()
            cp.newton_step(xs)   # warm-up (allocations)

            def one():
                xs.copy_(x0)
                return cp.newton_step(xs)
            ms, inf = med(one)
            nxt["psd_modes"][name] = {"ms_per_step": ms, "pcg_iters": inf["pcg_iters"],
                                      "energy_ratio": inf["energy_new"] / inf["energy"] if inf["energy"] else None,
                                      "alpha": inf["alpha"]}
            cp.close()
        # the PCG to its tolerance: one step with each preconditioner, iterations and the
        # relative residual reached (block Jacobi may stop at its iteration cap first)
        nxt["pcg_preconditioners"] = {}
        for name, pc in (("block_jacobi", ttie.PCG_BLOCK_JACOBI), ("chebyshev", ttie.PCG_CHEBYSHEV)):
            cp = ttie.Context(precision=precision, pair_mode=mode, pcg_precond=pc, profile=1)
            cp.build_bvh(x0, tri, grp)
            xs = x0.clone()
            cp.newton_step(xs)

            def one():
                xs.copy_(x0)
                return cp.newton_step(xs)
            ms, inf = med(one)
            nxt["pcg_preconditioners"][name] = {
                "ms_per_step": ms, "pcg_ms": inf["ms_pcg"], "pcg_iters": inf["pcg_iters"],
                "pcg_rel_residual": inf["pcg_rel_residual"], "rtol": cp.params.pcg_rtol,
                "max_it": cp.params.pcg_max_it,
                "energy_ratio": inf["energy_new"] / inf["energy"] if inf["energy"] else None}
            cp.close()
        cx = ttie.Context(precision=precision, pair_mode=mode)
        cx.build_bvh(x0, tri, grp)
        _, n_act0 = cx.eval_pairs(x0, ttie.EVAL_E | ttie.EVAL_H)
        vv = torch.randn_like(x0)
        ms_hx, _ = med(lambda: cx.hvp(x0, vv, exact=True))
        ms_hp, _ = med(lambda: cx.hvp(x0, vv, exact=False))
        cx.eval_pairs(x0, ttie.EVAL_E | ttie.EVAL_H)
        ms_du, _ = med(lambda: cx.dual_gradients(x0))
        nxt["hvp_exact_ms"] = ms_hx
        nxt["hvp_psd_ms"] = ms_hp
        nxt["dual_gradients"] = {"ms": ms_du, "pairs": n_act0, "pairs_per_s": n_act0 / (ms_du / 1e3)}
        cx.close()

    cpu = cpu_all = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(m, mode)
        cpu_all = cpu_baseline_all_cores(m, mode)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if precision == 0 else "f64",
            "data": "synthetic",
            "config": {"workload": desc, "triangles": m.F, "vertices": m.V,
                       "candidates_per_step": last["n_candidates"], "intersecting_per_step": last["n_active"],
                       "swept_candidates_per_step": last["n_candidates_swept"],
                       "line_search_trials": last["ls_trials"], "pcg_iters": last["pcg_iters"],
                       "bsr_rows": last["n_rows"], "bsr_blocks": last["nnzb"],
                       "l2": "flushed (256 MiB write) before every timed step",
                       "pcg_precond": args.pcg_precond, "pcg_kernel": args.pcg_kernel, "traversal": args.traversal,
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "stage_ms_per_step": main_t["stage_ms_per_step"],
            **step_launches(last),
            "active_pairs_per_s": main_t["active"] / (total_ms / 1e3),
            "roofline": roofline,
            "roofline_pair_eval": r_cls,
            "roofline_assembly": r_asm,
            "roofline_eval": r_ev,
            "cpu_baseline": cpu,
            "cpu_baseline_all_cores": cpu_all,
            "fp64_form": fp64,
            "e2e": {"value": e2e_pairs / (e2e_ms / 1e3) if e2e_ms > 0 else None, "unit": UNIT,
                    "h2d_bytes_per_step": e2e_bytes, "d2h_bytes_per_step": e2e_bytes},
            "gpu_launches": launches,
            "gpu_launches_per_step": launches / args.steps,
            "clocks": clk,
            "time_to_intersection_free": solve,
            "configs": configs,
            "time_to_intersection_free_substitutes": reach,
            "quasi_static": qs,
            "next_rows": nxt,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
