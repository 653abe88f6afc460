#!/usr/bin/env python
"""PM particle-steps/s and fraction of the HBM roofline at 512^3 on GB300 (FP32 vs FP64 plain).

Workload: 512^3 particles on a 512^3 CIC mesh, L = 5000 Mpc/h, Newtonian PM from
Zel'dovich ICs at z = 50 (Lambda-CDM, Eisenstein-Hu no-wiggle P(k), sigma_8 = 0.81),
kick-drift-kick steps on a uniform a-grid to z = 0.  A step is one force evaluation
plus update: CIC deposit, r2c FFT, Green's function and spectral gradient, c2r FFT,
CIC interpolation + kick + drift.  Inputs (3.2 GB of particles, 0.5 GB per mesh) are
larger than L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  Under torchrun every rank runs an independent
realisation (replicas, no collective on the data path); value sums over ranks and
time is the maximum over ranks.

--impl reference times the FP64 CPU oracle (oracle/) on this host's cores on a
bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PM particle-steps/s and fraction of HBM roofline at 512^3, FP32 vs FP64 plain"
UNIT = "particle-steps/s"
A_INIT, A_FINAL = 1.0 / 51.0, 1.0
GRID_STEPS = 100  # the headline run: 100 KDK steps from z = 50 to z = 0, whatever --steps asks to time
PHASES = ("deposit", "fft_zy_fwd", "fft_x_green", "fft_yz_inv", "kick_drift")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def fused_update(np_side, n, fp64):
    """The FP32 lattice path deposits the next density inside the kick-drift pass."""
    r = n // np_side
    return (not fp64) and n >= 64 and r in (1, 2, 4) and np_side >= 32 // r


def fused_middle(n, fp64):
    """FP32 meshes of 256^3 and up run the forward y, x and inverse y passes as one persistent
    kernel over the kz planes (pm_set_fused_fft)."""
    return (not fp64) and n >= 256


def launches_per_step(np_side, n, fp64, fused_fft=True):
    """Kernels of this library launched per step (one force evaluation + one update): z r2c,
    the middle passes (one fused kernel, or y, x with the Green's function and y with the y
    gradient), z c2r of the three force components, and the update (+ the deposit when it is
    not fused into the update)."""
    fft = 3 if (fused_fft and fused_middle(n, fp64)) else 5
    return fft + (1 if fused_update(np_side, n, fp64) else 2)


def kernel_bytes(np_side, n, fp64, fused_fft=True):
    """Algorithmic bytes per launch of each phase (each array it must touch, once)."""
    s = 8 if fp64 else 4
    P = np_side**3
    R = n**3 * s
    S = (n // 2 + 1) * n * n * 2 * s
    kb = {
        "deposit": 3 * s * P + R,            # read x, write rho
        "fft_zy_fwd": R + S,                 # read rho, write the y-transformed half spectrum
        "fft_x_green": 3 * S,                # read delta_k, write IFFT_x(phi), IFFT_x(-i kx phi)
        "fft_yz_inv": 2 * S + 3 * R,         # read the two x-inverted spectra, write 3 force meshes
        "kick_drift": 12 * s * P + 3 * R,    # read + write x, p; gather 3 meshes once
    }
    if fused_fft and fused_middle(n, fp64):
        kb["fft_zy_fwd"] = R + S             # z r2c only: read rho, write its half spectrum
        kb["fft_x_green"] = 4 * S            # read the z pass's spectrum, write the three y-inverted ones
        kb["fft_yz_inv"] = 3 * S + 3 * R     # the three z c2r
    if fused_update(np_side, n, fp64):
        kb["deposit"] = 0                    # no launch: the inverse z pass clears rho ...
        kb["fft_yz_inv"] += R                # ... beside the force rows it writes
        kb["kick_drift"] += R                # the drifted positions are deposited in the same pass
    return kb


def step_bytes(np_side, n, fp64):
    """Algorithmic bytes of one whole PM step: 60 B/particle + 40 B/cell (x2 in FP64)."""
    f = 2 if fp64 else 1
    return f * (60 * np_side**3 + 40 * n**3)


def csrc_sha(names=None):
    """Digest of the named files of the CUDA sources (all of them by default)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2404_02783_gb300", "csrc")
    for name in sorted(names if names else os.listdir(d)):
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it matches the current kernels."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    if d.get("source_sha") != csrc_sha(d.get("sources")):  # the kernel's own sources
        return None
    v = d.get("bytes_per_launch", {}).get(kernel)
    return None if v is None else float(v)


class Clocks:
    """nvidia-smi sampler running across the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "50"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [c.strip() for c in line.split(",")]))

    def mark(self, which):
        setattr(self, which, time.time())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.2)
        self.proc.terminate()
        self.proc.wait(timeout=5)
        rows = [r for t, r in self.rows if self.t0 - 0.06 <= t <= self.t1 + 0.06] or [r for _, r in self.rows]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def time_steps(pm, torch, run, k, world):
    """CUDA-event time (ms) of k steps on the library's stream (the current torch stream)."""
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(st)
    run.step(k)
    e1.record(st)
    e1.synchronize()
    torch.cuda.synchronize()
    barrier(world)
    return e0.elapsed_time(e1)


def start_of_timed_steps(pm, torch, run, k):
    """Put the run at step GRID_STEPS - k of its a-grid (ICs, then the untimed steps before
    the timed ones), so that the k timed steps end at z = 0."""
    run.ic(seed=run.seed)
    run.step(GRID_STEPS - k)
    torch.cuda.synchronize()


def bench_precision(pm, torch, args, prec, rank, world, clocks=None, fft_threads=None):
    """The last K steps of the fixed GRID_STEPS-step run (z = 50 -> 0; the closing half kick
    included), after W warm-up steps taken on the same context from the ICs; then the same K
    steps again with the library's per-phase events on (the kernel rooflines cover the same
    steps as the headline)."""
    cfg = pm.make_config(args.np, args.nmesh, args.box, A_INIT, A_FINAL, GRID_STEPS, precision=prec)
    run = pm.PMRun(cfg)
    run.seed = 1 + rank
    run.ic(seed=run.seed)
    run.step(args.warmup)
    if fft_threads is None:  # the autotuner picks the form of the middle FFT passes
        tuned = pm.pm_autotune_fft(run.ctx)
    else:
        pm.pm_set_fused_fft(run.ctx, fft_threads)
        tuned = (fft_threads, None)
    start_of_timed_steps(pm, torch, run, args.steps)
    if clocks:
        clocks.mark("t0")
    ms = time_steps(pm, torch, run, args.steps, world)
    if clocks:
        clocks.mark("t1")
    ms = max_over_ranks(ms, world)
    start_of_timed_steps(pm, torch, run, args.steps)
    pm.pm_profile(run.ctx, True)
    pm.pm_timings(run.ctx)
    run.step(args.steps)
    phases = pm.pm_timings(run.ctx)
    pm.pm_profile(run.ctx, False)
    del run
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return ms, phases, tuned


def roofline(phases, np_side, n, fp64, peak, peak_kind, fused_fft=True):
    kb = kernel_bytes(np_side, n, fp64, fused_fft)
    dom = max(PHASES, key=lambda p: phases[p][0])
    ms, launches = phases[dom]
    per_launch_ms = ms / max(launches, 1)
    achieved = kb[dom] / (per_launch_ms * 1e-3) / 1e9
    table = {}
    for p in PHASES:
        t, c = phases[p]
        pl = t / max(c, 1)
        table[p] = {"ms_per_launch": round(pl, 4), "launches": c,
                    "GBps": round(kb[p] / (pl * 1e-3) / 1e9, 1) if pl > 0 else None,
                    "frac": round(kb[p] / (pl * 1e-3) / 1e9 / peak, 4) if pl > 0 else None}
    return {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": ncu_traffic(dom), "algorithmic_bytes": kb[dom],
            "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured" else "fallback"}, table


FP64_NOMINAL_TFLOPS = 1.25  # GB300 dense FP64, nominal
FP32_ALU_TFLOPS = round(152 * 128 * 2 * 2.07e9 / 1e12, 2)  # CUDA-core FP32 FMA rate at the maximum SM clock


def fp64_peak(torch):
    """Measured FP64 arithmetic ceiling of this GPU: a float64 torch.matmul (cuBLAS DGEMM) of
    4096^3, best of 5 (TFLOP/s); the nominal figure if the measurement fails."""
    try:
        n = 4096
        a = torch.randn((n, n), dtype=torch.float64, device="cuda")
        b = torch.randn((n, n), dtype=torch.float64, device="cuda")
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.matmul(a, b)
        best = float("inf")
        for _ in range(5):
            e0.record(st)
            torch.matmul(a, b)
            e1.record(st)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) * 1e-3)
        del a, b
        torch.cuda.empty_cache()
        return {"tflops": 2.0 * n**3 / best / 1e12, "source": "measured: float64 torch.matmul 4096^3, best of 5"}
    except RuntimeError:
        return {"tflops": FP64_NOMINAL_TFLOPS, "source": "nominal GB300 dense FP64 (measurement failed)"}


def fft_flops(n):
    """Flops of the FFT passes per phase of one FP32/FP64 force evaluation on an n^3 mesh,
    counting 5 L log2 L for a length-L complex transform and 10 flops per element of the
    r2c / c2r half-length split and of the per-mode Green / gradient operators."""
    import math
    M = n // 2
    cfft = lambda L: 5.0 * L * math.log2(L)
    rows = (M + 1) * n                      # rows of the half spectrum along y and columns along x
    zero = n * n * (cfft(M) + 10.0 * M)     # one r2c or c2r z pass of one mesh
    return {"fft_zy_fwd": zero + rows * cfft(n),
            "fft_x_green": rows * (3 * cfft(n) + 20.0 * n),   # forward, then phi and -i kx phi back
            "fft_yz_inv": 3 * rows * cfft(n) + 3 * zero}


def alu_roofline(phases, n, peak):
    """The FP64 passes are bound by FP64 arithmetic on this part: flops per launch of the
    slowest FFT phase against the measured FP64 matmul rate."""
    fl = fft_flops(n)
    dom = max(fl, key=lambda p: phases[p][0] / max(phases[p][1], 1))
    ms = phases[dom][0] / max(phases[dom][1], 1)
    achieved = fl[dom] / (ms * 1e-3) / 1e12
    return {"kernel": dom, "bound": "alu", "achieved": round(achieved, 3), "peak": round(peak["tflops"], 3),
            "unit": "TFLOP/s", "frac": round(achieved / peak["tflops"], 4), "flops_per_launch": fl[dom],
            "peak_source": peak["source"]}


def e2e(pm, torch, args, rank, world, n_jobs=2, form=0):
    """Public-API end to end over the headline's own steps: the state at step GRID_STEPS - K
    (positions and momenta, held in pinned host memory) copied to the device, restored with
    pm_set_state, the last K steps to z = 0 (FFT passes in the headline's tuned form), P(k) in
    64 bins read back to the host."""
    cfg = pm.make_config(args.np, args.nmesh, args.box, A_INIT, A_FINAL, GRID_STEPS)
    run = pm.PMRun(cfg)
    run.seed = 1 + rank
    pm.pm_set_fused_fft(run.ctx, form)
    start_of_timed_steps(pm, torch, run, args.steps)
    s0, _, sync0 = run.state()
    x0, p0 = run.particles()
    x_h = torch.empty_like(x0, device="cpu").pin_memory()
    p_h = torch.empty_like(p0, device="cpu").pin_memory()
    x_h.copy_(x0)
    p_h.copy_(p0)
    # the host state goes straight into the context's own arrays (pm_particles), positions and
    # momenta on two streams at once; pm_set_state then copies nothing and sets the integrator
    x, p = x0, p0
    cs = [torch.cuda.Stream(), torch.cuda.Stream()]
    torch.cuda.synchronize()
    import numpy as np
    edges = np.geomspace(1.0, args.nmesh / 2.0, 65)
    times = []
    for _ in range(n_jobs):
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        main = torch.cuda.current_stream()
        for s_c, dst, src in zip(cs, (x, p), (x_h, p_h)):
            s_c.wait_stream(main)
            with torch.cuda.stream(s_c):
                dst.copy_(src, non_blocking=True)
            main.wait_stream(s_c)
        pm.pm_set_state(run.ctx, x, p, s0, sync0)
        run.step(args.steps)
        k, pk, nm = run.power(edges)  # synchronises and copies P(k) to the host
        times.append(time.perf_counter() - t0)
    t = max_over_ranks(min(times), world)
    h2d = (x.numel() * x.element_size() + p.numel() * p.element_size()) / args.steps
    d2h = 3 * (len(edges) - 1) * 8 / args.steps
    del run
    torch.cuda.empty_cache()
    return {"value": world * args.np**3 * args.steps / t, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h),
            "what": f"the state at step {s0} of {GRID_STEPS} copied from pinned host memory into the "
                    f"context's arrays (positions and momenta on two streams) and restored (pm_set_state), "
                    f"the last {args.steps} PM steps to z = 0, P(k) (64 bins) read back"}


def batched(pm, torch, args):
    """64 realisations x 64^3 particles on 128^3 meshes, boxes cycling {1000, 2000, 4000} Mpc/h,
    FP32: one graph-replayed batched run against the same realisations stepped one by one."""
    import numpy as np
    B, np_side, n, grid_steps = args.batch, 64, 128, 50
    k = min(args.steps, grid_steps - 2)
    boxes = [(1000.0, 2000.0, 4000.0)[r % 3] for r in range(B)]
    seeds = list(range(1, B + 1))
    cfg = pm.make_config(np_side, n, 1000.0, A_INIT, A_FINAL, grid_steps)
    b = pm.PMBatch(cfg, boxes=boxes)
    chunk, tune_ms = b.autotune()  # realisations per launch and FFT form, picked by timing each candidate
    _, fft_form = b.tuning()
    b.ic(seeds)
    b.step(1, graph=False)  # initial deposits + attribute set-up, untimed
    b.step(k, graph=True)   # records the graph (untimed warm-up of the replay path)
    b.ic(seeds)
    b.step(1, graph=False)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    b.step(k, graph=True)   # replays the cached graph: one launch for k steps of all realisations
    e1.record(st)
    e1.synchronize()
    t_batch = e0.elapsed_time(e1) * 1e-3
    # the ensemble's purpose: the halo-proxy b1 of every realisation (top 5% of cells, 16 log bins,
    # k < 0.05 h/Mpc) and its spread across the realisations of each box, after the timed steps
    edges_b = pm.log_edges(16, 1.0, n / 2.0)
    b.bias(edges_b, k_max=0.05)  # bin tables and mode counts of each box's geometry, untimed
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b1 = b.bias(edges_b, k_max=0.05)[:, 0]
    ms_bias = 1e3 * (time.perf_counter() - t0)
    a_now = b.state()[1]
    by_box = {}
    for box in sorted(set(boxes)):
        v = np.array([b1[r] for r in range(B) if boxes[r] == box])
        by_box[f"{box:g}"] = {"n": int(v.size), "b1_mean": round(float(v.mean()), 4),
                              "b1_std": round(float(v.std(ddof=1)), 4) if v.size > 1 else None}
    bias = {"what": f"halo-proxy b1 (top 5% of cells, 16 log bins, k < 0.05 h/Mpc) of all {B} realisations "
                    f"at a = {a_now:.3f} (pm_batch_bias: proxy selection, cross and auto spectra, host fit)",
            "ms_all_realisations": round(ms_bias, 3), "by_box_mpc_h": by_box}
    del b
    torch.cuda.empty_cache()
    runs = {box: pm.PMRun(pm.make_config(np_side, n, box, A_INIT, A_FINAL, grid_steps)) for box in set(boxes)}
    for run in runs.values():  # the single runs take their own fastest FFT form too
        pm.pm_autotune_fft(run.ctx)
    t_seq = 0.0
    for r in range(B):
        run = runs[boxes[r]]
        run.ic(seed=seeds[r])
        run.step(1)
        torch.cuda.synchronize()
        e0.record(st)
        run.step(k)
        e1.record(st)
        e1.synchronize()
        t_seq += e0.elapsed_time(e1) * 1e-3
    units = B * np_side**3 * k
    return {"workload": f"{B} realisations x {np_side}^3 particles on {n}^3 meshes, boxes cycling "
                        "{1000, 2000, 4000} Mpc/h, FP32, one CUDA graph launch for all steps",
            "value": units / t_batch, "unit": UNIT, "ms_per_step": 1e3 * t_batch / k,
            "sequential_value": units / t_seq, "sequential_ms_per_step": 1e3 * t_seq / k,
            "speedup_vs_sequential": t_seq / t_batch, "steps": k, "bias": bias,
            "autotune": {"chunk": chunk, "fft_form": fft_form, "ms_per_step_at_tuning": round(tune_ms, 4),
                         "candidates": "middle FFT passes as separate launches (0) or on whole kz planes in "
                                       "shared memory (1), each with realisations per launch B, B/2, ..., 1"}}


def adjoint(pm, torch, args):
    """Gradient of the field-level loss against the plain forward run: 128^3 particles on a
    128^3 mesh, L = 2000 Mpc/h, 50 FP32 steps, checkpoints every 10 steps."""
    np_side = n = 128
    steps, every = 50, 10
    cfg = pm.make_config(np_side, n, 2000.0, A_INIT, A_FINAL, steps)
    run = pm.PMRun(cfg)
    run.ic(seed=2)
    run.step(steps)
    target = run.density().clone()
    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    w = torch.randn((np_side,) * 3, generator=g, device="cuda", dtype=torch.float32)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def forward():
        run.ic(white_noise=w)
        run.step(steps)
        return run.density()

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0.record(st)
            fn()
            e1.record(st)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) * 1e-3)
        return best

    t_fwd = timed(forward)
    t_grad = timed(lambda: run.loss_grad(w, target, checkpoint_every=every))
    # the general path: record the run, then the reverse sweep with cotangents on the final
    # density, displacements and momenta (what run_fields' backward hands to pm_adjoint_run)
    cot_d = torch.randn((n,) * 3, generator=g, device="cuda", dtype=torch.float32)
    cot_x = torch.randn((3, np_side**3), generator=g, device="cuda", dtype=torch.float32)
    cot_p = torch.randn((3, np_side**3), generator=g, device="cuda", dtype=torch.float32)

    def record_and_adjoint(r):
        r.record(w, every)
        return r.adjoint(d_delta=cot_d, d_disp=cot_x, d_mom=cot_p)

    t_vjp = timed(lambda: record_and_adjoint(run))
    del run
    # the same in the Poisson gauge on the horizon-scale box (lagged constraint, FP64 island)
    gr = pm.PMRun(pm.make_config(np_side, n, 4000.0, A_INIT, A_FINAL, steps, mode=pm.PM_GR_POISSON, n_lo=4))

    def forward_gr():
        gr.ic(white_noise=w)
        gr.step(steps)
        return gr.density()

    t_fwd_gr = timed(forward_gr)
    t_vjp_gr = timed(lambda: record_and_adjoint(gr))
    del gr
    torch.cuda.empty_cache()
    return {"workload": f"{np_side}^3 particles, {n}^3 mesh, L=2000 Mpc/h, {steps} FP32 steps, "
                        f"checkpoints every {every} steps; gradient with respect to the white-noise field",
            "forward_ms": 1e3 * t_fwd, "loss_grad_ms": 1e3 * t_grad, "cost_ratio": t_grad / t_fwd,
            "record_and_adjoint_ms": 1e3 * t_vjp, "record_and_adjoint_cost_ratio": t_vjp / t_fwd,
            "poisson_gauge": {"workload": f"as above in the Poisson gauge at L=4000 Mpc/h (n_lo=4)",
                              "forward_ms": 1e3 * t_fwd_gr, "record_and_adjoint_ms": 1e3 * t_vjp_gr,
                              "record_and_adjoint_cost_ratio": t_vjp_gr / t_fwd_gr},
            "what": "loss_grad: mean-square density loss (forward with checkpoints + reverse sweep); "
                    "record_and_adjoint: pm_adjoint_record + pm_adjoint_run with cotangents on the final "
                    "density, displacements and momenta (any loss)",
            "value": np_side**3 * steps / t_grad, "unit": "particle-steps/s (forward + reverse)"}


def estimators(pm, torch, args):
    """The per-output steps on the headline configuration (FP32, 512^3 particles on a 512^3
    mesh, L = 5000 Mpc/h, a few steps from the ZA ICs): P(k) in 64 log bins from the particles
    and from a mesh, B(k) for all triplets of 24 linear bins up to k = 0.05 h/Mpc on the
    alias-free m = 128 grid, the halo-proxy linear-bias fit (top 5%, k < 0.02 h/Mpc), and the GR
    displacement combination from a 256^3 pair onto the 512^3 lattice.  Each is timed with CUDA
    events (median of a few calls) next to the FP64 oracle on a small sample of the same kind."""
    import numpy as np
    from oracle import cic as ocic, combine as ocomb, stats as ostats
    peak, _ = peaks()
    np_side, n, box = args.np, args.nmesh, args.box
    s = 4
    R, S, P = s * n**3, 8 * (n // 2 + 1) * n * n, np_side**3
    run = pm.PMRun(pm.make_config(np_side, n, box, A_INIT, A_FINAL, 100))
    run.ic(seed=1)
    run.step(3)
    delta = run.density()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0.record(st)
            fn()
            e1.record(st)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    def host_timed(fn, reps=3):
        fn()
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)
        return 1e3 * float(np.median(ts))

    def line(ms, nbytes, what):
        gbs = nbytes / (ms * 1e-3) / 1e9
        return {"ms": round(ms, 4), "algorithmic_bytes": int(nbytes), "GBps": round(gbs, 1),
                "frac": round(gbs / peak, 4), "bytes_model": what}

    out = {"workload": f"{np_side}^3 particles on a {n}^3 mesh, L={box:g} Mpc/h, FP32, after 3 steps from z=50"}
    # the ICs themselves (Philox phases and Box-Muller in FP64, the Zel'dovich x pass, three
    # inverse transforms, placement); timed on a second context so the run above stays put
    ic_run = pm.PMRun(pm.make_config(np_side, n, box, A_INIT, A_FINAL, 100))
    ms_ic = timed(lambda: ic_run.ic(seed=2), reps=3)
    out["zeldovich_ics"] = {"ms": round(ms_ic, 3), "particles_per_s": round(P / (ms_ic * 1e-3), 1),
                            "bound": "FP64 Box-Muller of the phases (once per run)"}
    ms_ic2 = timed(lambda: ic_run.ic(seed=2, lpt_order=2), reps=3)
    out["lpt2_ics"] = {"ms": round(ms_ic2, 3), "particles_per_s": round(P / (ms_ic2 * 1e-3), 1),
                       "what": "second-order LPT ICs: the Zel'dovich chain plus four more three-output "
                               "FFT chains (derivatives of each Psi1 component, then Psi2) and the source"}
    del ic_run
    e64 = pm.log_edges(64, 1.0, n / 2.0)
    # after a step the fused update has left the density of the current positions in rho, which
    # P(k) of the particles then transforms directly
    out["power_particles"] = line(timed(lambda: run.power(e64)), R + S,
                                  "after a step: the step's density, one pass over its half spectrum")
    # standalone: the positions just set (pm_set_particles, untimed), so each call deposits them
    xs, ps = (t.clone() for t in run.particles())
    ts = []
    for rep in range(4):
        pm.pm_set_particles(run.ctx, xs, ps)
        torch.cuda.synchronize()
        e0.record(st)
        run.power(e64)
        e1.record(st)
        e1.synchronize()
        if rep:
            ts.append(e0.elapsed_time(e1))
    del xs, ps
    out["power_particles_standalone"] = line(float(np.median(ts)), 12 * P + 16 * n**3,
                                             "read x (12 B/particle), deposit and transform (16 B/cell)")
    out["power_field"] = line(timed(lambda: run.power(e64, field=delta)), R + S,
                              "read the field, one pass over its half spectrum")
    kf = 2 * np.pi / box
    e24 = np.linspace(0.0, 0.05 / kf, 25)
    ms_bk = timed(lambda: run.bispectrum(e24, 128, field=delta), reps=3)
    ntri = 24 * 25 * 26 // 6
    flops = 3.0 * ntri * 128**3  # S_ijl = sum_x I_i I_j I_l: two multiplies and an add a point
    tf = flops / (ms_bk * 1e-3) / 1e12
    out["bispectrum"] = {"ms": round(ms_bk, 3), "bins": 24, "triangles": ntri, "m": 128,
                         "triangle_sum_flops": flops, "TFLOPs": round(tf, 2),
                         "bound": "alu", "peak": FP32_ALU_TFLOPS, "frac": round(tf / FP32_ALU_TFLOPS, 4),
                         "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz",
                         "what": "FP32 triangle sums on the m-grid (integer counts cached) plus 24 masked "
                                 "spectra and their inverse FFTs of 128^3, over the whole call"}
    dh = torch.empty_like(delta)
    e32 = pm.log_edges(32, 1.0, n / 2.0)

    def bias():
        pm.pm_halo_proxy(run.ctx, dh, field=delta, fraction=0.05)
        pm.pm_linear_bias(run.ctx, dh, delta, e32, 0.02, terms=1)
    out["bias_fit"] = line(timed(bias, reps=3), 2 * R + 2 * (R + S),
                           "select the top 5% (read the field twice), cross and auto spectra")
    pair = [pm.PMRun(pm.make_config(np_side // 2, n // 2, box, A_INIT, A_FINAL, 100, mode=mode)) for mode in
            (pm.PM_GR_POISSON, pm.PM_NEWTON)]
    for r in pair:
        r.ic(seed=1)
    out["displacement_combination"] = line(
        timed(lambda: pm.pm_displacement_correction(run.ctx, pair[0].ctx, pair[1].ctx)),
        24 * P + 2 * 12 * (np_side // 2)**3, "read + write the target positions, read both pair positions")
    # cuFFT (through torch.fft) as a timing baseline for the transforms of one force evaluation:
    # one r2c of the density and three c2r of the gradient spectra (its Green's function and
    # gradient multiplies would be extra elementwise passes, not counted)
    spec = torch.fft.rfftn(delta)
    ms_r2c = timed(lambda: torch.fft.rfftn(delta), reps=5)
    ms_c2r = timed(lambda: torch.fft.irfftn(spec, s=delta.shape), reps=5)
    out["cufft_baseline"] = {"r2c_ms": round(ms_r2c, 4), "c2r_ms": round(ms_c2r, 4),
                             "force_transforms_ms": round(ms_r2c + 3 * ms_c2r, 4),
                             "what": f"torch.fft (cuFFT) on a {n}^3 FP32 mesh: one r2c + three c2r, without the "
                                     "Green's function and gradient passes; never on the product path"}
    del spec
    del pair, run, delta, dh
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    # the FP64 oracle beside them, on small samples of the same kind (one host core)
    rng = np.random.default_rng(5)
    f64 = rng.standard_normal((64, 64, 64))
    f32 = rng.standard_normal((32, 32, 32))
    e_o = ostats.log_edges(16, 1.0, 32.0)
    ms_pk = host_timed(lambda: ostats.power_spectrum(f64, 625.0, e_o))
    ms_bko = host_timed(lambda: ostats.bispectrum(f32, 312.5, np.linspace(0.0, 10.0, 7), M=32), reps=1)
    xt = (rng.integers(0, 2**32, size=(3, 64**3), dtype=np.uint64)).astype(np.uint32)
    xg = (rng.integers(0, 2**32, size=(3, 32**3), dtype=np.uint64)).astype(np.uint32)
    ms_co = host_timed(lambda: ocomb.combine(xt, ocomb.interpolate_lagrangian(ocomb.displacement(xg, xg), 32, 64)))
    out["cpu_oracle"] = {"cores": 1, "kind": "oracle",
                         "power_field_64^3_ms": round(ms_pk, 2),
                         "power_field_cells_per_s": round(64**3 / (ms_pk * 1e-3), 1),
                         "bispectrum_32^3_6bins_M32_ms": round(ms_bko, 2),
                         "combination_32^3_to_64^3_ms": round(ms_co, 2),
                         "combination_particles_per_s": round(64**3 / (ms_co * 1e-3), 1)}
    # the linearised Poisson-gauge step (Newtonian-form kick with the GR constraint, |n| <= 4 in FP64)
    gsteps, gwarm = 20, 3
    gr = pm.PMRun(pm.make_config(np_side, n, box, A_INIT, A_FINAL, gsteps + gwarm, mode=pm.PM_GR_POISSON, n_lo=4))
    gr.ic(seed=3)
    gr.step(gwarm)
    e0.record(st)
    gr.step(gsteps)
    e1.record(st)
    e1.synchronize()
    ms_gr = e0.elapsed_time(e1) / gsteps
    gr.ic(seed=3)
    gr.step(gwarm)
    pm.pm_profile(gr.ctx, True)
    pm.pm_timings(gr.ctx)
    gr.step(gsteps)
    ph_gr = pm.pm_timings(gr.ctx)
    pm.pm_profile(gr.ctx, False)
    out["gr_poisson_step"] = {"ms_per_step": round(ms_gr, 4), "steps": gsteps,
                              "phases_ms_per_launch": {k: round(v[0] / max(v[1], 1), 4) for k, v in ph_gr.items()
                                                       if v[1]},
                              "what": f"{np_side}^3 particles, {n}^3 mesh, Poisson-gauge Green's function "
                                      "with Phi_old and the FP64 island |n| <= 4, otherwise as the headline"}
    del gr
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    # the first-order gradient option (the paper's PM force): one inverse transform of the
    # potential, the update differentiating its CIC interpolant from eight corners
    fd = pm.PMRun(pm.make_config(np_side, n, box, A_INIT, A_FINAL, gsteps + gwarm, gradient=pm.PM_GRAD_FD1))
    fd.ic(seed=1)
    fd.step(gwarm)
    e0.record(st)
    fd.step(gsteps)
    e1.record(st)
    e1.synchronize()
    ms_fd = e0.elapsed_time(e1) / gsteps
    fd.ic(seed=1)
    fd.step(gwarm)
    pm.pm_profile(fd.ctx, True)
    pm.pm_timings(fd.ctx)
    fd.step(gsteps)
    ph = pm.pm_timings(fd.ctx)
    pm.pm_profile(fd.ctx, False)
    fd_bytes = 60 * P + 24 * n**3
    peak = peaks()[0]
    out["fd1_step"] = {"ms_per_step": round(ms_fd, 4), "steps": gsteps,
                       "particle_steps_per_s": round(P / (ms_fd * 1e-3), 1),
                       "step_roofline": {"bytes_per_step": fd_bytes,
                                         "frac": round(fd_bytes / (ms_fd * 1e-3) / 1e9 / peak, 4),
                                         "bytes_model": "60 B/particle + 24 B/cell (one inverse transform, "
                                                        "one mesh gathered)"},
                       "phases_ms_per_launch": {k: round(v[0] / max(v[1], 1), 4) for k, v in ph.items() if v[1]},
                       "what": f"{np_side}^3 particles, {n}^3 mesh, PM_GRAD_FD1 (first-order gradient of the CIC "
                               "interpolant of the potential), otherwise as the headline"}
    del fd
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    out["gpu_power_field_cells_per_s"] = round(n**3 / (out["power_field"]["ms"] * 1e-3), 1)
    out["gpu_combination_particles_per_s"] = round(P / (out["displacement_combination"]["ms"] * 1e-3), 1)
    return out


def host_cores():
    """(cores this process may run on, how that was found): the affinity mask where the
    platform has one, else the logical CPU count."""
    try:
        return len(os.sched_getaffinity(0)), "sched_getaffinity"
    except (AttributeError, OSError):
        return max(1, os.cpu_count() or 1), "os.cpu_count"


def gr_pair(pm, torch, n_lo=None):
    """The paired runs of the horizon-scale configuration: 128^3 particles on a 256^3 mesh,
    L = 4000 Mpc/h, the same Zel'dovich ICs at z = 100, 100 steps to z = 0 in the Newtonian and
    the Poisson-gauge (GR) mode, then the per-particle GR - Newtonian displacement xi and P(k)
    of both runs (32 log bins).  One job = both ICs, both runs, xi and both spectra."""
    import numpy as np
    np_side, n, box, a_i, steps = 128, 256, 4000.0, 1.0 / 101.0, 100
    lo = pm.DEFAULT_N_LO if n_lo is None else n_lo
    runs = [pm.PMRun(pm.make_config(np_side, n, box, a_i, 1.0, steps, mode=mode, n_lo=lo if mode else 0))
            for mode in (pm.PM_NEWTON, pm.PM_GR_POISSON)]
    target = pm.PMRun(pm.make_config(np_side, n, box, a_i, 1.0, steps))
    xi = torch.empty((3, np_side**3), dtype=torch.int32, device="cuda")
    edges = pm.log_edges(32, 1.0, n / 2.0)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def job():
        for r in runs:
            r.ic(seed=1)
            r.step(steps)
        target.ic(seed=1)
        pm.pm_displacement_correction(target.ctx, runs[1].ctx, runs[0].ctx, xi)
        return [r.power(edges) for r in runs]

    job()
    best = float("inf")
    for _ in range(3):
        torch.cuda.synchronize()
        e0.record(st)
        job()
        e1.record(st)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    xi_rms = float(xi.to(torch.float64).pow(2).mean().sqrt().item()) * box / 2.0**32
    del runs, target, xi
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return {"workload": f"{np_side}^3 particles on a {n}^3 mesh, L={box:g} Mpc/h, Zel'dovich ICs at z=100, {steps} "
                        f"steps to z=0, Newtonian and Poisson-gauge (n_lo={lo}) runs from the same seed, xi = "
                        "x_GR - x_N per particle, P(k) of both (32 log bins)",
            "ms_per_job": round(best, 3), "ms_per_step_per_run": round(best / (2 * steps), 4),
            "particle_steps_per_s": round(2 * np_side**3 * steps / (best * 1e-3), 1),
            "xi_rms_mpc_h": xi_rms}


def _oracle_sample(seconds, np_side=64, seed=1, gate=None, max_steps=99):
    """One process: the FP64 oracle on an np_side^3 sample of the workload at the same mesh
    spacing (L = 5000 np_side / 512 Mpc/h).  The ICs are built first; then the process waits
    at `gate` (shared by all processes, so their timed windows line up) and steps for about
    `seconds` (at least one step).  Returns (steps, wall start, wall end)."""
    from oracle import ic, pm as opm
    from oracle.cosmology import Cosmology
    box = 5000.0 * np_side / 512.0
    c = Cosmology()
    x, p = ic.zeldovich(c, np_side, box, A_INIT, seed=seed, fixed=True)
    run = opm.PMRun(c, np_side, box, A_INIT, A_FINAL, GRID_STEPS, x, p)
    if gate is not None:
        gate.wait()
    t0 = time.time()
    steps = 0
    while steps < max_steps and (time.time() - t0 < seconds or steps < 1):
        run.step(1)
        steps += 1
    return steps, t0, time.time()


class _OneThread:
    """OMP / OpenBLAS / MKL thread counts of 1 for spawned workers, restored on exit."""
    VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")

    def __enter__(self):
        self.saved = {v: os.environ.get(v) for v in self.VARS}
        for v in self.VARS:
            os.environ[v] = "1"

    def __exit__(self, *exc):
        for v, old in self.saved.items():
            if old is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = old


def _oracle_processes(nproc, seconds, np_side, max_steps):
    """nproc spawned single-threaded oracle processes released together by a barrier
    (spawned, so nothing forks after CUDA started).  Returns their results, or None when
    this host cannot start a process pool."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    try:
        with _OneThread(), ctx.Manager() as mgr:
            gate = mgr.Barrier(nproc)
            with ctx.Pool(nproc) as pool:
                return pool.starmap(_oracle_sample,
                                    [(seconds, np_side, 1 + i, gate, max_steps) for i in range(nproc)])
    except (OSError, EOFError):
        return None


def cpu_oracle(seconds, np_side=64):
    """The FP64 oracle on this host's cores: one single-threaded process per core, each
    stepping its own np_side^3 sample for about `seconds` after a common start; value =
    the particle-steps of all processes / the wall time from the common start to the
    last end."""
    cores, how = host_cores()
    t0 = time.perf_counter()
    res = _oracle_processes(cores, seconds, np_side, 99) if cores > 1 else None
    threads = "one thread a process"
    if res is None:  # no process pool on this host: one in-process sample
        cores, res = 1, [_oracle_sample(seconds, np_side)]
        threads = "numpy's thread pools as inherited"
    wall = time.perf_counter() - t0
    units = np_side**3
    span = max(e for _, _, e in res) - min(b for _, b, _ in res)
    rates = [units * n / (e - b) for n, b, e in res]
    box = 5000.0 * np_side / 512.0
    per_step_ms = statistics.median(1e3 * (e - b) / n for n, b, e in res)
    return {"value": units * sum(n for n, _, _ in res) / span, "unit": UNIT, "cores": cores, "cores_from": how,
            "kind": "oracle", "per_core_value": statistics.median(rates), "ms_per_step_per_process": per_step_ms,
            "sample": f"{cores} processes x {np_side}^3 particles on a {np_side}^3 mesh, L={box:g} Mpc/h "
                      f"(same cell size as 512^3 at L=5000), {min(n for n, _, _ in res)}-"
                      f"{max(n for n, _, _ in res)} KDK steps of the 100-step run from z=50 each, timed from a "
                      f"common start, FP64 numpy oracle, {threads}, {wall:.1f} s wall"}


def cpu_rows(sizes, all_cores_up_to=256, steps_per_row=1):
    """Per-step wall time of the oracle at each size: one process alone (steps_per_row steps
    after its ICs), and -- up to all_cores_up_to^3 -- one process per core stepping together
    (aggregate particle-steps/s over their common window)."""
    cores, how = host_cores()
    rows = {}
    for n in sizes:
        steps, b, e = _oracle_sample(1e9, n, 1, None, steps_per_row)
        row = {"one_process_ms_per_step": round(1e3 * (e - b) / steps, 1),
               "one_process_particle_steps_per_s": round(n**3 * steps / (e - b), 1)}
        if n <= all_cores_up_to and cores > 1:
            res = _oracle_processes(cores, 1e9, n, steps_per_row)
            if res:
                span = max(t for _, _, t in res) - min(t for _, t, _ in res)
                row["all_cores_particle_steps_per_s"] = round(n**3 * sum(k for k, _, _ in res) / span, 1)
                row["all_cores_ms_per_step_per_process"] = round(
                    statistics.median(1e3 * (t1 - t0) / k for k, t0, t1 in res), 1)
                row["cores"] = cores
        rows[f"{n}^3"] = row
    return {"kind": "oracle", "cores_from": how, "rows": rows,
            "what": "FP64 numpy oracle, particles = mesh cells, L = 5000 n / 512 Mpc/h (the headline's cell "
                    f"size), {steps_per_row} KDK step(s) of the 100-step run from z = 50 after the ICs, "
                    "per-step time = their wall time / their count"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--np", type=int, default=512)
    ap.add_argument("--nmesh", type=int, default=512)
    ap.add_argument("--box", type=float, default=5000.0)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-estimators", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the separate-FFT-passes comparison")
    ap.add_argument("--cpu-row-steps", type=int, default=1, help="oracle steps timed per --cpu-rows size")
    ap.add_argument("--fft-form", type=int, default=None,
                    help="form of the FFT passes (pm_set_fused_fft) instead of pm_autotune_fft's pick; profiler "
                         "runs use it, since timings taken under a profiler do not rank the forms")
    ap.add_argument("--cpu-rows", default="128",
                    help="comma-separated oracle sizes timed per step (e.g. 128,256,512); empty: none")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if not 1 <= args.steps <= GRID_STEPS:
        ap.error(f"--steps times the last K steps of the {GRID_STEPS}-step run: 1 <= K <= {GRID_STEPS}")
    world, rank, local = dist_setup()
    workload = (f"{args.np}^3 particles, {args.nmesh}^3 CIC mesh, L={args.box:g} Mpc/h, Newtonian PM, "
                f"ZA ICs at z=50, {GRID_STEPS} KDK steps on a uniform a-grid to z=0 (LCDM Om=0.31, EH no-wiggle, "
                f"sigma8=0.81); the last {args.steps} steps timed")
    config = {"workload": workload, "np": args.np, "nmesh": args.nmesh, "box_mpc_h": args.box,
              "a_grid_steps": GRID_STEPS, "timed_steps": f"{GRID_STEPS - args.steps}..{GRID_STEPS - 1} (ending at z=0)",
              "positions": "uint32 fixed point", "parallelism": f"replicas x{world}",
              "l2": "inputs larger than L2 (3.2 GB particles, 0.5 GB per mesh); no flush"}

    if args.impl == "reference":
        if rank != 0:
            return
        ms_t0 = time.perf_counter()
        cb = cpu_oracle(max(args.cpu_seconds, 5.0))
        total = time.perf_counter() - ms_t0
        sample_cfg = {"workload": "the FP64 oracle on a sample of the workload: " + cb["sample"],
                      "np": 64, "nmesh": 64, "box_mpc_h": 625.0, "a_grid_steps": GRID_STEPS,
                      "parallelism": f"{cb['cores']} host processes", "sample_of": workload}
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": cb["ms_per_step_per_process"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded Philox phases)", "config": sample_cfg,
                "cpu_baseline": {**cb}, "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                                "d2h_bytes_per_step": 0},
                "note": f"FP64 CPU oracle timed on a bounded sample ({total:.1f} s wall); ms_per_step is the "
                        "median wall time of one oracle step of one 64^3 process"}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group(backend="nccl")
    else:
        torch.cuda.set_device(0)
    import paper_2404_02783_gb300 as pm
    pm.lib()
    peak, peak_kind = peaks()
    clocks = Clocks(local if world > 1 else 0)
    clocks.start()
    ms32, ph32, tuned = bench_precision(pm, torch, args, pm.PM_FP32_FIXED, rank, world, clocks,
                                        fft_threads=args.fft_form)
    clk = clocks.stop()
    value = world * args.np**3 * args.steps / (ms32 * 1e-3)
    ms_step = ms32 / args.steps
    fused = tuned[0] > 0
    roof, table32 = roofline(ph32, args.np, args.nmesh, False, peak, peak_kind, fused_fft=fused)
    sb = step_bytes(args.np, args.nmesh, False)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded Philox phases, EH no-wiggle LCDM)",
           "config": config, "clocks": clk,
           "gpu_launches": launches_per_step(args.np, args.nmesh, False, fused) * (args.steps + 1),  # + closing kick
           "roofline": roof,
           "step_roofline": {"bytes_per_step": sb, "achieved": round(sb / (ms_step * 1e-3) / 1e9, 1),
                             "peak": peak, "unit": "GB/s", "frac": round(sb / (ms_step * 1e-3) / 1e9 / peak, 4),
                             "bytes_model": "60 B/particle + 40 B/cell"},
           "phases_fp32": table32,
           "fft_middle": {"threads": tuned[0], "tuned_ms": tuned[1],
                          "what": "form of the forward y / x / inverse y passes picked by pm_autotune_fft: "
                                  "0 = three launches, else the CTA size of the fused persistent kernel"}}
    if fused_middle(args.nmesh, False) and not args.no_compare:
        other = 0 if fused else 512
        ms_o, ph_o, _ = bench_precision(pm, torch, args, pm.PM_FP32_FIXED, rank, world, fft_threads=other)
        _, table_o = roofline(ph_o, args.np, args.nmesh, False, peak, peak_kind, fused_fft=other > 0)
        out["fft_middle"]["other_form"] = {
            "threads": other, "ms_per_step": ms_o / args.steps,
            "value": world * args.np**3 * args.steps / (ms_o * 1e-3),
            "step_roofline_frac": round(sb / (ms_o / args.steps * 1e-3) / 1e9 / peak, 4),
            "phases": table_o}
    if not args.no_fp64:
        ms64, ph64, _ = bench_precision(pm, torch, args, pm.PM_FP64, rank, world)
        sb64 = step_bytes(args.np, args.nmesh, True)
        roof64, table64 = roofline(ph64, args.np, args.nmesh, True, peak, peak_kind)
        out["fp64_plain"] = {"value": world * args.np**3 * args.steps / (ms64 * 1e-3), "unit": UNIT,
                             "ms_per_step": ms64 / args.steps,
                             "step_roofline_frac": round(sb64 / (ms64 / args.steps * 1e-3) / 1e9 / peak, 4),
                             "dominant": roof64, "alu_roofline": alu_roofline(ph64, args.nmesh, fp64_peak(torch)),
                             "phases": table64}
    if not args.no_e2e:
        out["e2e"] = e2e(pm, torch, args, rank, world, form=tuned[0])
    if not args.no_batch:
        out["batched"] = batched(pm, torch, args)
    if not args.no_adjoint:
        out["adjoint"] = adjoint(pm, torch, args)
    if not args.no_estimators and rank == 0:
        out["estimators"] = estimators(pm, torch, args)
        cb = out["estimators"]["cufft_baseline"]
        cb["ours_fft_phases_ms"] = round(sum(table32[p]["ms_per_launch"] for p in ("fft_zy_fwd", "fft_x_green",
                                                                                   "fft_yz_inv")), 4)
    if not args.no_estimators and rank == 0:
        out["gr_pair"] = gr_pair(pm, torch)
    if rank == 0:
        out["cpu_baseline"] = cpu_oracle(args.cpu_seconds)
        sizes = [int(v) for v in args.cpu_rows.split(",") if v.strip()]
        if sizes:
            out["cpu_baseline"]["per_size"] = cpu_rows(sizes, steps_per_row=max(1, args.cpu_row_steps))
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
