"""Benchmark of the MBL eigensolver hot path on GB300.

One step = one full pass of the hot path on the L = 20 periodic chain (S^z = 0,
n = 184,756, delta = 1, h ~ U[-8, 8] from seed 1): basis build, spectrum bounds
(sigma = (E_min + E_max)/2, ||H|| = max |E|), and the folded LOBPCG for the 16
eigenpairs nearest sigma with block width 32 in mixed precision (FP32 Jacobi-PCG,
FP64 Rayleigh-Ritz and residuals), accepted at ||Hy - lambda y|| <= 1e-8 ||H||.
Metric: eigenpairs per second.  Also reported: the same solve in plain FP64, the
block-product bandwidth sweep on L = 22..28 open chains (the roofline), the e2e
figure through the C ABI with host buffers, and the CPU oracle on a bounded sample.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

CFG = wl.SOLVE_L20
PCG_ITERS = 320
METRIC = "eigenpairs/s at ||r||/||H|| <= 1e-8 (mixed FP32-PCG / FP64-LOBPCG)"
L2_FLUSH_BYTES = 512 << 20
# Residual tolerance of the extreme Ritz pairs: their eigenvalues are then accurate to
# about tol^2 |E| / gap, far below what sigma and ||H|| need.
BOUNDS_TOL = 1e-7


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self):
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", "bench_clocks.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        if sm:
            out = {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def _setup(torch, mbl, dev):
    L, k, nev = CFG["L"], CFG["k"], CFG["nev"]
    h = wl.fields(L, CFG["W"], CFG["seed"])
    n = mbl.basis_size(L, L // 2)
    chain = mbl.make_chain(L, h, CFG["delta"], CFG["periodic"])
    X0_host = torch.from_numpy(wl.initial_block(n, k, CFG["seed"])).pin_memory()
    Xb_host = torch.from_numpy(wl.block(n, 4, CFG["seed"] + 100)).pin_memory()
    return dict(L=L, k=k, nev=nev, h=h, n=n, chain=chain, X0_host=X0_host, Xb_host=Xb_host)


class Step:
    """Device buffers and one pass of the hot path."""

    def __init__(self, torch, mbl, dev, s, mode):
        self.torch, self.mbl, self.s, self.mode = torch, mbl, s, mode
        self.opts = mbl.make_opts(s["nev"], s["k"], tol=1e-8, max_iter=400, pcg_iters=PCG_ITERS, mode=mode,
                                  use_graph=1)
        ws = max(mbl.lobpcg_workspace_size(s["chain"], self.opts), mbl.bounds_workspace_size(s["chain"], 4))
        self.ws = torch.empty(ws, dtype=torch.uint8, device=dev)
        self.states = torch.empty(s["n"], dtype=torch.int32, device=dev)
        self.X0 = s["X0_host"].to(dev)
        self.Xb = s["Xb_host"].to(dev)
        self.evecs = torch.empty((s["n"], s["nev"]), dtype=torch.float64, device=dev)
        self.last = None

    def run(self):
        mbl, s = self.mbl, self.s
        mbl.basis_build(s["L"], s["L"] // 2, self.states)
        emin, emax, bit = mbl.spectrum_bounds(s["chain"], self.Xb, self.ws, tol=BOUNDS_TOL, max_iter=1000)
        sigma = 0.5 * (emin + emax)
        self.opts.norm_h = max(abs(emin), abs(emax))
        evals, resid, stats, rc = mbl.lobpcg_solve(s["chain"], sigma, self.opts, self.X0, self.ws, self.evecs)
        self.last = dict(evals=evals, resid=resid, stats=stats, sigma=sigma, emin=emin, emax=emax,
                         bounds_iters=bit)
        return self.last

    def run_e2e(self, X0_host, Xb_host, evecs_host):
        """Same pass with host inputs and outputs: H2D of the start blocks, D2H of the
        eigenvectors (evals/resid come back through the ABI's host arrays)."""
        self.X0.copy_(X0_host, non_blocking=True)
        self.Xb.copy_(Xb_host, non_blocking=True)
        out = self.run()
        evecs_host.copy_(self.evecs, non_blocking=True)
        return out


def _time_steps(torch, step_fn, steps, flush):
    st = torch.cuda.current_stream()
    times = []
    for _ in range(steps):
        flush.add_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        step_fn()
        e1.record(st)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    return times


def _graph_time(torch, fn, reps, flush=None):
    """Average device time of fn() per call: reps calls captured in one CUDA graph and
    replayed (no host launch overhead).  With flush, L2 is flushed by a write of
    L2_FLUSH_BYTES before each call, and that write is timed separately and subtracted."""
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        fn()  # first call outside the capture (attributes, lazy setup)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            for _ in range(reps):
                if flush is not None:
                    flush.add_(1.0)
                fn()
        gf = None
        if flush is not None:
            gf = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gf, stream=st):
                for _ in range(reps):
                    flush.add_(1.0)
    torch.cuda.current_stream().wait_stream(st)
    torch.cuda.synchronize()

    def run(graph):
        graph.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        graph.replay()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3

    t = run(g)
    if gf is not None:
        t -= run(gf)
    return t / reps


def matvec_roofline(torch, mbl, dev, peak_gbs, quick=False):
    """Block product bandwidth on the open-chain sweep (FP32 and FP64), L2 flushed
    before every launch; algorithmic bytes = read X once + write Y once = 2 n k b."""
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    rows = []
    sweep = wl.MATVEC_SWEEP if not quick else wl.MATVEC_SWEEP[:1]
    for cfg in sweep:
        L = cfg["L"]
        h = wl.fields(L, cfg["W"], cfg["seed"])
        chain = mbl.make_chain(L, h, cfg["delta"], cfg["periodic"])
        n = mbl.basis_size(L, L // 2)
        for dtype, tdt in (("f32", torch.float32), ("f64", torch.float64)):
            for k in cfg["ks"]:
                es = 4 if dtype == "f32" else 8
                if n * k * es * 2 > 24e9:
                    continue
                g = torch.Generator(device=dev)
                g.manual_seed(k)
                X = torch.randn((n, k), generator=g, device=dev, dtype=tdt)
                Y = torch.empty_like(X)
                reps = 5 if n * k * es > 1e9 else 20
                t = _graph_time(torch, lambda: mbl.hamiltonian_apply(chain, 0.0, X, Y), reps, flush)
                gbs = 2.0 * n * k * es / t / 1e9
                rows.append(dict(L=L, k=k, dtype=dtype, n=n, us=t * 1e6, gbs=gbs, frac=gbs / peak_gbs,
                                 l2_resident=bool(2 * n * k * es < 126e6)))
                del X, Y
    return rows


def solve_kernel_roofline(torch, mbl, dev, s, peak_gbs):
    """The dominant kernel of the step: the FP32 block product of every PCG step
    (n = 184,756, k = 32).  Timed alone with CUDA events over a replayed graph: back to
    back as in the solve (its 47 MB of operands stay in L2) and with L2 flushed."""
    chain, n, k = s["chain"], s["n"], s["k"]
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    X = torch.randn((n, k), generator=g, device=dev, dtype=torch.float32)
    Y = torch.empty_like(X)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    fn = lambda: mbl.hamiltonian_apply(chain, 0.1, X, Y)  # noqa: E731
    t_warm = _graph_time(torch, fn, 50)
    t_cold = _graph_time(torch, fn, 20, flush)
    alg = 2.0 * n * k * 4
    return dict(kernel="k_apply<float,32> (PCG block product)", alg_bytes=alg, t_l2_warm_us=t_warm * 1e6,
                t_cold_us=t_cold * 1e6, gbs_cold=alg / t_cold / 1e9, gbs_warm=alg / t_warm / 1e9)


def cpu_baseline(s, gpu_iters, budget_s=20.0):
    """The oracle as it stands on this host: one LOBPCG iteration of the same workload
    (bounds + setup + 1 iteration with the same PCG count), extrapolated to the GPU's
    iteration count; returns eigenpairs/s."""
    from oracle import hamiltonian as ham
    from oracle import solver
    threads = os.cpu_count() or 1
    ch = ham.Chain(s["L"], s["h"], delta=CFG["delta"], periodic=CFG["periodic"])
    X0 = wl.initial_block(s["n"], s["k"], CFG["seed"])
    t0 = time.perf_counter()
    # one matvec to price the rest
    ham.apply(ch, 0.0, X0[:, :4])
    t_mv = time.perf_counter() - t0
    # PCG count reduced so the sample stays within the budget
    m = PCG_ITERS
    per_iter_est = t_mv / 4 * s["k"] * (2 * m + 8)
    m_sample = int(max(4, min(m, m * budget_s / max(per_iter_est, 1e-9))))
    t0 = time.perf_counter()
    r = solver.lobpcg_folded(ch, 0.0, X0, s["nev"], 1e-30, 1.0, max_iter=1, pcg_iters=m_sample)
    t_sample = time.perf_counter() - t0
    t_iter = t_sample * (2 * m + 8) / (2 * m_sample + 8)  # scale PCG work to the full count
    t_solve = t_iter * max(gpu_iters, 1)
    return dict(value=s["nev"] / t_solve, unit="eigenpairs/s", cores=threads, kind="oracle",
                sample="1 LOBPCG iteration of the L=20 solve with %d of %d PCG steps (%.1f s), "
                       "scaled to %d PCG steps x %d iterations" % (m_sample, m, t_sample, m, gpu_iters))


def run_reference(args):
    """--impl reference: the CPU oracle as it stands, each step a bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch  # noqa: F401
    s = dict(L=CFG["L"], k=CFG["k"], nev=CFG["nev"], h=wl.fields(CFG["L"], CFG["W"], CFG["seed"]),
             n=wl.sector_dim(CFG["L"]))
    vals = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(s, gpu_iters=30, budget_s=8.0)
        if i >= args.warmup:
            vals.append(cb["value"])
    v = float(np.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "eigenpairs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": CFG["name"], "n": s["n"], "nev": s["nev"], "k": s["k"], "pcg_iters": PCG_ITERS},
            "cpu_baseline": dict(cb, value=v),
            "e2e": {"value": v, "unit": "eigenpairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_profile(args):
    """Small fixed workloads for ncu: 'product' launches the L = 20 (k = 32) and L = 26
    (k = 64) FP32 block products three times each; 'pcg' runs a 3-iteration solve;
    'bounds' runs the spectrum bounds of the bench workload once."""
    import torch
    import paper_2012_00217_gb300 as mbl
    dev = torch.device("cuda:0")
    mbl.binding.lib()
    if args.profile == "product":
        for L, periodic, k in ((20, True, 32), (26, False, 64)):
            h = wl.fields(L, 8.0, 1 if L == 20 else 0)
            chain = mbl.make_chain(L, h, 1.0, periodic)
            n = mbl.basis_size(L, L // 2)
            g = torch.Generator(device=dev)
            g.manual_seed(3)
            X = torch.randn((n, k), generator=g, device=dev, dtype=torch.float32)
            Y = torch.empty_like(X)
            for _ in range(3):
                mbl.hamiltonian_apply(chain, 0.0, X, Y)
            torch.cuda.synchronize()
            del X, Y
    elif args.profile == "bounds":
        s = _setup(torch, mbl, dev)
        step = Step(torch, mbl, dev, s, mbl.MODE_MIXED)
        mbl.spectrum_bounds(s["chain"], step.Xb, step.ws, tol=BOUNDS_TOL, max_iter=1000)
        torch.cuda.synchronize()
    else:
        s = _setup(torch, mbl, dev)
        step = Step(torch, mbl, dev, s, mbl.MODE_MIXED)
        step.opts.max_iter = 3
        step.opts.use_graph = 0
        mbl.basis_build(s["L"], s["L"] // 2, step.states)
        emin, emax, _ = -37.11044143972399, 33.466977761420935, 0
        step.opts.norm_h = max(abs(emin), abs(emax))
        mbl.lobpcg_solve(s["chain"], 0.5 * (emin + emax), step.opts, step.X0, step.ws, step.evecs,
                         allow_not_converged=True)
        torch.cuda.synchronize()
    print(json.dumps({"profile": args.profile, "ok": True}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="skip the sweep and the CPU baseline")
    ap.add_argument("--profile", choices=["product", "pcg", "bounds"], default=None,
                    help="profiling driver: only run the block products (L=20 k=32 FP32 and L=26 k=64 "
                         "FP32) or a 3-iteration solve, for an ncu capture")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile(args)

    import torch
    import paper_2012_00217_gb300 as mbl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda:%d" % local)
    torch.cuda.set_device(dev)
    mbl.binding.lib()
    peaks, peak_kind = _peaks()

    s = _setup(torch, mbl, dev)
    step = Step(torch, mbl, dev, s, mbl.MODE_MIXED)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        step.run()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks()
    clocks.start()
    times = _time_steps(torch, step.run, args.steps, flush)
    ck = clocks.stop()
    t_step = float(np.max(times))
    t_med = float(np.median(times))
    if world > 1:
        tt = torch.tensor([t_med], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_med = float(tt.item())
    res = step.last
    value = world * s["nev"] / t_med
    # e2e through the ABI with host buffers
    evecs_host = torch.empty((s["n"], s["nev"]), dtype=torch.float64).pin_memory()
    e2e_times = _time_steps(torch, lambda: step.run_e2e(s["X0_host"], s["Xb_host"], evecs_host),
                            max(2, args.steps // 2), flush)
    h2d = s["X0_host"].numel() * 8 + s["Xb_host"].numel() * 8
    d2h = evecs_host.numel() * 8 + 2 * s["nev"] * 8
    # plain FP64 solve for comparison
    step64 = Step(torch, mbl, dev, s, mbl.MODE_FP64)
    step64.run()
    t64 = _time_steps(torch, step64.run, 1, flush)[0]
    res64 = step64.last
    # spectrum bounds alone (the first part of every step)
    t_b = _time_steps(torch, lambda: mbl.spectrum_bounds(s["chain"], step.Xb, step.ws, tol=BOUNDS_TOL,
                                                         max_iter=1000), 1, flush)[0]
    # per-phase device time of one solve (events between phases; graphs off)
    step.opts.timing = 1
    step.run()
    step.opts.timing = 0
    phases = {kk: v for kk, v in step.last["stats"].items() if kk.startswith("t_")}
    kern = solve_kernel_roofline(torch, mbl, dev, s, peaks["hbm_gbs"])
    sweep = [] if args.quick else matvec_roofline(torch, mbl, dev, peaks["hbm_gbs"])
    big = [r for r in sweep if r["L"] == 26 and r["k"] == 64 and r["dtype"] == "f32"]
    head = big[0] if big else None

    line = {
        "metric": METRIC,
        "value": value,
        "unit": "eigenpairs/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_med * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": CFG["name"], "L": s["L"], "n": s["n"], "nev": s["nev"], "k": s["k"],
                   "pcg_iters": PCG_ITERS, "tol": 1e-8, "mode": "mixed", "l2": "flushed between steps",
                   "parallelism": "replicas" if world > 1 else "single"},
        "solve": {"iters": res["stats"]["iters"], "matvecs": res["stats"]["matvecs"],
                  "max_rel_resid": res["stats"]["max_rel_resid"], "sigma": res["sigma"],
                  "emin": res["emin"], "emax": res["emax"], "bounds_iters": res["bounds_iters"],
                  "step_ms_all": [t * 1e3 for t in times]},
        "fp64": {"eigenpairs_per_s": s["nev"] / t64, "ms": t64 * 1e3, "iters": res64["stats"]["iters"],
                 "max_rel_resid": res64["stats"]["max_rel_resid"],
                 "max_eval_diff_vs_mixed_rel": float(np.max(np.abs(res64["evals"] - res["evals"])) /
                                                     res["stats"]["norm_h"])},
        "e2e": {"value": world * s["nev"] / float(np.median(e2e_times)), "unit": "eigenpairs/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": None,
        "roofline": None,
        "solve_kernel": kern,
        "solve_phases_s": phases,
        "bounds_s": t_b,
        "matvec_sweep": sweep,
        "clocks": ck,
    }
    if head is not None:
        line["roofline"] = {"bound": "hbm", "achieved": head["gbs"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                            "frac": head["gbs"] / peaks["hbm_gbs"], "traffic": None,
                            "kernel": "k_apply<float,64> L=26 open k=64 (block product)",
                            "peak_kind": peak_kind + " (hbm_gbs)"}
    if rank == 0 and world == 1 and not args.quick:
        line["cpu_baseline"] = cpu_baseline(s, res["stats"]["iters"])
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
