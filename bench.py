"""Benchmark: one MAHI step (E, F, dE/dlambda) on the 1M-atom / 512-site water
workload, mixed precision (tensor-core M2L), next to the FP64 GPU path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Inputs are synthetic (seeded generator, the
paper's random/solvated workload shapes); positions are resident in HBM when
the timed region starts.  Each timed step is one replay of the handle's CUDA
graph (captured once with mahi_batch_create, as an MD loop would run it); the
same steps as plain mahi_eval calls are reported beside it.  The L2 (129 MB) is
flushed between timed steps by writing a 256 MB buffer; only the steps
themselves are inside the CUDA-event windows.  Under torchrun every rank evaluates its own replica (the method has
no exchange step on one GPU), so scaling is weak and the step time is the max
over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="water_1M_512sites", config="C", seed=1, order=12, depth=5)
METRIC = "MAHI E+F+dV/dλ step ms at 1M atoms/512 sites vs FP64 GPU path, force err≤1e-4"
TF32_PER_BF16 = 1.1 / 2.25          # nominal dense TF32 / BF16 tensor rates (GB300)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples, time-stamped on arrival, so that the
    summary can keep those taken while the timed region ran.  Start it before
    the warm-up: nvidia-smi takes a while to come up."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0, period_ms=20):
        self.index = index
        self.period_ms = period_ms
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def wait_ready(self, timeout=5.0):
        t0 = time.perf_counter()
        while self.proc and not self.lines and time.perf_counter() - t0 < timeout:
            time.sleep(0.01)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0=None, t1=None):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, ln in self.lines:
            # a sample stamped up to one period after the window still reports it
            if t0 is not None and not (t0 <= ts <= t1 + self.period_ms * 1e-3):
                continue
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "period_ms": self.period_ms}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("MAHI_BENCH_GLOO") is None else "gloo")
        return dist, rank, ws
    return None, 0, 1


def _max_over_ranks(dist, v, device):
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args):
    import torch

    import paper_2410_01754_gb300 as pkg
    import synth
    from paper_2410_01754_gb300 import build as pkg_build

    pkg_build.build()
    dist, rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s = synth.make(args.case, WORKLOAD["seed"])
    N, S, L = len(s["qA"]), len(s["lam"]), s["L"]
    stream = torch.cuda.Stream(device=dev)
    x = torch.tensor(s["x"], dtype=torch.float32, device=dev)
    lam = torch.tensor(s["lam"], dtype=torch.float64, device=dev)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    F = torch.empty_like(x)
    g = torch.zeros(S, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def make(prec):
        h = pkg.mahi_create(L, N, S, WORKLOAD["order"], WORKLOAD["depth"], prec, stream)
        pkg.mahi_set_charges(h, s["qA"], s["qB"], s["site_of"])
        return h

    h = make("mixed")
    clk = ClockSampler(local).__enter__()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            pkg.mahi_eval(h, x, lam, E, F, g)
        stream.synchronize()
        clk.wait_ready()
        launches = pkg.mahi_launch_count(h)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        t_clk0 = t_wall
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            pkg.mahi_eval(h, x, lam, E, F, g)
            ev[k][1].record(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        step_ms = [a.elapsed_time(b) for a, b in ev]
        graph_ms = None
        if not args.kernels_only:
            # the same step replayed as a CUDA graph of the handle (how an MD
            # loop runs it: capture once, update the positions in place)
            batch = pkg.MahiBatch([h], stream, [x], [lam], [E], [F], [g])
            for _ in range(args.warmup):
                batch.launch()
            stream.synchronize()
            evg = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            for k in range(args.steps):
                flush.fill_(float(k))
                evg[k][0].record(stream)
                batch.launch()
                evg[k][1].record(stream)
            stream.synchronize()
            graph_ms = [a.elapsed_time(b) for a, b in evg]
            batch.close()
        t_clk1 = time.perf_counter()
        t_wall = t_clk1 - t_wall
        if dist:
            dist.barrier()
    clk.__exit__()
    ms_eager = _max_over_ranks(dist, float(np.mean(step_ms)), dev)
    ms = _max_over_ranks(dist, float(np.mean(graph_ms)), dev) if graph_ms else ms_eager
    if args.kernels_only:
        # the timed steps alone (profiling runs): no stages, e2e, comparator
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": round(ms, 4), "unit": "ms", "n_gpus": ws,
                              "steps": args.steps, "warmup": args.warmup, "kernels_only": True,
                              "gpu_launches": int(launches * args.steps)}), flush=True)
        pkg.mahi_destroy(h)
        if dist:
            dist.destroy_process_group()
        return

    # stage breakdown and the dominant kernel (tensor-core M2L) timed with the
    # library's CUDA events on the same stream
    pkg.mahi_set_timing(h, True)
    stages = {}
    with torch.cuda.stream(stream):
        for k in range(3):
            flush.fill_(1.0)
            pkg.mahi_eval(h, x, lam, E, F, g)
            st = pkg.mahi_stage_times(h)
            for kk, v in st.items():
                stages.setdefault(kk, []).append(v)
    pkg.mahi_set_timing(h, False)
    stages = {k: float(np.median(v)) for k, v in stages.items()}
    Em = E.item()
    Fm = F.double().cpu().numpy()
    gm = g.cpu().numpy()

    # end to end through the C ABI with host buffers (pinned)
    xh = torch.tensor(s["x"], dtype=torch.float32).pin_memory().numpy()
    lh = torch.tensor(s["lam"], dtype=torch.float64).pin_memory().numpy()
    Eh = torch.zeros(1, dtype=torch.float64).pin_memory().numpy()
    Fh = torch.zeros((N, 3), dtype=torch.float32).pin_memory().numpy()
    gh = torch.zeros(S, dtype=torch.float64).pin_memory().numpy()
    for _ in range(2):
        pkg.mahi_eval_host(h, xh, lh, Eh, Fh, gh)
    e2e = []
    for k in range(max(3, args.steps // 2)):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pkg.mahi_eval_host(h, xh, lh, Eh, Fh, gh)
        e2e.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = _max_over_ranks(dist, float(np.mean(e2e)), dev)
    pkg.mahi_destroy(h)

    # FP64 GPU path on the same input (the comparator of the metric)
    h64 = make("fp64")
    E64 = torch.zeros(1, dtype=torch.float64, device=dev)
    F64 = torch.empty_like(x)
    g64 = torch.zeros(S, dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        pkg.mahi_eval(h64, x, lam, E64, F64, g64)
        stream.synchronize()
        t64 = []
        for k in range(max(2, min(3, args.steps))):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pkg.mahi_eval(h64, x, lam, E64, F64, g64)
            b.record(stream)
            stream.synchronize()
            t64.append(a.elapsed_time(b))
    pkg.mahi_destroy(h64)
    ms64 = _max_over_ranks(dist, float(np.mean(t64)), dev)
    F64n = F64.double().cpu().numpy()
    err = dict(energy_rel=abs(Em - E64.item()) / abs(E64.item()),
               force_rel_rms=float(np.sqrt(((Fm - F64n) ** 2).sum() / (F64n ** 2).sum())),
               dEdl_max_abs=float(np.abs(gm - g64.cpu().numpy()).max()))

    peaks, src = _peaks()
    K = (WORKLOAD["order"] + 1) ** 2
    translations = 189 * sum(8 ** l for l in range(1, WORKLOAD["depth"] + 1))
    m2l_flop = 2.0 * K * K * translations
    # tensor work: per translation and 8-coefficient K chunk, N = 176 padded outputs; the two
    # chunks of degree <= 2 take three products (hi*hi, hi*lo, lo*hi), the other 20 one
    Kp = ((K + 15) // 16) * 16
    nch, nsplit = Kp // 8, 2
    tensor_flop = 2.0 * Kp * 8 * (3 * nsplit + (nch - nsplit)) * translations
    m2l_ms = stages.get("m2l")
    # the M2L is timed inside a ~5 ms step whose timed loop lasts well under a
    # second: the burst figure applies
    peak_tf32 = peaks["bf16_tflops"] * TF32_PER_BF16
    achieved = m2l_flop / (m2l_ms * 1e-3) / 1e12 if m2l_ms else None
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "m2l_tc_traffic.json")
    if os.path.exists(tpath):
        try:
            traffic = json.load(open(tpath)).get("bytes_per_launch")
        except (OSError, ValueError):
            traffic = None
    clocks = clk.summary(t_clk0, t_clk1)
    out = {
        "metric": METRIC, "value": round(ms, 4), "unit": "ms", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 + tf32 M2L (3 products to degree 2) + f64 lattice/site terms/energy",
        "data": "synthetic",
        "config": {"workload": WORKLOAD["name"], "n_atoms": N, "n_sites": S, "box_nm": L,
                   "order_p": WORKLOAD["order"], "depth": WORKLOAD["depth"], "precision": "mixed",
                   "positions": "float32", "l2": "flushed between timed steps (256 MB write)",
                   "launch": "each step one replay of the handle's CUDA graph (mahi_batch_create); "
                             "ms_per_step_eager: the same steps as mahi_eval calls",
                   "parallelism": f"replicas x{ws}"},
        "ms_per_step_eager": round(ms_eager, 4),
        "atoms_per_s": round(ws * N / (ms * 1e-3), 1),
        "fp64_gpu_ms_per_step": round(ms64, 3), "speedup_vs_fp64_gpu": round(ms64 / ms, 2),
        "errors_vs_fp64_gpu": err,
        "stage_ms": {k: round(v, 4) for k, v in stages.items()},
        "e2e": {"value": round(e2e_ms, 4), "unit": "ms", "h2d_bytes_per_step": int(xh.nbytes + lh.nbytes),
                "d2h_bytes_per_step": int(Eh.nbytes + Fh.nbytes + gh.nbytes)},
        "gpu_launches": int(launches * args.steps),
        "roofline": {"bound": "tensor", "kernel": "k_m2l_tc (+ source layout)", "achieved": round(achieved, 2) if achieved else None,
                     "peak": round(peak_tf32, 1), "unit": "TFLOP/s",
                     "frac": round(achieved / peak_tf32, 4) if achieved else None, "traffic": traffic,
                     "peak_source": f"{src} bf16 burst x {TF32_PER_BF16:.4f} (nominal tf32/bf16)",
                     "algorithmic_flop_per_launch": m2l_flop, "tensor_flop_per_launch": tensor_flop},
        "clocks": clocks,
        "wall_s_timed": round(t_wall, 3),
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(s)
        out["cpu_baseline"]["validation"] = cpu_baseline_validation()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def _time_steps(h, x, lam, E, F, g, flush, stream, steps, warmup):
    """Mean event-timed step (ms) and the median site-stage time (ms)."""
    import torch

    import paper_2410_01754_gb300 as pkg
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            pkg.mahi_eval(h, x, lam, E, F, g)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            pkg.mahi_eval(h, x, lam, E, F, g)
            ev[k][1].record(stream)
        stream.synchronize()
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        pkg.mahi_set_timing(h, True)
        site = []
        for _ in range(3):
            flush.fill_(1.0)
            pkg.mahi_eval(h, x, lam, E, F, g)
            site.append(pkg.mahi_stage_times(h).get("site", 0.0))
        pkg.mahi_set_timing(h, False)
    return ms, float(np.median(site))


def run_sweep(args):
    """Overhead of the per-site work over the plain FMM (no sites), the
    paper's sites / forms and particle-count benchmarks (Secs. "Scaling with
    Increasing Number of Sites", "Scaling with Increasing Number of Particles"):
    sites: the 1,000,002-atom water box with S = 0, 1, 8, 64, 256, 512 sites;
    atoms: water boxes of 3k to 4M atoms at the same density with one site of
    6-12 atoms per ~4,000 atoms, each against the same box without sites.
    One JSON line per point (mixed precision, p = 12, depth for ~30 atoms per
    leaf; L2 flushed between timed steps)."""
    import math

    import torch

    import paper_2410_01754_gb300 as pkg
    import synth
    from paper_2410_01754_gb300 import build as pkg_build

    pkg_build.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    spacing = 21.5 / 70  # lattice spacing of the 1M-atom box (0.307 nm)
    if args.sweep == "sites":
        pts = [(333334, S) for S in (0, 1, 8, 64, 256, 512)]
    else:
        pts = []
        for nw in (1000, 10667, 83334, 333334, 1333334):
            pts += [(nw, 0), (nw, max(1, round(3 * nw / 4000)))]
    base = {}
    for nw, S in pts:
        grid = math.ceil((nw * 1.0001) ** (1.0 / 3.0))
        while grid ** 3 < nw:
            grid += 1
        L = round(grid * spacing, 4)
        d = max(1, min(6, round(math.log(3 * nw / 30.0, 8))))
        s = synth.make_water(n_water=nw, grid=grid, L=L, n_sites=S, seed=1, depth=d, order=12)
        N = len(s["qA"])
        h = pkg.mahi_create(L, N, S, 12, d, "mixed", stream)
        pkg.mahi_set_charges(h, s["qA"], s["qB"], s["site_of"])
        x = torch.tensor(s["x"], dtype=torch.float32, device=dev)
        lam = torch.tensor(s["lam"], dtype=torch.float64, device=dev)
        E = torch.zeros(1, dtype=torch.float64, device=dev)
        F = torch.empty_like(x)
        g = torch.zeros(max(1, S), dtype=torch.float64, device=dev)
        ms, site_ms = _time_steps(h, x, lam, E, F, g, flush, stream, args.steps, args.warmup)
        pkg.mahi_destroy(h)
        if S == 0:
            base[nw] = ms
        rec = {"sweep": args.sweep, "n_atoms": N, "n_sites": S, "box_nm": L, "depth": d, "order_p": 12,
               "precision": "mixed", "ms_per_step": round(ms, 4), "site_stage_ms": round(site_ms, 4),
               "atoms_per_s": round(N / (ms * 1e-3), 1)}
        if S > 0 and nw in base:
            rec["overhead_vs_no_sites"] = round(ms / base[nw] - 1.0, 4)
        print(json.dumps(rec), flush=True)


def e1_point(s, prec, p, d, oracle_dEdl):
    """One point of the accuracy sweep: dE/dlambda of the GPU path at order p,
    depth d, against (a) the oracle (exact periodic HI) and (b) the paper's
    reference, the same path's energies of the 2^m end states (separate
    evaluations at the same p and d) combined by the multilinear
    interpolation's derivative, Eqs. "ref_two_forms" / "ref_four_forms" read
    as the derivative of Eq. "rek_ham_lambda"."""
    import torch

    import paper_2410_01754_gb300 as pkg
    N = len(s["q_env"])
    m = pkg.Mahi(s["L"], N, 1, p, d, prec)
    status = 0
    try:
        if len(s["forms"][0]) == 2:
            m.set_charges(s["qA"], s["qB"], s["site_of"])
        else:
            m.set_forms(s["q_env"], s["site_of"], s["forms"])
        xdt = torch.float64 if prec == "fp64" else torch.float32
        x = torch.tensor(s["x"], dtype=xdt, device="cuda")
        lam0 = np.asarray(s["lams"][0], dtype=np.float64)
        nl = len(lam0)
        _, _, g = m.eval(x, torch.tensor(lam0, device="cuda"))
        dEdl = g.cpu().numpy()
        status = m.status()
        H = {}
        for rho in range(1 << nl):
            corner = np.array([(rho >> l) & 1 for l in range(nl)], dtype=np.float64)
            E, _, _ = m.eval(x, torch.tensor(corner, device="cuda"))
            H[rho] = E.item()
        status = status or m.status()
    except pkg.MahiError as e:   # a device-side failure of one point is recorded, not fatal
        return {"dEdl": None, "rel_dev_vs_oracle": [float("nan")], "rel_dev_vs_same_order_fmm": [float("nan")],
                "status": e.code}
    finally:
        m.close()
    ref_same = np.zeros(nl)
    for l in range(nl):
        for rho in range(1 << nl):
            w = 1.0
            for k in range(nl):
                if k == l:
                    w *= 1.0 if (rho >> k) & 1 else -1.0
                else:
                    w *= lam0[k] if (rho >> k) & 1 else 1.0 - lam0[k]
            ref_same[l] += w * H[rho]
    return {"dEdl": dEdl.tolist(), "rel_dev_vs_oracle": (np.abs(dEdl - oracle_dEdl) / np.abs(oracle_dEdl)).tolist(),
            "rel_dev_vs_same_order_fmm": (np.abs(dEdl - ref_same) / np.abs(ref_same)).tolist(), "status": status}


def run_accuracy_sweep(args):
    """The paper's accuracy test (Sec. "Accuracy of the Random System with Two
    Forms and Four Forms", Fig. "accuracy"): 1,000 + 10 random charges, one
    site of 10 particles with 2 or 4 forms, clustered ("typical") or scattered
    ("worst") site particles, lambda = 0.345 / (0.345, 0.721); relative
    deviation of dE/dlambda for depths 0-3 and orders 2-16 in FP64 and mixed
    precision, against the oracle and against the same-order end-state energies
    (the paper's reference).  One JSON line per point."""
    from oracle import hi
    import synth
    from paper_2410_01754_gb300 import build as pkg_build

    pkg_build.build()
    for layout in ("typical", "worst"):
        for forms in (2, 4):
            s = synth.make_e1(layout, forms, 1)
            ref = hi.multiform_eval(s)["dEdl"]
            for prec, orders in (("fp64", (2, 4, 6, 8, 10, 12, 16, 20)), ("mixed", (2, 4, 6, 8, 10, 12, 15))):
                for d in (0, 1, 2, 3):
                    for p in orders:
                        r = e1_point(s, prec, p, d, ref)
                        print(json.dumps({"sweep": "accuracy", "layout": layout, "forms": forms, "precision": prec,
                                          "depth": d, "order_p": p, "oracle_dEdl": ref.tolist(), **r}), flush=True)


def run_replicas(args):
    """16 independent replicas of uneven size (48k to 250k atoms, 16 to 256
    sites, each its own box and lambdas; p = 12, d = 4, mixed precision): one
    step evaluates all of them, either as 16 mahi_eval calls or as one launch
    of the CUDA graph that mahi_batch_create captured (after mahi_autotune on
    each replica).  L2 flushed between timed steps."""
    import math

    import torch

    import paper_2410_01754_gb300 as pkg
    import synth
    from paper_2410_01754_gb300 import build as pkg_build

    pkg_build.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    spacing = 21.5 / 70
    R = 16
    reps = []
    for k in range(R):
        nw = int(round(16000 + (83334 - 16000) * ((k * 7) % R) / (R - 1)))  # uneven order of sizes
        S = int(round(16 + (256 - 16) * ((k * 5) % R) / (R - 1)))
        grid = math.ceil(nw ** (1.0 / 3.0))
        while grid ** 3 < nw:
            grid += 1
        L = round(grid * spacing, 4)
        s = synth.make_water(n_water=nw, grid=grid, L=L, n_sites=S, seed=100 + k, depth=4, order=12)
        N = len(s["qA"])
        h = pkg.mahi_create(L, N, S, 12, 4, "mixed", stream)
        pkg.mahi_set_charges(h, s["qA"], s["qB"], s["site_of"])
        x = torch.tensor(s["x"], dtype=torch.float32, device=dev)
        lam = torch.tensor(s["lam"], dtype=torch.float64, device=dev)
        out = (torch.zeros(1, dtype=torch.float64, device=dev), torch.empty_like(x),
               torch.zeros(S, dtype=torch.float64, device=dev))
        reps.append((h, x, lam, out, N, S))
    n_atoms = sum(r[4] for r in reps)

    def timed(step):
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                step()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            for k in range(args.steps):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                step()
                ev[k][1].record(stream)
            stream.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in ev]))

    def eager():
        for h, x, lam, (E, F, g), N, S in reps:
            pkg.mahi_eval(h, x, lam, E, F, g)

    t_eager = timed(eager)
    tune = []
    for h, x, lam, out, N, S in reps:
        pkg.mahi_autotune(h, x, lam, 2)
        tune.append(list(pkg.mahi_get_tuning(h)) + [int(pkg.mahi_get_option(h, "m2l_single_tile")),
                                                     int(pkg.mahi_get_option(h, "m2l_b_stages"))])
    t_tuned = timed(eager)
    batch = pkg.MahiBatch([r[0] for r in reps], stream, [r[1] for r in reps], [r[2] for r in reps],
                          [r[3][0] for r in reps], [r[3][1] for r in reps], [r[3][2] for r in reps])
    t_graph = timed(batch.launch)
    batch.close()
    for r in reps:
        pkg.mahi_destroy(r[0])
    print(json.dumps({"mode": "replicas", "replicas": R, "n_atoms_total": n_atoms,
                      "atoms": [r[4] for r in reps], "sites": [r[5] for r in reps], "order_p": 12, "depth": 4,
                      "precision": "mixed", "ms_per_step_eager": round(t_eager, 4),
                      "ms_per_step_tuned_eager": round(t_tuned, 4), "ms_per_step_graph": round(t_graph, 4),
                      "atoms_per_s_graph": round(n_atoms / (t_graph * 1e-3), 1),
                      "tuning_p2p_threads_site_blocks_m2l_single_m2l_stages": tune}), flush=True)


def cpu_baseline(s, n_targets=8192, atom_frac=1 / 8):
    """The oracle (FP64 Ewald + HI closed form) timed on the host cores on a
    bounded sample, extrapolated to one full evaluation of the workload:
    structure factors over a random fraction of the atoms (linear in atoms) and
    the real- and reciprocal-space sums at random target atoms of the full
    system (linear in targets)."""
    import oracle
    from oracle import hi
    N = len(s["qA"])
    L = s["L"]
    rc = oracle.default_rc(L, N)
    rng = np.random.default_rng(0)
    qt = hi.scaled_charges(s["qA"], s["qB"], s["site_of"], s["lam"])
    sub = rng.choice(N, int(N * atom_frac), replace=False)
    tgt = rng.choice(N, n_targets, replace=False)
    t0 = time.perf_counter()
    oracle.ewald(s["x"][sub], qt[sub], L, rc=rc, targets=np.arange(1), parts=2)   # SF(sub) + 1 target
    t_sf = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.ewald(s["x"][sub], qt[sub], L, rc=rc, targets=np.arange(n_targets), parts=2)  # SF(sub) + targets
    t_rec = max(time.perf_counter() - t0 - t_sf, 0.0)
    t0 = time.perf_counter()
    oracle.ewald(s["x"], qt, L, rc=rc, targets=tgt, parts=1)                       # real space, full density
    t_real = time.perf_counter() - t0
    full_s = t_sf / atom_frac + (t_rec + t_real) * N / n_targets
    return {"value": round(full_s * 1e3, 1), "unit": "ms", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"Ewald structure factors over {atom_frac:.4f} of the atoms plus real- and reciprocal-space "
                      f"sums at {n_targets} target atoms of the {N:,}-atom system, extrapolated linearly to "
                      f"one full E/F/dE/dlambda evaluation (rc={rc:.2f} nm); a model, checked in "
                      f"'validation' against a full evaluation of a smaller system",
            "measured_s": round(t_sf * 2 + t_rec + t_real, 2)}


def cpu_baseline_validation():
    """The sampling model of cpu_baseline checked on a system the oracle can
    evaluate in full: the 96,000-atom, 32-site water box (p = 10, d = 4
    workload).  One complete oracle evaluation (HI energy, every force, every
    dE/dlambda) is timed on the host cores, next to the model's prediction from
    the same kind of sample (an eighth of the atoms, 8,192 targets)."""
    import oracle
    import synth
    from oracle import hi
    s = synth.make("B", 1)
    t0 = time.perf_counter()
    hi.hi_eval(s)
    full = time.perf_counter() - t0
    model = cpu_baseline(s)["value"] * 1e-3
    return {"workload": "water_96k_32sites", "n_atoms": len(s["qA"]), "cores": oracle.num_threads(),
            "measured_full_s": round(full, 2), "model_s": round(model, 2),
            "model_over_measured": round(model / full, 3)}


def run_reference(args):
    """The oracle as the reference arm (there is no reference implementation)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth
    s = synth.make(WORKLOAD["config"], WORKLOAD["seed"])
    vals = []
    for k in range(args.warmup + args.steps):
        cb = cpu_baseline(s, n_targets=1024, atom_frac=1 / 64)
        if k >= args.warmup:
            vals.append(cb["value"])
    v = float(np.mean(vals))
    cb["value"] = round(v, 1)
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": "ms",
           "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(v, 1), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD["name"], "n_atoms": len(s["qA"]), "n_sites": len(s["lam"]),
                      "box_nm": s["L"]},
           "cpu_baseline": cb, "e2e": {"value": round(v, 1), "unit": "ms", "h2d_bytes_per_step": 0,
                                      "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernels-only", action="store_true",
                    help="time the mixed steps only (for profiler runs); skips stages, e2e, FP64 comparator")
    ap.add_argument("--replicas", action="store_true",
                    help="16 uneven replicas per step: eager calls vs autotuned vs one CUDA graph")
    ap.add_argument("--sweep", choices=["sites", "atoms", "accuracy"], default=None,
                    help="overhead of the per-site work over the plain FMM vs sites (1M atoms) or vs atoms; "
                         "accuracy: the paper's 1,010-particle dE/dlambda deviation sweep over depth and order")
    ap.add_argument("--case", default=WORKLOAD["config"], choices=[WORKLOAD["config"], "C_quarter"],
                    help="C_quarter: 250,002 atoms in the same box and tree (identical M2L work), for "
                         "profiler captures together with --kernels-only")
    args = ap.parse_args()
    if args.case != WORKLOAD["config"] and not args.kernels_only:
        ap.error("--case C_quarter is a profiler case: use it with --kernels-only")
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.sweep == "accuracy":
        run_accuracy_sweep(args)
    elif args.sweep:
        run_sweep(args)
    elif args.replicas:
        run_replicas(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
