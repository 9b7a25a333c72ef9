"""Benchmark of the GB300 average-spectrum sampler (blocked modes sampling).

Workload: the blocked-modes problem -- fermionic kernel, beta = 20,
N_tau = 100, N_omega = 400 on a Gaussian-density grid (sigma 3) on [-8, 8],
levels {global, 8 blocks of 50}, correlated noise 1e-4 exp(-|dtau|/0.5),
1024 chains, 1000 burn-in + 10^4 sweeps per step.  Synthetic inputs from
paper_1912_01379_gb300.workloads (seeded).

One step = one asm_sample call over the whole workload (burn-in included) in
the mixed FP32/FP64 path.  `value` = chain-mode updates per second
(chains x sweeps x N_omega per step, burn-in included) with the inputs resident
on the device; `e2e` runs asm_setup from host arrays + asm_sample + asm_average
(device->host results) per step.  The plain FP64 path and ESS/s of <A(omega)> (ESS from the binned Monte Carlo error, minimum over the grid)
are reported beside it, and, as side measurements outside the timed region,
the batching workload (256 uneven problems in one handle), the grid-size
sweep (N_omega 250..2000, 8192 chains), each in both paths, and ESS/s of the
blocked-modes problem under four partition schemes (modes, components, the
workload's two levels, the full hierarchy), and the paper's own test case
(optical conductivity on Matsubara data) on its uniform and non-uniform grids.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1912_01379_gb300 import replicas  # noqa: E402
from paper_1912_01379_gb300 import workloads as W  # noqa: E402

METRIC = "chain-mode updates/s and ESS/s of <A(omega)>: mixed-prec vs plain FP64, 1 GB300"
UNIT = "chain-mode updates/s"
WORKLOAD = "blocked_modes_fermionic_b20_Ntau100_Nomega400_gauss3_8x50_1024chains"
L2_FLUSH_BYTES = 512 << 20


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--burn", type=int, default=1000)
    ap.add_argument("--sweeps", type=int, default=10000)
    ap.add_argument("--chains", type=int, default=1024)
    ap.add_argument("--fp64-sweeps", type=int, default=10000,
                    help="kept sweeps of the plain FP64 leg (burn-in in the headline's proportion)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="heuristic launch shape instead of asm_tune's")
    ap.add_argument("--batch-sweeps", type=int, default=256,
                    help="sweeps of the batching side measurement (0: skip)")
    ap.add_argument("--largest-sweeps", type=int, default=1000,
                    help="kept sweeps of the largest-configuration timed line (0: skip)")
    ap.add_argument("--largest-burn", type=int, default=200)
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-ASM FP64 line")
    ap.add_argument("--grid-sweeps", type=int, default=64,
                    help="sweeps per N_omega of the grid-size side measurement (0: skip)")
    ap.add_argument("--paper-sweeps", type=int, default=5000,
                    help="sweeps per grid of the paper-test-case side measurement (0: skip)")
    ap.add_argument("--hierarchy-sweeps", type=int, default=3000,
                    help="sweeps per partition scheme of the hierarchy side measurement (0: skip)")
    ap.add_argument("--diff-sweeps", type=int, default=2000,
                    help="kept sweeps per run of the differentiation side measurement (0: skip)")
    ap.add_argument("--diff-budget-s", type=float, default=30.0,
                    help="time budget of the differentiation side measurement (seconds)")
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    lrank = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, lrank


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                smax.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 4 + k and r[4 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _level_sequence(seed, n_sweeps, n_levels, problem_id=0):
    """Levels drawn by the sampler (Philox4x64-10 word 0 of ctr {2^64-1, s, 0, p}).
    numpy's Philox adds one to its counter before each block."""
    out = np.empty(n_sweeps, dtype=np.int64)
    key = np.array([seed, 0], dtype=np.uint64)
    for s in range(n_sweeps):
        bg = np.random.Philox(key=key, counter=np.array([2**64 - 2, s, 0, problem_id], dtype=np.uint64))
        w = int(bg.random_raw(1)[0])
        u = ((w >> 12) + 0.5) * 2.0 ** -52
        out[s] = min(int(u * n_levels), n_levels - 1)
    return out


def _ops_per_level(p):
    """Algorithmic work per chain and sweep at every level, as two arrays:
    pass elements (n_b elements per move, n_b moves per block: update FMA,
    clamp, bound product and two bound minima per element, counted as 6 FP32
    lane operations as the method states them, Sec. IV.B) and the FMAs of the
    block's entry and exit projections (2 M min(M, n_b), Sec. IV.D)."""
    elems, fmas = [], []
    for starts in p.levels:
        ends = list(starts[1:]) + [p.N]
        e_tot, f_tot = 0, 0
        for s, e in zip(starts, ends):
            n = int(e - s)
            e_tot += n * n
            f_tot += 2 * p.M * min(p.M, n)
        elems.append(e_tot)
        fmas.append(f_tot)
    return np.array(elems, dtype=np.float64), np.array(fmas, dtype=np.float64)


OPS_PER_ELEMENT = 6


def measured_ceilings(asm):
    """Rates of the chain kernel's instruction mixes on this GPU
    (asm_measure_ceiling): the fused pass (elements/s) and the FMA alone, in
    FP32 and FP64, each with the SM clock seen during its launch."""
    out = {}
    for k in ("pass_f32", "pass_f32_smem", "ffma", "fmnmx", "imnmx", "pass_f64", "pass_f64_smem", "dfma",
              "dmnmx", "i64mnmx"):
        out[k] = asm.measure_ceiling(k, 40.0)
    return out


def roofline(elems, fmas, kernel_s, ceil, prec):
    """Achieved and peak algorithmic lane operations per second of the chain
    kernel: work = 6 per pass element + 1 per projection FMA; the peak is the
    time the same work takes at the measured rates of the pass mix and of the
    FMA alone (register operands), i.e. a weighted harmonic mean of the two."""
    pk, fk = ("pass_f32", "ffma") if prec == "f32" else ("pass_f64", "dfma")
    ops = OPS_PER_ELEMENT * elems + fmas
    t_min = elems / ceil[pk]["rate"] + fmas / ceil[fk]["rate"]
    peak = ops / t_min / 1e12
    achieved = ops / kernel_s / 1e12 if kernel_s > 0 else None
    return achieved, peak


def _captured_traffic():
    """DRAM bytes per sweep-kernel launch from the committed ncu summary of this
    workload, or None when the kernel source has changed since that capture."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", "sweep_kernel_f32_blocked_modes.md")
    src = os.path.join(ROOT, "paper_1912_01379_gb300", "csrc", "asm_sweep.cuh")
    try:
        fields = dict(l.split(":", 1) for l in open(prof).read().splitlines() if ":" in l and " " not in l.split(":")[0])
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if fields.get("kernel_source_sha256", "").strip() == sha:
            return int(fields["dram_bytes_per_launch"].strip())
    except (OSError, ValueError, KeyError):
        pass
    return None


def cpu_baseline(p, seconds_target=12.0):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of
    the same workload: chains x sweeps from the same initial state."""
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    op = O.OracleProblem(p.K, p.G, p.C, p.levels)
    chains = cores
    t0 = time.perf_counter()
    op.run(chains, 0, 2, seed=5, threads=cores)
    dt = max(time.perf_counter() - t0, 1e-3)
    sweeps = int(max(2, min(400, 2 * seconds_target / dt)))
    t0 = time.perf_counter()
    op.run(chains, 0, sweeps, seed=6, threads=cores)
    dt = time.perf_counter() - t0
    upd = chains * sweeps * p.N
    return {"value": upd / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{chains} chains x {sweeps} sweeps of the same workload (FP64 oracle, OpenMP over chains)",
            "seconds": dt}


def _spec(p):
    return dict(K=p.K, G=p.G, C=p.C, levels=p.levels, w=p.w)


def _timed(torch, stream, fn):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def batch_side(args, asm, torch, stream):
    """Batching workload (256 problems with uneven N_omega, N_tau and blocks, 64
    chains each) in one handle: persistent launches replayed from the CUDA
    graph, launch shape picked by asm_tune; mixed path and plain FP64 path."""
    probs = W.batch_problems()
    chains = probs[0].chains
    b = asm.Batch([_spec(p) for p in probs])
    sumN = sum(p.N for p in probs)
    out = {"workload": "batch_256_problems_Nomega100-1000_Ntau50-200_64chains", "problems": len(probs),
           "chains_per_problem": chains, "sweeps": args.batch_sweeps}
    for prec, key, sweeps in ((asm.ASM_MIXED, "mixed", args.batch_sweeps),
                              (asm.ASM_FP64, "fp64", max(64, args.batch_sweeps // 4))):
        b.tune(chains, precision=prec)
        b.sample(chains, 0, 1, 11, precision=prec)   # warm-up launch
        t = _timed(torch, stream, lambda: b.sample(chains, 0, sweeps, 12, precision=prec))
        st = b.status()
        out[key] = {"updates_per_s": chains * sweeps * sumN / t, "seconds": t, "sweeps": sweeps,
                    "team_lanes": st["team_lanes"], "consumers_per_cta": st["consumers_per_cta"],
                    "ctas_per_sm_budget": st["min_blocks"],
                    "ctas": st["ctas"], "work_items": st["work_items"], "graph_replays": st["graph_replays"],
                    "timeouts": st["timeouts"]}
    out["speedup_mixed_vs_fp64"] = out["mixed"]["updates_per_s"] / out["fp64"]["updates_per_s"]
    return out


def grid_side(args, asm, torch, stream):
    """Grid-size sweep (N_tau = 400, beta = 50, 16 blocks, 8192 chains) at
    N_omega in {250, 500, 1000, 2000}: mixed path (tensor-core refresh) and
    plain FP64 path rates over one refresh period, each with the launch shape
    asm_tune picks."""
    rows = []
    for N in (250, 500, 1000, 2000):
        p = W.grid_sweep_problem(N, "uniform")
        gp = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
        chains = p.chains
        row = {"N_omega": N, "N_tau": p.M, "chains": chains}
        for prec, key, sweeps in ((asm.ASM_MIXED, "mixed", args.grid_sweeps),
                                  (asm.ASM_FP64, "fp64", max(2, args.grid_sweeps // 8))):
            gp.tune(chains, precision=prec)
            gp.sample(chains, 0, 1, 21, precision=prec)
            t = _timed(torch, stream, lambda: gp.sample(chains, 0, sweeps, 22, precision=prec))
            st = gp.status()
            row[key] = {"updates_per_s": chains * sweeps * N / t, "sweeps": sweeps,
                        "tc_refreshes": st["tc_refreshes"], "timeouts": st["timeouts"],
                        "shape": {"team_lanes": st["team_lanes"], "consumers_per_cta": st["consumers_per_cta"],
                                  "ctas_per_sm_budget": st["min_blocks"]}}
        row["speedup_mixed_vs_fp64"] = row["mixed"]["updates_per_s"] / row["fp64"]["updates_per_s"]
        rows.append(row)
        del gp
    return {"workload": "grid_sweep_fermionic_b50_Ntau400_uniform_16blocks_8192chains", "rows": rows}


def largest_side(args, asm, torch, stream, ceil):
    """The largest single-GPU configuration of the grid-size sweep (N_tau = 400,
    N_omega = 2000 uniform on [-10, 10], 16 blocks, 8192 chains, noise
    1e-5 e^{-|dtau|}) as a full timed line in the mixed path: updates/s,
    ESS/s (binned error, min over the grid), the sweep kernel's roofline
    against the measured ceilings, and end to end from host arrays
    (asm_setup + asm_sample + asm_average per step)."""
    p = W.grid_sweep_problem(2000, "uniform")
    chains, burn, sweeps = p.chains, args.largest_burn, args.largest_sweeps
    gp = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
    tuned = gp.tune(chains)
    gp.sample(chains, 0, 64, 51)
    seed = 52
    t = _timed(torch, stream, lambda: gp.sample(chains, burn, sweeps, seed, timing=True))
    st = gp.status()
    ess = gp.mc_error()["ess"]
    elems, fmas = _ops_per_level(p)
    lv = _level_sequence(seed, burn + sweeps, len(p.levels))
    achieved, peak = roofline(chains * float(np.sum(elems[lv])), chains * float(np.sum(fmas[lv])),
                              st["sweep_kernel_ms"] / 1e3, ceil, "f32")
    upd = chains * (burn + sweeps) * p.N
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    q = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
    q.sample(chains, burn, sweeps, seed + 1)
    q.average()
    torch.cuda.synchronize()
    te = time.perf_counter() - t0
    del q
    return {"workload": "grid_sweep_fermionic_b50_Ntau400_Nomega2000_uniform_16blocks_8192chains",
            "chains": chains, "burn_in": burn, "sweeps": sweeps, "updates_per_s": upd / t, "seconds": t,
            "ess_min": float(np.nanmin(ess)), "ess_per_s": float(np.nanmin(ess)) / t,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T lane-op/s",
                         "frac": achieved / peak if achieved else None, "kernel": "sweep_kernel<float>",
                         "avg_launch_ms": st["sweep_kernel_ms"] / max(st["timed_launches"], 1)},
            "e2e": {"value": upd / te, "unit": UNIT,
                    "h2d_bytes_per_step": int(sum(a.nbytes for a in (p.K, p.G, p.C, p.w))),
                    "d2h_bytes_per_step": int(4 * p.N * 8)},
            "launch_shape": {"tuned": tuned, "team_lanes": st["team_lanes"],
                             "consumers_per_cta": st["consumers_per_cta"], "ctas": st["ctas"]}}


def plain_side(args, asm, torch, stream):
    """The plain-ASM workload (fermionic, beta = 10, N_tau = 20, N_omega = 50,
    global modes only, 16 chains, 1000 burn-in + 10^4 sweeps) in the plain FP64
    path, with its binned ESS/s, beside the FP64 oracle on one host core on a
    bounded sample of the same workload (the per-core rate)."""
    from oracle import oracle as O
    p = W.plain_modes_problem()
    chains, burn, sweeps = p.chains, p.burn_in, p.sweeps
    gp = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
    gp.sample(chains, 0, 64, 61, precision=asm.ASM_FP64)
    t = _timed(torch, stream, lambda: gp.sample(chains, burn, sweeps, 62, precision=asm.ASM_FP64))
    ess = gp.mc_error()["ess"]
    op = O.OracleProblem(p.K, p.G, p.C, p.levels)
    t0 = time.perf_counter()
    op.run(chains, 0, 400, seed=63, threads=1)
    t1 = time.perf_counter() - t0
    return {"workload": "plain_modes_fermionic_b10_Ntau20_Nomega50_16chains", "chains": chains,
            "burn_in": burn, "sweeps": sweeps, "precision": "fp64",
            "updates_per_s": chains * (burn + sweeps) * p.N / t, "seconds": t,
            "ess_min": float(np.nanmin(ess)), "ess_per_s": float(np.nanmin(ess)) / t,
            "oracle_1core": {"updates_per_s": chains * 400 * p.N / t1, "cores": 1,
                             "sample": f"{chains} chains x 400 sweeps (FP64 oracle, one thread)"}}


def hierarchy_side(args, asm, torch, stream):
    """The blocked-modes workload's problem under four partition schemes (Sec.
    IV): modes only (one block), components only (one point per block), the
    workload's {global, 8 x 50} levels, and the full hierarchy of
    asm_partition_hierarchy.  Mixed path, 1024 chains; updates/s and ESS/s
    (min over the grid) after a burn-in."""
    p = W.blocked_modes_problem()
    schemes = {"modes": [[0]], "components": [np.arange(p.N)], "global_8x50": p.levels,
               "hierarchy": asm.partition_hierarchy(p.N)}
    chains, burn, sweeps = 1024, 500, args.hierarchy_sweeps
    out = {"workload": WORKLOAD, "chains": chains, "burn_in": burn, "sweeps": sweeps}
    for name, levels in schemes.items():
        gp = asm.Problem(p.K, p.G, p.C, levels, w=p.w)
        gp.sample(chains, 0, 1, 31)
        t = _timed(torch, stream, lambda: gp.sample(chains, burn, sweeps, 32))
        r = gp.mc_error()                      # binned error (catches drifts all chains share)
        rc = gp.average()                      # spread of the chain means only
        out[name] = {"levels": len(levels), "blocks": int(sum(len(l) for l in levels)),
                     "updates_per_s": chains * (burn + sweeps) * p.N / t,
                     "ess_min": float(np.nanmin(r["ess"])), "ess_median": float(np.nanmedian(r["ess"])),
                     "ess_per_s": float(np.nanmin(r["ess"])) / t,
                     "ess_min_chain_spread": float(np.nanmin(rc["ess"]))}
        del gp
    return out


def diff_side(args, asm, torch, stream):
    """Differentiation workload (N_tau = 64, N_omega = 200 on the grid of an
    8-parameter Gaussian-mixture density on [-6, 6], beta = 16, noise 1e-4,
    4096 chains, global level plus 8 blocks of 25): mixed-precision sampling
    with the snapshot moments, then the vector-Jacobian products of <A> with
    respect to G and the 8 grid parameters (asm_backward).  Independent runs
    (seeds) are added until the relative standard error of the mean of each
    product is at most 2.5e-4 (the workload's stopping rule), or the time
    budget is spent."""
    p = W.theta_problem()
    chains, burn, sweeps = p.chains, 500, args.diff_sweeps
    gp = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w, dK_dtheta=p.extra["dK_dtheta"],
                     dw_dtheta=p.extra["dw_dtheta"])
    v = np.random.default_rng(7).standard_normal(p.N)
    t_sample, t_back, gG, gT = [], [], [], []

    def rel_sem(x):
        x = np.array(x)
        return float(np.linalg.norm(x.std(axis=0, ddof=1) / np.sqrt(len(x))) / np.linalg.norm(x.mean(axis=0)))

    target, t0 = 2.5e-4, time.perf_counter()
    while True:
        r = len(gG)
        t_sample.append(_timed(torch, stream, lambda: gp.sample(chains, burn, sweeps, 100 + r,
                                                                precision=asm.ASM_MIXED, moments=True)))
        tb = time.perf_counter()
        g, t = gp.backward(v)
        t_back.append(time.perf_counter() - tb)
        gG.append(g)
        gT.append(t)
        done = len(gG) >= 3 and rel_sem(gG) <= target and rel_sem(gT) <= target
        if done or time.perf_counter() - t0 > args.diff_budget_s:
            break
    return {"workload": "differentiation_b16_Ntau64_Nomega200_theta8_4096chains", "chains": chains,
            "burn_in": burn, "sweeps": sweeps, "runs": len(gG), "target_rel_sem": target,
            "converged": bool(done), "seconds": time.perf_counter() - t0,
            "updates_per_s": chains * (burn + sweeps) * p.N / float(np.mean(t_sample)),
            "backward_ms": 1e3 * float(np.mean(t_back)),
            "grad_G_rel_sem": rel_sem(gG), "grad_theta_rel_sem": rel_sem(gT),
            "grad_theta": np.mean(gT, axis=0).tolist()}


def paper_side(args, asm, torch, stream):
    """The paper's own test case (optical conductivity model 2, accurate data,
    60 bosonic Matsubara frequencies, beta = 15) over the full partition
    hierarchy: uniform grids d_omega = 0.25 with N = 32, 64, 128, 256 (cutoff 8 ...
    64) and the Gaussian, exponential and Lorentzian grids of N = 64.  Mixed
    path, 1024 chains; updates/s, binned ESS/s, the seconds to an ESS of 1000
    at every grid point (burn-in included), and the largest <sigma(omega)> beyond
    omega = 8, where the spectrum is essentially zero (the paper finds spurious
    peaks there as the uniform grid's cutoff grows)."""
    from paper_1912_01379_gb300 import default_model
    cases = [("uniform", n, None) for n in (32, 64, 128, 256)] + [(g, 64, None) for g in
                                                                 ("gaussian", "exponential", "lorentzian")]
    # the Gaussian grid whose default model fits the data best (Sec. VI)
    p0 = W.paper_problem(2, 1e-3, "gaussian", 64)
    alpha, _ = default_model.fit_grid_density("gaussian", p0.extra["omega_m"], p0.G)
    cases.append(("gaussian", 64, alpha))
    chains, burn, sweeps = 1024, 500, args.paper_sweeps
    rows = []
    for grid, N, param in cases:
        p = W.paper_problem(2, 1e-3, grid, N, grid_param=param)
        gp = asm.Problem(p.K, p.G, p.C, asm.partition_hierarchy(N), w=p.w)
        gp.sample(chains, 0, 1, 41)
        t = _timed(torch, stream, lambda: gp.sample(chains, burn, sweeps, 42))
        e = gp.mc_error()
        a = gp.average()
        ess = float(np.nanmin(e["ess"]))
        tail = p.omega > 8.0
        rows.append({"grid": grid, "N": N, "grid_param": param, "omega_max": float(p.omega[-1] + 0.5 * p.w[-1]),
                     "updates_per_s": chains * (burn + sweeps) * N / t, "seconds": t, "ess_min": ess,
                     "seconds_to_ess_1000": t * 1000.0 / ess if ess > 0 else None,
                     "max_sigma_beyond_8": float(a["mean_A"][tail].max()) if tail.any() else None})
        del gp
    # Fig. MCsteps: step sizes Delta_s = |f(s+1) - f(s)| / |f(s)| of components, modes and
    # blocked modes sampling on model 1 (accurate data, omega_n = 0.1 (n - 1/2), N = 40 and 120)
    steps = []
    for N in (40, 120):
        p = W.paper_problem(1, 1e-3, "uniform", N, d_omega=0.1)
        row = {"N": N, "cutoff": 0.1 * N}
        for name, lev in (("components", [np.arange(N)]), ("modes", [[0]]),
                          ("blocked_modes", asm.partition_hierarchy(N))):
            gp = asm.Problem(p.K, p.G, p.C, lev, w=p.w)
            gp.sample(chains, 0, 400, 43, step_trace=True)
            d = gp.step_trace()[100:]
            row[name] = {"mean_step": float(d.mean()), "median_step": float(np.median(d))}
            del gp
        steps.append(row)
    return {"workload": "optical_conductivity_model2_noise1e-3_beta15_60matsubara_hierarchy", "chains": chains,
            "burn_in": burn, "sweeps": sweeps, "rows": rows,
            "mc_steps": {"workload": "optical_conductivity_model1_noise1e-3_uniform_0.1", "sweeps": 400,
                         "averaged_over": "sweeps 100-399, all chains", "rows": steps}}


def run_reference(args):
    """--impl reference: the CPU oracle is the reference arm for this method."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    p = W.blocked_modes_problem(chains=args.chains)
    for _ in range(args.warmup):
        cpu_baseline(p, seconds_target=2.0)
    vals, secs = [], 0.0
    last = None
    for _ in range(args.steps):
        last = cpu_baseline(p, seconds_target=6.0)
        vals.append(last["value"])
        secs += last["seconds"]
    v = float(np.mean(vals))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD},
        "cpu_baseline": {"kind": "oracle", "cores": last["cores"], "sample": last["sample"], "value": v,
                         "unit": UNIT},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    from paper_1912_01379_gb300 import asm
    ws, rank, lrank = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(lrank)
    dev = torch.cuda.current_device()

    p = W.blocked_modes_problem(chains=args.chains)
    gp = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
    chains, burn, sweeps = args.chains, args.burn, args.sweeps
    # replicas: every rank samples its own `chains` chains, keyed by global chain id
    gp.set_stream_ids(0, rank * chains)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    seed_base = 1000

    # launch shape: the autotuner's pick for this workload (set-up, untimed)
    tuned = gp.tune(chains) if not args.no_tune else None
    # warm-up (untimed), full steps
    for w in range(args.warmup):
        gp.sample(chains, burn, sweeps if w == args.warmup - 1 else max(sweeps // 10, 64), seed_base + w)
    torch.cuda.synchronize()

    # timed region: K steps, L2 flushed between steps, CUDA events per step
    elems_lvl, fmas_lvl = _ops_per_level(p)
    clk = ClockSampler(dev)
    clk.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    step_ms, sweep_ms, sweep_launches, other_launches, elems_total, fmas_total = [], 0.0, 0, 0, 0.0, 0.0
    ess_min = []
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        seed = seed_base + 100 + k
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gp.sample(chains, burn, sweeps, seed, timing=True)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        st = gp.status()
        sweep_ms += st["sweep_kernel_ms"]
        sweep_launches += st["timed_launches"]
        other_launches += st["other_launches"]
        r = gp.average()
        ess = gp.mc_error()["ess"]   # binned Monte Carlo error
        if ws > 1:   # the one exchange of the replicas: FP64 sums across ranks
            r = replicas.combine(replicas.partial_from_average(r["mean_fbar"], r["sem_fbar"], r["ess"], chains))
            e = torch.tensor(ess, device="cuda", dtype=torch.float64)
            torch.distributed.all_reduce(e)   # independent replicas: their ESS add
            ess = e.cpu().numpy()
        ess_min.append(float(np.nanmin(ess)))
        lv = _level_sequence(seed, burn + sweeps, len(p.levels))
        elems_total += chains * float(np.sum(elems_lvl[lv]))
        fmas_total += chains * float(np.sum(fmas_lvl[lv]))
    torch.cuda.synchronize()
    t_local = sum(step_ms) / 1e3
    if ws > 1:
        t = torch.tensor([t_local], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_max = float(t.item())
    else:
        t_max = t_local
    clocks = clk.stop()
    updates_per_step = chains * (burn + sweeps) * p.N
    value = ws * args.steps * updates_per_step / t_max
    ms_per_step = 1e3 * t_max / args.steps
    ess_per_s = float(np.mean(ess_min)) / (ms_per_step / 1e3)

    # dominant kernel roofline: algorithmic lane operations against the measured
    # rates of the kernel's own instruction mix (ALU/issue-bound path)
    ceil = measured_ceilings(asm)
    achieved, peak = roofline(elems_total, fmas_total, sweep_ms / 1e3, ceil, "f32")

    # plain FP64 path, same workload; at the default length the same run as a mixed step, so
    # that its binned ESS (and ESS/s) is estimated from as many sweeps as the mixed path's
    fp64 = None
    if args.fp64_sweeps > 0:
        f64s = args.fp64_sweeps
        gp.sample(chains, 0, 64, seed_base + 999, precision=asm.ASM_FP64)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        seed64, burn64 = seed_base + 1000, max(1, (args.burn * f64s) // max(args.sweeps, 1))
        e0.record(stream)
        gp.sample(chains, burn64, f64s, seed64, precision=asm.ASM_FP64, timing=True)
        e1.record(stream)
        e1.synchronize()
        t64 = e0.elapsed_time(e1) / 1e3
        st64 = gp.status()
        r64 = gp.mc_error()
        upd64 = chains * (f64s + burn64) * p.N
        lv64 = _level_sequence(seed64, burn64 + f64s, len(p.levels))
        a64, pk64 = roofline(chains * float(np.sum(elems_lvl[lv64])), chains * float(np.sum(fmas_lvl[lv64])),
                             st64["sweep_kernel_ms"] / 1e3, ceil, "f64")
        fp64 = {"updates_per_s": upd64 / t64, "ess_per_s": float(np.nanmin(r64["ess"])) / t64,
                "sweeps": f64s, "burn_in": burn64,
                "roofline": {"bound": "alu", "achieved": a64, "peak": pk64, "unit": "T lane-op/s",
                             "frac": a64 / pk64 if a64 else None,
                             "peak_source": "measured: FP64 pass mix and DFMA (asm_measure_ceiling)",
                             "kernel": "sweep_kernel<double>",
                             "avg_launch_ms": st64["sweep_kernel_ms"] / max(st64["timed_launches"], 1)}}

    # end to end through the C ABI from host buffers
    e2e = None
    if not args.no_e2e:
        h2d = sum(a.nbytes for a in (p.K, p.G, p.C, p.w)) + sum(np.asarray(l).nbytes for l in p.levels)
        d2h = 4 * p.N * 8
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nst = max(1, args.steps)
        for k in range(nst):
            q = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
            q.sample(chains, burn, sweeps, seed_base + 200 + k)
            q.average()
            del q
        torch.cuda.synchronize()
        te = (time.perf_counter() - t0) / nst
        e2e = {"value": ws * updates_per_step / te, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": nst}

    batch = batch_side(args, asm, torch, stream) if (args.batch_sweeps > 0 and rank == 0) else None
    grid = grid_side(args, asm, torch, stream) if (args.grid_sweeps > 0 and rank == 0) else None
    largest = largest_side(args, asm, torch, stream, ceil) if (args.largest_sweeps > 0 and rank == 0) else None
    plain = plain_side(args, asm, torch, stream) if (not args.no_plain and rank == 0) else None
    hier = hierarchy_side(args, asm, torch, stream) if (args.hierarchy_sweeps > 0 and rank == 0) else None
    paper = paper_side(args, asm, torch, stream) if (args.paper_sweeps > 0 and rank == 0) else None
    diff = diff_side(args, asm, torch, stream) if (args.diff_sweeps > 0 and rank == 0) else None

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(p)
        cpu.pop("seconds", None)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "chains_per_gpu": chains, "burn_in": burn, "sweeps": sweeps,
                       "N_omega": p.N, "N_tau": p.M, "levels": "global + 8x50", "precision": "mixed FP32/FP64",
                       "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)"},
            "ess_per_s": ess_per_s,
            "fp64": fp64,
            "speedup_vs_fp64": (value / ws) / fp64["updates_per_s"] if fp64 else None,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T lane-op/s",
                         "frac": (achieved / peak) if achieved else None, "traffic": _captured_traffic(),
                         "traffic_unit": "DRAM bytes per launch (ncu capture, profiles/)",
                         "peak_source": "measured: FP32 pass mix and FFMA on this GPU (asm_measure_ceiling, "
                                        "register operands), weighted by the workload's pass and projection work",
                         "kernel": "sweep_kernel<float>", "avg_launch_ms": sweep_ms / max(sweep_launches, 1),
                         "work": {"pass_elements": elems_total, "projection_fmas": fmas_total,
                                  "lane_ops_per_element": OPS_PER_ELEMENT}},
            "ceilings": {k: {"rate": v["rate"], "sm_mhz": v["sm_mhz"]} for k, v in ceil.items()},
            "launch_shape": {"tuned": tuned, "team_lanes": st["team_lanes"],
                             "consumers_per_cta": st["consumers_per_cta"], "ctas": st["ctas"],
                             "ctas_per_sm_budget": st["min_blocks"]},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "batch": batch,
            "grid_sweep": grid,
            "largest_config": largest,
            "plain_asm_fp64": plain,
            "partition_schemes": hier,
            "paper_test_case": paper,
            "differentiation": diff,
            "gpu_launches": int(sweep_launches + other_launches + args.steps),
            "clocks": clocks,
        }
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
