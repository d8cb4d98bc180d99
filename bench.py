"""Benchmark: RTA linewidths of the Si-like 40^3 x 40^3 workload on B300.

One step = one full ``phoebe_gpu_linewidths_rta`` pass (grid band structure,
phonons, window, stage 1, stage 2 with the fused rotation/delta epilogue,
degenerate averaging) over all active states of the synthetic Si-like crystal
(8 Wannier functions, 2 atoms, 429 R_e and 429 R_p vectors, 40^3 k x 40^3 q,
T = 300 K, sigma = 0.02 eV, window +-0.5 eV), inputs already resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision P] [--impl reference]

The default mode evaluates stage 2 as a separable DFT over the R_p residues (FP32,
exact on the grid); the tensor-core stage 2 (split FP16) is timed beside it.
Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

PREC_NAMES = {0: "fp64", 1: "split_bf16", 2: "split_tf32", 3: "bf16", 4: "tf32", 5: "split_fp16", 6: "bf16x3",
              7: "fp32_grid_dft", 8: "fp64_grid_dft"}
PREC_DTYPE = {0: "f64", 1: "bf16x6+f32acc", 2: "tf32x3+f32acc", 3: "bf16+f32acc", 4: "tf32+f32acc",
              7: "f32", 8: "f64",
              5: "f16x3+f32acc", 6: "bf16x3+f32acc"}
METRIC = "Gamma_nk linewidths/s (el-ph RTA, Si-like 40^3 k x 40^3 q)"
WORKLOAD = "si_like_fcc_nw8_na2_R429_k40x40x40_q40x40x40_T300_sigma0.02_window0.5"


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_over_ranks(ms: float, units, dist, device) -> tuple:
    """Whole-job figures of a step loop run on every rank: the slowest rank's time (MAX) and the units
    all ranks processed (SUM; each rank runs its own problem instance, so the counts may differ).
    ``units`` is a sequence of counts; ``dist`` the torch.distributed module or None (one process)."""
    units = [float(u) for u in units]
    if dist is None:
        return ms, units
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor(units, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), [float(x) for x in u.tolist()]


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        power = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(power) if power else None}


def _blas_threads() -> int:
    """Threads numpy's BLAS uses (the oracle's matrix products)."""
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        if info:
            return int(max(i.get("num_threads", 1) for i in info))
    except ImportError:
        pass
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(var, "").isdigit():
            return int(os.environ[var])
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def roofline(precision: int, stats: list, k_limit: int) -> dict:
    """Roofline object of the dominant stage-2 kernel from the library's per-launch CUDA-event times."""
    peaks, peak_src = _peaks()
    s2_ms = sum(s["stage2_ms"] for s in stats)
    s2_launch = sum(s["stage2_launches"] for s in stats)
    s2_flops = sum(s["stage2_flops"] for s in stats)
    achieved = s2_flops / (s2_ms / 1e3) / 1e12 if s2_ms > 0 else None
    split_factor = {0: 1, 1: 6, 2: 3, 3: 1, 4: 1, 5: 3, 6: 3, 7: 1, 8: 1}[precision]
    kpad = (-(-2 * 429 // 64) * 64) / (2 * 429)
    if precision == 7:
        # CUDA-core FP32: 148 SMs x 128 FP32 lanes x 2 flop per FMA x the maximum SM clock
        fp32_peak = 148 * 128 * 2 * 2.032e9 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak if achieved else None, "traffic": None,
                "peak_source": "FP32 FMA rate from unit counts and the 2032 MHz maximum clock",
                "kernel": "k_dft_z + k_dft_yx_elph (stage 2 as a separable grid DFT: z sum, then the fused "
                          "y sum / windowed x sum / rotation and delta epilogue)",
                "algorithmic_flops_per_launch": s2_flops / max(s2_launch, 1),
                "avg_launch_ms": s2_ms / max(s2_launch, 1),
                "note": "flops count the DFT's complex MACs as evaluated (8 flop each; x sum only for the q "
                        "whose final bands reach the delta window) and the epilogue's two rotations (U_{k+q}^dagger: "
                        "N_w 3N_at, Z_q: (3N_at)^2 complex MACs) once per evaluated (state, q), a lower bound (99% of "
                        "the listed q have one final band); the Gaussian and occupation arithmetic is not counted"}
    elif precision in (0, 8):
        roof = {"bound": "alu", "achieved": achieved, "peak": 1.25, "unit": "TFLOP/s",
                "frac": achieved / 1.25 if achieved else None, "traffic": None,
                "peak_source": "nominal FP64 1.25 TFLOP/s",
                "kernel": "k_zgemm (dense R_p sum)" if precision == 0 else
                          "k_dft_z64 + k_dft_yx64 (FP64 separable grid DFT)",
                "algorithmic_flops_per_launch": s2_flops / max(s2_launch, 1),
                "avg_launch_ms": s2_ms / max(s2_launch, 1)}
    else:
        peak = peaks.get("bf16_tflops_sustained", 1400.0)
        if precision in (2, 4):
            peak *= 0.5     # TF32 dense rate is half the BF16 rate (nominal ratio)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None, "traffic": None,
                "peak_source": f"{peak_src} bf16_tflops_sustained" + (" x 0.5 (tf32)" if precision in (2, 4) else ""),
                "kernel": "k_tc_gemm<ElphEpi<8,6>> (stage 2, R_p contraction + fused epilogue)",
                "algorithmic_flops_per_launch": s2_flops / max(s2_launch, 1),
                "avg_launch_ms": s2_ms / max(s2_launch, 1),
                "issued_tensor_tflops": achieved * split_factor * kpad if achieved else None,
                "issued_frac": achieved * split_factor * kpad / peak if achieved else None}
    # DRAM bytes of one captured launch, scaled by algorithmic flop (the units processed) to this
    # run's average launch
    traffic_path = os.path.join(ROOT, "profiles", "stage2_traffic.txt")
    prefix = {5: "tc_capture_", 7: "dft_capture_"}.get(precision)
    if prefix and os.path.exists(traffic_path) and k_limit == 0 and s2_launch:
        vals = {}
        with open(traffic_path) as f:
            for ln in f:
                if ln.startswith(prefix) and "=" in ln:
                    k, v = ln.strip().split("=", 1)
                    vals[k[len(prefix):]] = float(v)
        if "bytes" in vals and vals.get("flops"):
            roof["traffic"] = vals["bytes"] * (s2_flops / s2_launch) / vals["flops"]
    return roof


def cpu_baseline_oracle(n_k: int, seed: int = 0) -> dict:
    """The FP64 oracle as it stands, on a bounded sample of the workload (n_k active k points)."""
    from oracle import elph
    from workloads import synthetic as W
    mat, prm = W.si_like(seed=seed)
    t0 = time.perf_counter()
    tab = elph.electron_table(mat, prm)
    eg = tab[1][tab[3]]
    ks, _ = elph.active_states(eg, prm.mu_eV, prm.window_eV)
    pick = np.sort(np.random.default_rng(seed).choice(np.unique(ks), n_k, replace=False))
    k2, b2, g = elph.linewidths_rta(mat, prm, k_indices=pick, table=tab)
    el = time.perf_counter() - t0
    threads = _blas_threads()
    return {"value": len(g) / el, "unit": "linewidths/s", "cores": int(threads), "kind": "oracle",
            "sample": f"{len(g)} active states on {n_k} seeded k points of the Si-like 40^3 x 40^3 workload, "
                      f"including the oracle's own band structure on the 40^3 grid ({el:.1f} s)",
            "seconds": el, "states": int(len(g))}


def learned_leg(pg, W, dev, stream, args) -> dict:
    """Learned q proposal: trained on the q terms of a Si-like 20^3 full-grid run, evaluated on
    40^3 k x 80^3 q (a seeded subset of k) at 5% of q against the full q sum of the same
    precision; the uniform proposal and the FP64 full sum (a smaller sample) beside it."""
    import torch
    prec = args.precision if args.precision not in (0, 7) else 5   # sampled q sums run on the tensor-core modes
    ctx = pg.PhoebeGPU(dev, stream=stream)
    ctx.set_profiling(True)
    mat20, p20 = W.si_like(seed=0, nk=20)
    ctx.set_material(mat20)
    ctx.sampler_init(1)
    t0 = time.perf_counter()
    loss = ctx.sampler_train(p20.with_(precision=prec), **({"epochs": args.learned_epochs} if args.learned_epochs else {}))
    train_s = time.perf_counter() - t0
    mat, prm = W.si_like(seed=0, nk=40, nq=80)
    ctx.set_material(mat)
    kk = np.sort(np.random.default_rng(2).choice(64000, args.learned_k, replace=False))
    pe = prm.with_(precision=prec, k_subset=kk)

    def timed(p):
        torch.cuda.synchronize()
        t = time.perf_counter()
        out = ctx.linewidths_rta(p)
        torch.cuda.synchronize()
        return out, time.perf_counter() - t, ctx.stats()
    timed(pe)                                     # warm-up (allocations, 80^3 tables)
    (_, _, full), full_s, full_st = timed(pe)
    res = {}
    for name, smp in (("learned", 1), ("shell", 3), ("uniform", 2)):
        errs, walls, st = [], [], None
        for seed in range(4):
            (_, _, g), w, st = timed(pe.with_(sampler=smp, sample_fraction=0.05, seed=seed))
            errs.append(float(np.linalg.norm(g - full) / np.linalg.norm(full)))
            walls.append(w)
        res[name] = {"l2_rel_err": errs, "wall_s": float(np.median(walls)),
                     "sampler_ms": st["sampler_ms"], "pairs_ms": st["stage2_ms"], "total_ms": st["total_ms"]}
    n = len(full)
    # the full q sum by the separable grid DFT in FP32 (the benchmarked mode) on the same states
    p7 = prm.with_(precision=7, k_subset=kk)
    timed(p7)
    (_, _, g7), w7, st7 = timed(p7)
    f64k = kk[:6]
    (_, _, g64), w64, st64 = timed(prm.with_(precision=0, k_subset=f64k))
    ctx.close()
    lw = n / res["learned"]["wall_s"]
    return {
        "workload": "si_like 40^3 k x 80^3 q, seeded subset of k; trained on the si_like 20^3 x 20^3 q terms",
        "states": int(n), "sample_fraction": 0.05, "mix_alpha": 0.1, "precision": PREC_NAMES[prec],
        "train_s": train_s, "train_loss_first_last": [float(loss[0]), float(loss[-1])],
        "proposal": "(1 - alpha) softmax(z + log phi) + alpha phi / sum phi, phi the shell factor (the bracket of "
                    "Eq. 29 with |g|^2 replaced by 1/(hbar w))",
        "l2_rel_err_learned": res["learned"]["l2_rel_err"], "l2_rel_err_shell_only": res["shell"]["l2_rel_err"],
        "l2_rel_err_uniform": res["uniform"]["l2_rel_err"],
        "variance_ratio_uniform_over_learned": float(np.mean(np.square(res["uniform"]["l2_rel_err"])) /
                                                     np.mean(np.square(res["learned"]["l2_rel_err"]))),
        "variance_ratio_shell_only_over_learned": float(np.mean(np.square(res["shell"]["l2_rel_err"])) /
                                                        np.mean(np.square(res["learned"]["l2_rel_err"]))),
        "gate_l2_1pct_met": bool(np.mean(res["learned"]["l2_rel_err"]) <= 0.01),
        "linewidths_per_s_shell_only": n / res["shell"]["wall_s"],
        "linewidths_per_s_learned": lw, "linewidths_per_s_full_same_precision": n / full_s,
        "linewidths_per_s_full_fp32_grid_dft": len(g7) / w7,
        "max_rel_diff_fp32_grid_dft_vs_full_same_precision": float(np.max(np.abs(g7 - full) / np.abs(full))),
        "linewidths_per_s_fp64_gpu_full": len(g64) / w64,
        "speedup_learned_vs_fp64_gpu": lw / (len(g64) / w64),
        "learned_ms": {"network_proposal_draws": res["learned"]["sampler_ms"], "sampled_pairs": res["learned"]["pairs_ms"],
                       "total": res["learned"]["total_ms"]},
        "full_ms": {"stage2": full_st["stage2_ms"], "total": full_st["total_ms"]},
        "full_fp32_grid_dft_ms": {"stage2": st7["stage2_ms"], "total": st7["total_ms"]},
    }


def mlp_leg(pg, dev, n_states: int = 49, n: int = 80, reps: int = 4) -> dict:
    """The proposal network's tensor-core scoring alone: every q of an n^3 grid for n_states seeded
    feature rows, randomly initialised parameters; device time of the scoring by CUDA events (the
    fastest of reps calls after a warm-up)."""
    ctx = pg.PhoebeGPU(dev)
    ctx.sampler_init(1)
    rng = np.random.default_rng(3)
    feat = np.column_stack([rng.uniform(-0.5, 0.5, n_states), rng.normal(0, 1.5, (n_states, 3))]).astype(np.float32)
    ctx.set_profiling(True)
    ctx.mlp_scores(feat, (n, n, n), tensor_cores=True)
    times = []
    for _ in range(reps):
        ctx.mlp_scores(feat, (n, n, n), tensor_cores=True)
        times.append(ctx.stats()["sampler_ms"])
    best = min(times)
    ctx.close()
    rows = n_states * n ** 3
    return {"rows": rows, "ms": best, "rows_per_s": rows / (best / 1e3),
            "network_tflops": rows * 2.0 * (2 * 128 * 128 + 8 * 128 + 128) / (best / 1e3) / 1e12,
            "workload": f"{n_states} seeded feature rows x every q of {n}^3, tensor-core scoring"}


def prate_leg(pg, ctx, prm, mat, ms_linewidths: float) -> dict:
    """Phonon-electron rates P_{q nu} (Sec. 4.3) of the same Si-like workload: one call runs the whole
    linewidth pipeline with the rate accumulated in the grid-DFT epilogue; timed against the
    linewidth step alone."""
    import torch
    p7 = pg.make_params(prm, precision=7)
    nm = 3 * mat.na
    P = ctx.phonon_rates_elph(p7, nm)                   # warm-up
    torch.cuda.synchronize()
    reps = 3
    t0 = time.perf_counter()
    for _ in range(reps):
        P = ctx.phonon_rates_elph(p7, nm)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / reps
    return {"workload": "si_like 40^3 k x 40^3 q, every (q, nu) of the q grid", "values": int(P.size),
            "ms_per_call": ms, "ms_linewidths_only": ms_linewidths,
            "overhead_vs_linewidths": ms / ms_linewidths - 1.0, "unit": "host-timed call incl. download of P",
            "max_P_eV": float(np.max(P)), "nonzero_fraction": float(np.mean(P > 0))}


def adaptive_leg(pg, ctx, prm, ms_linewidths: float, n_states: int) -> dict:
    """The same linewidth step with adaptive Gaussian smearing (Sec. 4.7): a width per pair of states
    from the band velocities at k and k+q (floor 1e-3 eV); host-timed calls."""
    import torch
    pa = pg.make_params(prm, precision=7, smearing=1, sigma_min_eV=1e-3)
    ks, bs, g = ctx.linewidths_rta(pa, capacity=n_states)       # warm-up
    torch.cuda.synchronize()
    reps = 3
    t0 = time.perf_counter()
    for _ in range(reps):
        ks, bs, g = ctx.linewidths_rta(pa, capacity=n_states)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / reps
    st = ctx.stats()
    return {"workload": "si_like 40^3 k x 40^3 q, adaptive widths", "ms_per_call": ms,
            "linewidths_per_s": len(g) / (ms / 1e3), "ms_fixed_width_step": ms_linewidths,
            "pairs_evaluated_fraction": st["pairs_executed"] / max(st["pairs_dense"], 1),
            "unit": "host-timed call incl. download of Gamma", "median_gamma_eV": float(np.median(g))}


def three_phonon_leg(pg, W, dev) -> dict:
    """Three-phonon diagonal of the phonon scattering matrix (Sec. 3.1 V3 interpolation, Sec. 4.3)
    for every (q, nu) of a 16^3 grid of the Si-like two-atom crystal (169 (R, R') pairs, 13 R');
    host-timed calls, the stage-2 kernel timed by CUDA events inside the library."""
    import torch
    mat, anh, prm = W.three_phonon_si_like(seed=0, nq=16)
    with pg.PhoebeGPU(dev) as c:
        c.set_material(mat)
        c.set_force_constants3(anh)
        c.set_profiling(True)
        p3 = pg.make_params(prm)
        A = c.three_phonon_rates(p3, 6)                  # warm-up
        torch.cuda.synchronize()
        reps = 3
        t0 = time.perf_counter()
        for _ in range(reps):
            A = c.three_phonon_rates(p3, 6)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / reps
        st = c.stats()
    q = int(np.prod(prm.nq))
    return {"workload": "si_like two-atom 16^3 q grid, 169 (R, R') pairs, every (q, nu)", "q_points": q,
            "ms_per_call": ms, "mode_rates_per_s": q * 6 / (ms / 1e3),
            "stage2_ms": st["stage2_ms"], "stage2_tflops": st["stage2_flops"] / (st["stage2_ms"] / 1e3) / 1e12,
            "unit": "host-timed call incl. phonons and download", "max_A_eV": float(np.max(A))}


def batch_leg(pg, W, dev, args) -> dict:
    """64 uneven materials (N_w 4-24, 1-6 atoms, |R| 100-1200, grids 16^3-40^3, a seeded subset of k
    per material, split BF16): one call per material against one batch call whose stage 2 for all
    materials is a single CUDA graph with autotuned tiles."""
    import torch
    t0 = time.perf_counter()
    mats = [W.batch_material(i, g_budget_bytes=128e6) for i in range(64)]
    gen_s = time.perf_counter() - t0
    ctxs, jobs = [], []
    for i, (mat, prm) in enumerate(mats):
        c = pg.PhoebeGPU(dev)
        c.set_material(mat)
        n = prm.nk[0]
        kk = np.sort(np.random.default_rng([5, i]).choice(n ** 3, min(args.batch_k, n ** 3), replace=False))
        ctxs.append(c)
        jobs.append((c, pg.make_params(prm, precision=1, k_subset=kk)))
    caps = [c.count_states(p) for c, p in jobs]
    for (c, p), cap in zip(jobs, caps):          # warm-up
        c.linewidths_rta(p, capacity=cap)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    eager = [c.linewidths_rta(p, capacity=cap) for (c, p), cap in zip(jobs, caps)]
    torch.cuda.synchronize()
    eager_s = time.perf_counter() - t0
    for c, p in jobs:
        c.set_profiling(True)
    agg = {}
    for (c, p), cap in zip(jobs, caps):          # per-stage breakdown (not timed as a whole)
        c.linewidths_rta(p, capacity=cap)
        st = c.stats()
        for key in ("bands_ms", "phonons_ms", "stage1_ms", "stage2_ms", "delta_ms", "stage2_flops"):
            agg[key] = agg.get(key, 0.0) + st[key]
    for c, p in jobs:
        c.set_profiling(False)
    t0 = time.perf_counter()
    _, info0 = pg.binding.linewidths_rta_batch(jobs, capacities=caps)   # warm-up; the autotuner times here
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    res, info = pg.binding.linewidths_rta_batch(jobs, capacities=caps)  # tiles reused from the first call
    torch.cuda.synchronize()
    batch_s = time.perf_counter() - t0
    states = int(sum(len(g) for _, _, g in eager))
    diff = 0.0
    for (_, _, g), (_, _, g1) in zip(res, eager):
        if len(g) and np.any(g1):
            diff = max(diff, float(np.max(np.abs(g - g1) / np.maximum(np.abs(g1), 1e-6 * np.median(np.abs(g1))))))
    for c in ctxs:
        c.close()
    tiles = {}
    for t in info["tiles"]:
        tiles[f"{t[0]}x{t[1]}"] = tiles.get(f"{t[0]}x{t[1]}", 0) + 1
    return {
        "workload": f"64 batch materials (seed 0), {args.batch_k} seeded k each, full q grids, split_bf16",
        "states": states, "generation_s": gen_s,
        "one_call_per_material": {"wall_s": eager_s, "linewidths_per_s": states / eager_s},
        "one_batch_call": {"wall_s": batch_s, "linewidths_per_s": states / batch_s, "plan_ms": info["plan_ms"],
                           "graph_ms": info["graph_ms"], "graph_nodes": info["graph_nodes"],
                           "finish_ms": info["finish_ms"], "graph_reused": info["graph_reused"],
                           "note": "tiles chosen by the first call, reused"},
        "first_batch_call_with_autotuning": {"wall_s": first_s, "linewidths_per_s": states / first_s,
                                             "plan_ms": info0["plan_ms"], "graph_reused": info0["graph_reused"]},
        "per_material_stage_ms_sum": {k: v for k, v in agg.items() if k.endswith("_ms")},
        "stage2_algorithmic_tflops_in_graph": agg["stage2_flops"] / (info["graph_ms"] / 1e3) / 1e12,
        "autotuned_tiles_columns_x_kblocks": tiles,
        "max_rel_diff_batch_vs_per_material": diff,
    }


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    steps, warmup = args.steps, args.warmup
    from oracle import elph
    from workloads import synthetic as W
    mat, prm = W.si_like(seed=0)
    tab = elph.electron_table(mat, prm)
    eg = tab[1][tab[3]]
    ks, _ = elph.active_states(eg, prm.mu_eV, prm.window_eV)
    uk = np.unique(ks)
    rng = np.random.default_rng(1)
    per_step_k = max(1, args.ref_k_per_step)
    for _ in range(warmup):
        elph.linewidths_rta(mat, prm, k_indices=np.sort(rng.choice(uk, per_step_k, replace=False)), table=tab)
    n_states = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        _, _, g = elph.linewidths_rta(mat, prm, k_indices=np.sort(rng.choice(uk, per_step_k, replace=False)),
                                      table=tab)
        n_states += len(g)
    el = time.perf_counter() - t0
    threads = _blas_threads()
    value = n_states / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "linewidths/s", "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": 1e3 * el / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_per_step": f"{per_step_k} seeded active k points (all their states)",
                   "precision": "fp64 (CPU oracle)"},
        "cpu_baseline": {"value": value, "unit": "linewidths/s", "cores": int(threads), "kind": "oracle",
                         "sample": f"{n_states} states over {steps} steps of {per_step_k} k points each; "
                                   "grid band structure precomputed once outside the timed steps"},
        "e2e": {"value": value, "unit": "linewidths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", type=int, default=7,
                    help="0 fp64, 1 split bf16, 2 split tf32, 5 split fp16 (tensor cores), 7 fp32 grid DFT, 8 fp64 grid DFT")
    ap.add_argument("--no-tc-leg", action="store_true", help="skip the tensor-core stage-2 legs beside the headline")
    ap.add_argument("--no-fp64-dft", action="store_true", help="skip the FP64 grid-DFT leg")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-k-per-step", type=int, default=2)
    ap.add_argument("--cpu-k", type=int, default=4, help="k points of the CPU-oracle baseline sample")
    ap.add_argument("--fp64-k", type=int, default=48, help="k points of the FP64 GPU comparison sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--k-limit", type=int, default=0,
                    help="profiling case: restrict to this many seeded active k points (0 = whole grid)")
    ap.add_argument("--k-planes", type=int, default=0,
                    help="profiling case: restrict to the active k of the first N kx planes of the k grid")
    ap.add_argument("--main-only", action="store_true", help="only the timed device leg (for ncu captures)")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-proposal leg")
    ap.add_argument("--no-batch", action="store_true", help="skip the many-materials leg")
    ap.add_argument("--no-prate", action="store_true", help="skip the phonon-electron rate leg")
    ap.add_argument("--learned-only", action="store_true", help="only the learned-proposal leg (profiling case)")
    ap.add_argument("--batch-only", action="store_true", help="only the many-materials leg (profiling case)")
    ap.add_argument("--mlp-only", action="store_true", help="only the proposal network's scoring rate (profiling case)")
    ap.add_argument("--learned-epochs", type=int, default=0, help="training epochs of the learned leg (0: default)")
    ap.add_argument("--batch-k", type=int, default=64, help="seeded k points per material in the many-materials leg")
    ap.add_argument("--learned-k", type=int, default=512, help="seeded k points of the learned-proposal evaluation")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2111_14999_b300 as pg
    from workloads import synthetic as W

    world, rank, local = _dist()
    if args.learned_only:
        dev = local if torch.cuda.is_available() else 0
        torch.cuda.set_device(dev)
        if rank == 0:
            print(json.dumps({"learned_sampler": learned_leg(pg, W, dev, torch.cuda.current_stream(), args)}), flush=True)
        return
    if args.mlp_only:
        dev = local if torch.cuda.is_available() else 0
        torch.cuda.set_device(dev)
        if rank == 0:
            print(json.dumps({"mlp_network": mlp_leg(pg, dev)}), flush=True)
        return
    if args.batch_only:
        dev = local if torch.cuda.is_available() else 0
        torch.cuda.set_device(dev)
        if rank == 0:
            print(json.dumps({"batched_materials": batch_leg(pg, W, dev, args)}), flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as td
        td.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        dist = td
    dev = local if torch.cuda.is_available() else 0
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()

    mat, prm = W.si_like(seed=rank)   # independent problem instance per rank (weak scaling)
    ctx = pg.PhoebeGPU(dev, stream=stream)
    ctx.set_material(mat)
    params = pg.make_params(prm, precision=args.precision)
    if args.k_limit > 0:
        kgrid = np.arange(prm.nk[0] * prm.nk[1] * prm.nk[2])
        pick = np.sort(np.random.default_rng(11).choice(kgrid, args.k_limit, replace=False))
        params = pg.make_params(prm, precision=args.precision, k_subset=pick)
    if args.k_planes > 0:
        pick = np.arange(args.k_planes * prm.nk[1] * prm.nk[2])
        params = pg.make_params(prm, precision=args.precision, k_subset=pick)
    n = ctx.count_states(params)
    k_out = torch.empty(n, dtype=torch.int32, device="cuda")
    b_out = torch.empty(n, dtype=torch.int32, device="cuda")
    g_out = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx.set_profiling(True)
    for _ in range(args.warmup):
        ctx.linewidths_rta_dev(params, k_out, b_out, g_out, n)
    torch.cuda.synchronize()

    sampler = ClockSampler(dev)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    e0.record(stream)
    for _ in range(args.steps):
        ctx.linewidths_rta_dev(params, k_out, b_out, g_out, n)
        stats.append(ctx.stats())
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    ms, (states_tot, coup_tot, coup_dense_tot) = reduce_over_ranks(
        ms, (n * args.steps, stats[-1]["couplings_executed"] * args.steps, stats[-1]["couplings_dense"] * args.steps),
        dist, "cuda")
    ms_per_step = ms / args.steps
    value = states_tot / (ms / 1e3)
    couplings = coup_tot / (ms / 1e3)
    couplings_dense = coup_dense_tot / (ms / 1e3)
    launches = int(sum(s["kernel_launches"] for s in stats))

    roof = roofline(args.precision, stats, args.k_limit or args.k_planes)
    if args.precision == 7 and roof.get("achieved") and clocks.get("sm_mhz") and clocks.get("sm_max_mhz"):
        # the FP32 peak scales with the SM clock: the fraction against the peak at the timed region's
        # median clock, beside the one at the maximum clock
        peak_med = roof["peak"] * clocks["sm_mhz"] / clocks["sm_max_mhz"]
        roof["peak_at_median_clock"] = peak_med
        roof["frac_at_median_clock"] = roof["achieved"] / peak_med
    if args.precision == 7 and roof.get("achieved"):
        # the FP32 FMA rate measured on this GPU by the library's probe (8 independent FMA chains per
        # thread, 8 blocks per SM), beside the rate from unit counts
        tf, tms = ctx.fp32_rate()
        roof["peak_measured_fp32_fma"] = tf
        roof["frac_of_measured_fp32_fma"] = roof["achieved"] / tf if tf > 0 else None
        roof["fp32_fma_probe_ms"] = tms

    extra = {}
    g_head = g_out.cpu().numpy().copy()
    ks_head = k_out.cpu().numpy().copy()

    def device_leg(prec, steps):
        """The same full step in another precision: one untimed call, then `steps` timed calls."""
        pp = pg.make_params(prm, precision=prec)
        ctx.linewidths_rta_dev(pp, k_out, b_out, g_out, n)
        torch.cuda.synchronize()
        sx = []
        t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0e.record(stream)
        for _ in range(steps):
            ctx.linewidths_rta_dev(pp, k_out, b_out, g_out, n)
            sx.append(ctx.stats())
        t1e.record(stream)
        torch.cuda.synchronize()
        msx = t0e.elapsed_time(t1e) / steps
        return msx, sx, g_out.cpu().numpy().copy()

    legs = {}
    if not args.main_only and not args.no_tc_leg:
        # the tensor-core stage 2 in each split precision on the same workload
        for prec in (5, 1, 2):
            if prec == args.precision:
                continue
            msx, sx, gx = device_leg(prec, min(args.steps, 3))
            fl = 1e-6 * np.median(np.abs(gx))
            legs[prec] = {
                "precision": PREC_NAMES[prec], "value": n / (msx / 1e3), "unit": "linewidths/s", "ms_per_step": msx,
                "roofline": roofline(prec, sx, args.k_limit or args.k_planes),
                "max_rel_diff_vs_headline": float(np.max(np.abs(gx - g_head) / np.maximum(np.abs(gx), fl))),
                "_g": gx}
        ctx.linewidths_rta_dev(params, k_out, b_out, g_out, n)     # headline outputs back for the checks below
        torch.cuda.synchronize()
    if args.main_only:
        line = {"metric": METRIC, "value": value, "unit": "linewidths/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "states_per_step": n, "roofline": roof,
                "gpu_launches": launches, "clocks": clocks, "note": "main leg only (profiling case)"}
        if rank == 0:
            print(json.dumps(line), flush=True)
        ctx.close()
        return
    # FP64 on the GPU: the dense R_p sum (every q, k_zgemm) on a sample of k, and the FP64 separable grid
    # DFT (the headline's algorithm in FP64) on the whole step; errors of every precision against FP64
    if rank == 0 and args.fp64_k > 0:
        uk = np.unique(ks_head)
        pick = np.sort(np.random.default_rng(5).choice(uk, min(args.fp64_k, len(uk)), replace=False))
        ctx.set_profiling(True)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        k64, b64, g64 = ctx.linewidths_rta(prm, precision=0, k_subset=pick)
        t1.record(stream)
        torch.cuda.synchronize()
        fp64_ms = t0.elapsed_time(t1)
        st64 = ctx.stats()
        sel = np.isin(ks_head, pick)
        floor = 1e-6 * np.median(np.abs(g64))

        def err_vs_fp64(g_all):
            return float(np.max(np.abs(g_all[sel] - g64) / np.maximum(np.abs(g64), floor)))
        fp64_rate = len(g64) / (fp64_ms / 1e3)
        extra["fp64_gpu"] = {"value": fp64_rate, "unit": "linewidths/s", "algorithm": "dense R_p sum over every q",
                             "sample": f"{len(g64)} states on {len(pick)} seeded k points",
                             "stage2_tflops": st64["stage2_flops"] / st64["stage2_ms"] / 1e9 if st64["stage2_ms"] else None}
        extra["speedup_vs_fp64_gpu"] = (value / world) / fp64_rate
        extra["max_rel_err_vs_fp64"] = err_vs_fp64(g_head)
        if args.precision != 8 and not args.no_fp64_dft:
            ms8, s8, g8 = device_leg(8, 1)
            extra["fp64_grid_dft"] = {
                "value": n / (ms8 / 1e3), "unit": "linewidths/s", "ms_per_step": ms8,
                "algorithm": "the headline's separable grid DFT in FP64 (precision 8), whole step",
                "roofline": roofline(8, s8, args.k_limit or args.k_planes),
                "max_rel_err_vs_fp64_dense": err_vs_fp64(g8)}
            fl8 = 1e-6 * np.median(np.abs(g8))
            extra["speedup_vs_fp64_grid_dft"] = (value / world) / (n / (ms8 / 1e3))
            extra["max_rel_err_vs_fp64_grid_dft"] = float(np.max(np.abs(g_head - g8) / np.maximum(np.abs(g8), fl8)))
            ctx.linewidths_rta_dev(params, k_out, b_out, g_out, n)
            torch.cuda.synchronize()
        for prec, leg in legs.items():
            leg["max_rel_err_vs_fp64"] = err_vs_fp64(leg["_g"])
    for prec, leg in legs.items():
        leg.pop("_g")
    if 5 in legs:
        extra["tensor_core_mode"] = legs.pop(5)
    if legs:
        extra["split_precision_legs"] = list(legs.values())

    # end to end through the public host-buffer API, inputs from pinned host memory every step
    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory() if a.dtype != np.complex128 else \
            torch.from_numpy(np.ascontiguousarray(a).view(np.float64)).pin_memory()
        return t
    pin = {name: pinned(getattr(mat, name)) for name in ("R_H", "w_H", "H", "mass_amu", "R_fc", "w_fc", "Phi",
                                                       "Re", "we", "Rp", "wp", "g")}
    h2d = int(sum(t.numel() * t.element_size() for t in pin.values()))
    lib = pg.lib
    import ctypes as C

    def e2e_step():
        c = ctx._ctx
        ctx._check(lib.phoebe_gpu_set_hamiltonian(c, mat.nw, len(mat.R_H), C.c_void_p(pin["R_H"].data_ptr()),
                                                  C.c_void_p(pin["w_H"].data_ptr()), C.c_void_p(pin["H"].data_ptr())))
        ctx._check(lib.phoebe_gpu_set_force_constants(c, mat.na, C.c_void_p(pin["mass_amu"].data_ptr()),
                                                      len(mat.R_fc), C.c_void_p(pin["R_fc"].data_ptr()),
                                                      C.c_void_p(pin["w_fc"].data_ptr()),
                                                      C.c_void_p(pin["Phi"].data_ptr())))
        ctx._check(lib.phoebe_gpu_set_elph_wannier(c, len(mat.Re), C.c_void_p(pin["Re"].data_ptr()),
                                                   C.c_void_p(pin["we"].data_ptr()), len(mat.Rp),
                                                   C.c_void_p(pin["Rp"].data_ptr()), C.c_void_p(pin["wp"].data_ptr()),
                                                   C.c_void_p(pin["g"].data_ptr())))
        return ctx.linewidths_rta(params)
    e2e_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        kk, bb, gg = e2e_step()
    el = time.perf_counter() - t0
    d2h = int(len(gg) * (8 + 4 + 4))
    el_ms, (e2e_units,) = reduce_over_ranks(el * 1e3, (len(gg) * args.steps,), dist, "cuda")
    e2e_value = e2e_units / (el_ms / 1e3)

    line = {
        "metric": METRIC, "value": value, "unit": "linewidths/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": PREC_DTYPE[args.precision], "data": "synthetic",
        "config": {"workload": WORKLOAD, "states_per_step": n, "q_points": 64000,
                   "precision": PREC_NAMES[args.precision],
                   "l2": ("inputs larger than L2 (g in FP32: 0.57 GB read per kx plane; X rows and Zs of a "
                          "batch: several GB)") if args.precision == 7 else
                         "inputs larger than L2 (stage-1 operand from g: 1.2 GB, q-phase operand 0.23 GB)",
                   "parallelism": f"{world} independent instance(s), one per GPU"},
        "couplings_per_s": couplings,
        "couplings_per_s_note": ("complex g_{m'n nu}(k,q) elements computed per second: (state, q) pairs whose "
                                 "contraction ran (the q whose final bands reach the delta window) x N_w x 3N_at"),
        "couplings_dense_equivalent_per_s": couplings_dense,
        "gpu_launches": launches,
        "roofline": roof,
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "linewidths/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        **extra,
    }
    if rank == 0 and args.precision == 7 and not args.no_prate:
        line["phonon_rates"] = prate_leg(pg, ctx, prm, mat, ms_per_step)
    if rank == 0 and args.precision == 7 and not args.no_prate:
        line["adaptive_smearing"] = adaptive_leg(pg, ctx, prm, ms_per_step, n)
    if rank == 0 and not args.no_prate:
        line["three_phonon"] = three_phonon_leg(pg, W, dev)
    if rank == 0 and not args.no_learned:
        line["learned_sampler"] = learned_leg(pg, W, dev, stream, args)
    if rank == 0 and not args.no_batch:
        line["batched_materials"] = batch_leg(pg, W, dev, args)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_oracle(args.cpu_k)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
