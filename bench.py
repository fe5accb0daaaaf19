"""Benchmark of the Einstein-MSD hot path on one 2D graphene sheet.

Workload (the large FP64 MSD case): a periodic sheet of 1024 x 512 rectangular
4-atom cells (N = 2048 x 1024 = 2,097,152 sites), 0.5 % random vacancies, 4
random-phase complex128 vectors per GPU, M = 3000 Chebyshev moments per
correlation time, time step dt = 2 hbar/gamma0 (tau = 6.3, Bessel series cut at
|J_m| < 1e-15, N_p = 28).  One benchmark step is one correlation time of
Algorithm 3: xi <- U(dt)xi + [X,U(dt)]psi, psi <- U(dt)psi (Eq. 44), then the M
moments of xi (Algorithm 5).  K steps = one kg_msd call with N_c = K + 1 (t_0 is
free: [X, U(0)] = 0).  The working set (8 vector blocks of 134 MB) exceeds L2.

Metric: Chebyshev site-updates/s executed, one update = one (site, vector, recursion
step) that a kernel performs (the moment loop runs M/2 doubling steps; the
propagator runs one step per Bessel term on the chains U(dt)xi, U(dt)psi and
[X, U(dt)]psi), over all GPUs.  The paper's algorithms do more recursion steps for
the same result (per vector M - 1 moment steps and 4 (N_p - 1) propagator steps);
that count over the same time is reported beside it as
paper_equivalent_site_updates_per_s, a time-to-solution figure.

The roofline denominator of the FP64 step, the device's FP64 FMA rate, is measured in
the run (kg_fp64_fma_rate) before the timed region.  The line also carries a
complex64 record: the same K correlation times with complex64 recursion vectors
(FP64 moments and sums), its time, and the relative error of its sigma^E1(E, t) on
201 energies against the timed FP64 run's.

--impl reference times the CPU oracle on the host cores on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import kg_inputs as ki  # noqa: E402

TOL = 1e-15
# name -> (cells, vacancy concentration, vectors per GPU, moments, dt, precision)
WORKLOADS = {
    "msd-sheet-2048x1024-vac0.5pct-R4-M3000-dt2": ((1024, 512), 0.005, 4, 3000, 2.0, "f64"),
    "msd-sheet-4096x2048-vac1pct-R8-M6000-dt2-c64": ((2048, 1024), 0.01, 8, 6000, 2.0, "c64"),
    "msd-sheet-2048x1024-vac1pct-R8-M3000-dt2-c64": ((1024, 512), 0.01, 8, 3000, 2.0, "c64"),
}
DEFAULT_WORKLOAD = "msd-sheet-2048x1024-vac0.5pct-R4-M3000-dt2"
BATCHED_WORKLOAD = "dos-zgnr16-uneven-anderson-R64-M2000-batched"
SURROGATE_WORKLOAD = "surrogate-mlp-3x256x4-bf16-batch1M"
SMALL_WORKLOAD = "vac-sheet-64x64-vac1pct-R1-M512-Nc10-dt1"
CELLS, VAC, R, M, DT, PREC = WORKLOADS[DEFAULT_WORKLOAD]
METRIC = "Chebyshev site-updates/s and HBM GB/s vs peak; σ(E,t) time at 1e-5 err vs FP64"
UNIT = "site-updates/s"
FP64_NOMINAL_TFLOPS = 1.25   # nominal GB300 FP64 (profiling recipe table), for context only
# FP64 work of one doubling-KPM site-vector update on the DP pipe: the recursion
# y = c (a + b + d) - z costs 3 FMA per real component, 6 FMA = 12 flops per complex item.
# The two inner products per item are double-float sums on the FP32 pipe.
KPM_FP64_FLOPS_PER_ITEM = 12
CONFIG_NAME = DEFAULT_WORKLOAD


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def paper_work_per_step(n_sites: int, n_vec: int, n_moments: int, n_p: int) -> float:
    return float(n_sites) * n_vec * ((n_moments - 1) + 4 * (n_p - 1))


KPM_SOURCES = ("kg_kernels.cu", "kg_dot.cuh")


def _profiled_traffic(kernel_files, profile: str, n_sites: int = 0):
    """DRAM bytes per launch from a committed ncu summary, or None when the kernel
    sources (hashed in the given order, concatenated) changed since the counters
    were taken.  A summary captured on a smaller lattice states its
    ``sites_per_launch:``; its traffic is scaled to ``n_sites`` (the step's traffic is
    proportional to the site count at a fixed vector count)."""
    import hashlib
    try:
        src = b"".join(open(os.path.join(ROOT, "paper_1307_0288_gb300", "csrc", f), "rb").read()
                       for f in kernel_files)
        text = open(os.path.join(ROOT, "profiles", profile)).read()
    except OSError:
        return None
    sha = hashlib.sha256(src).hexdigest()[:16]
    fields = dict(line.split(":", 1) for line in text.splitlines()
                  if line.startswith(("kernel_source_sha256_16:", "traffic_bytes_per_launch:",
                                      "sites_per_launch:")))
    if fields.get("kernel_source_sha256_16", "").strip() != sha:
        return None
    try:
        traffic = int(fields["traffic_bytes_per_launch"].strip())
        if "sites_per_launch" in fields and n_sites:
            traffic = int(round(traffic * n_sites / int(fields["sites_per_launch"].strip())))
        return traffic
    except (KeyError, ValueError):
        return None


def fp64_peak_tflops(kg):
    """FP64 peak measured in this run: the library's FMA probe (best of 5 launches),
    2 flops per FMA."""
    return 2.0 * kg.fp64_fma_rate(5) / 1e12


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle legs

def oracle_step_sample(n_moments: int, with_evolution: bool):
    """One correlation time of Algorithm 3 for one vector on the full sheet, run by
    the oracle as it stands (single host thread).  Returns (paper work, seconds)."""
    import oracle
    w = ki.sheet_cells(*CELLS, vacancy_conc=VAC)
    ho = oracle.from_workload(w)
    phi = w.vectors(1)[:, 0]
    tau = oracle.tau_of(ho, DT)
    n_p = oracle.bessel_terms(tau, TOL)
    t0 = time.perf_counter()
    if with_evolution:
        xi0 = np.zeros_like(phi)
        xi = oracle.evolve(ho, xi0, tau, +1) + oracle.evolvex(ho, phi, tau)
        _ = oracle.evolve(ho, phi, tau, +1)
    else:
        xi = phi
    oracle.kpm_moments(ho, xi, xi, n_moments)
    dt = time.perf_counter() - t0
    work = float(w.n_sites) * ((n_moments - 1) + (4 * (n_p - 1) if with_evolution else 0))
    return work, dt


def _all_cores_worker(n_moments, vector_seed, barrier, queue):
    """One process of the all-cores oracle timing: its own random vector on the full
    sheet, then n_moments of Algorithm 5 started together with the other processes."""
    import oracle
    w = ki.sheet_cells(*CELLS, vacancy_conc=VAC, vector_seed=vector_seed)
    ho = oracle.from_workload(w)
    phi = w.vectors(1)[:, 0]
    barrier.wait(timeout=900)
    t0 = time.time()
    oracle.kpm_moments(ho, phi, phi, n_moments)
    t1 = time.time()
    queue.put((float(w.n_sites) * (n_moments - 1), t0, t1))


def cpu_baseline_all_cores(n_moments: int = 200):
    """The oracle as it stands on every host core: one spawned process per core, each
    with its own vector (random vectors are independent units of the method); the value
    is the processes' total work over the wall time from the first start to the last
    finish."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    n = max(1, min(n, 72))
    barrier, queue = ctx.Barrier(n), ctx.Queue()
    procs = [ctx.Process(target=_all_cores_worker, args=(n_moments, 5000 + i, barrier, queue))
             for i in range(n)]
    for p in procs:
        p.start()
    res = [queue.get(timeout=1800) for _ in range(n)]
    for p in procs:
        p.join(timeout=60)
    work = sum(r[0] for r in res)
    wall = max(r[2] for r in res) - min(r[1] for r in res)
    return {"value": work / wall, "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": f"{n} processes, each {n_moments} moments of Algorithm 5 for its own vector on the "
                      f"full 2,097,152-site sheet; {wall:.1f} s wall"}


def cpu_baseline():
    work, sec = oracle_step_sample(400, True)
    line = {"value": work / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "one MSD correlation time (U(dt)xi, [X,U(dt)]psi, U(dt)psi, N_p=28) + 400 "
                      "moments, 1 vector, full 2,097,152-site sheet; oracle single-threaded C; "
                      f"{sec:.1f} s"}
    line["all_cores"] = cpu_baseline_all_cores()
    return line


def run_reference(args):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return
    n_mom = 32   # each step: one 32-moment recursion on the full sheet, one vector
    for _ in range(args.warmup):
        oracle_step_sample(n_mom, False)
    total_w, total_s = 0.0, 0.0
    for _ in range(args.steps):
        wk, s = oracle_step_sample(n_mom, False)
        total_w += wk
        total_s += s
    value = total_w / total_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": CONFIG_NAME, "sites": 2 * CELLS[0] * 2 * CELLS[1]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "per step: 32-moment Chebyshev recursion (Algorithm 5), "
                                       "1 vector, full 2,097,152-site sheet, single host thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm

def run_ours(args):
    import torch
    import paper_1307_0288_gb300 as kg

    rank, world = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_1307_0288_gb300 import replicas
    w = ki.sheet_cells(*CELLS, vacancy_conc=VAC, vector_seed=replicas.rank_vector_seed(1000, rank, R),
                       n_vec=R)
    stream = torch.cuda.Stream()
    h = kg.from_workload(w, stream=stream)
    n_p = len(kg.bessel_series(h.emax_ev * DT / w.gamma0_ev, TOL))
    phi_host = torch.from_numpy(w.vectors(R)).pin_memory()
    phi_dev = phi_host.to("cuda")
    K, W = args.steps, args.warmup
    prec = kg.KG_C64 if PREC == "c64" else kg.KG_FP64

    fp64_peak = fp64_peak_tflops(kg)

    # warm-up: W correlation times
    out_w = torch.zeros((R, W + 1, M), dtype=torch.complex128, device="cuda")
    kg.msd(h, phi_dev, M, W + 1, DT, bessel_tol=TOL, out=out_w, precision=prec)
    torch.cuda.synchronize()

    # timed region (device-resident inputs and outputs)
    out = torch.zeros((R, K + 1, M), dtype=torch.complex128, device="cuda")
    kg.timing_enable(h, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    e0.record(stream)
    kg.msd(h, phi_dev, M, K + 1, DT, bessel_tol=TOL, out=out, precision=prec)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop() if clocks else None
    ms = e0.elapsed_time(e1)
    cnt = kg.timing_read(h)
    kg.timing_enable(h, False)
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    # end to end: host (pinned) input and output through the same public call
    out_host = torch.zeros((R, K + 1, M), dtype=torch.complex128).pin_memory()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    kg.msd(h, phi_host, M, K + 1, DT, bessel_tol=TOL, out=out_host, precision=prec)
    e2e_s = time.perf_counter() - t0
    barrier()
    if dist is not None:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())

    # sigma^E1(E, t) on 201 energies from the timed moments (host sums, Eqs. 9 and 31)
    def sigma_e1(mu):
        en = np.linspace(-3 * w.gamma0_ev, 3 * w.gamma0_ev, 201)
        mean = mu.mean(axis=0).real
        dens = kg.kpm_sum(mean, en, h.emax_ev, h.area_nm2)
        return kg.conductivity(kg.KG_SIGMA_E1, dens, DT * kg.HBAR_EV_FS / w.gamma0_ev)

    t0 = time.perf_counter()
    sig = sigma_e1(out.cpu().numpy())
    sums_s = time.perf_counter() - t0
    sigma = {"formula": "E1 (Eq. 9)", "energies": 201, "times": K + 1,
             "time_s": ms * 1e-3 + sums_s, "host_sums_s": sums_s}
    if PREC != "f64":
        out64 = torch.zeros((R, K + 1, M), dtype=torch.complex128, device="cuda")
        t0 = time.perf_counter()
        kg.msd(h, phi_dev, M, K + 1, DT, bessel_tol=TOL, out=out64, precision=kg.KG_FP64)
        f64_s = time.perf_counter() - t0
        sig64 = sigma_e1(out64.cpu().numpy())
        sigma["rel_err_vs_fp64_gpu"] = float(np.max(np.abs(sig - sig64)) / np.max(np.abs(sig64)))
        sigma["fp64_gpu_time_s"] = f64_s + sums_s

    # complex64 record: the same K correlation times on the same inputs with complex64
    # recursion vectors, timed on the library's stream; its sigma^E1 against the FP64 one
    c64 = None
    if PREC == "f64":
        out_c = torch.zeros((R, K + 1, M), dtype=torch.complex128, device="cuda")
        warm_c = torch.zeros((R, 2, M), dtype=torch.complex128, device="cuda")
        kg.msd(h, phi_dev, M, 2, DT, bessel_tol=TOL, out=warm_c, precision=kg.KG_C64)
        torch.cuda.synchronize()
        kg.timing_enable(h, True)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        kg.msd(h, phi_dev, M, K + 1, DT, bessel_tol=TOL, out=out_c, precision=kg.KG_C64)
        c1.record(stream)
        torch.cuda.synchronize()
        c_ms = c0.elapsed_time(c1)
        ccnt = kg.timing_read(h)
        kg.timing_enable(h, False)
        t0 = time.perf_counter()
        sig_c = sigma_e1(out_c.cpu().numpy())
        c_sums_s = time.perf_counter() - t0
        c_launch_ms = ccnt["kpm_ms"] / max(ccnt["kpm_launches"], 1)
        c_bytes = w.n_sites * (12 + 3 * 8 * R)
        c_gbs = c_bytes / (c_launch_ms * 1e-3) / 1e9
        c64 = {"precision": "complex64 recursion vectors; FP64 Bessel/Jackson coefficients, moments "
                            "and time integration",
               "times": K + 1, "ms_per_step": c_ms / K, "fp64_ms_per_step": ms / K,
               "speedup_vs_fp64": ms / c_ms,
               "sigma_time_s": c_ms * 1e-3 + c_sums_s, "fp64_sigma_time_s": ms * 1e-3 + sums_s,
               "sigma_rel_err_vs_fp64_gpu": float(np.max(np.abs(sig_c - sig)) / np.max(np.abs(sig))),
               "sigma_norm": "max over 201 energies and K + 1 times of |sigma_c64 - sigma_fp64| / "
                             "max |sigma_fp64| (sigma^E1, Eq. 9)",
               "executed_site_updates_per_s": (ccnt["kpm_site_steps"] + ccnt["evolve_site_steps"]) * world
               / (c_ms * 1e-3),
               "kpm_kernel": "kpm_sym_pair_kernel<4> (complex64 doubling KPM step)",
               "kpm_avg_launch_ms": c_launch_ms, "kpm_achieved_gbs": c_gbs,
               "kpm_hbm_frac": c_gbs / _peaks().get("hbm_gbs", 6800.0),
               "kpm_algorithmic_bytes": c_bytes}

    # sanity: the moments are finite and bounded by C_0 (|T_n| <= 1)
    c = out[:, 1:].real
    ok = bool(torch.isfinite(c).all()) and bool((c.abs() <= c[..., :1] * (1 + 1e-9) + 1e-300).all())

    paper_work = paper_work_per_step(w.n_sites, R, M, n_p) * K * world
    paper_value = paper_work / (ms * 1e-3)
    executed_work = (cnt["kpm_site_steps"] + cnt["evolve_site_steps"]) * world
    value = executed_work / (ms * 1e-3)
    kpm_launch_ms = cnt["kpm_ms"] / max(cnt["kpm_launches"], 1)
    flops_per_launch = KPM_FP64_FLOPS_PER_ITEM * w.n_sites * R
    achieved_tflops = flops_per_launch / (kpm_launch_ms * 1e-3) / 1e12
    vec_b = 16 if PREC == "f64" else 8
    bytes_per_launch = w.n_sites * (12 + 3 * vec_b * R)
    achieved_gbs = bytes_per_launch / (kpm_launch_ms * 1e-3) / 1e9
    peaks = _peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "MEASURED_PEAKS.json" if "hbm_gbs" in peaks else "fallback"
    if PREC == "f64":
        roofline = {"bound": "alu", "kernel": "kpm_sym_kernel<double> (FP64 doubling KPM step, 6 DFMA per site-vector)",
                    "achieved": achieved_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": achieved_tflops / fp64_peak,
                    "traffic": _profiled_traffic(KPM_SOURCES, "kpm_sym_kernel_msd_sheet_2M.md"),
                    "algorithmic_bytes": bytes_per_launch,
                    "peak_source": "measured in-run: kg_fp64_fma_rate (8 independent FP64 FMA chains per "
                                   "thread, 4 x 256-thread CTAs per SM, best of 5 launches), 2 flops per FMA",
                    "peak_nominal": FP64_NOMINAL_TFLOPS,
                    "avg_launch_ms": kpm_launch_ms,
                    "hbm": {"achieved_gbs": achieved_gbs, "peak_gbs": hbm_peak,
                            "frac": achieved_gbs / hbm_peak, "peak_source": hbm_src}}
    else:
        roofline = {"bound": "hbm", "kernel": "kpm_sym_kernel<float> (complex64 doubling KPM step)",
                    "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved_gbs / hbm_peak,
                    "traffic": _profiled_traffic(KPM_SOURCES, "kpm_sym_kernel_c64_sheet_2M.md", w.n_sites),
                    "algorithmic_bytes": bytes_per_launch, "peak_source": hbm_src,
                    "avg_launch_ms": kpm_launch_ms}
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": PREC, "data": "synthetic",
        "value_counts": "executed (site, vector, recursion step) updates",
        "config": {"workload": CONFIG_NAME, "sites": w.n_sites, "vacancies": len(w.vacancies),
                   "vectors_per_gpu": R, "moments": M, "dt_hbar_over_gamma0": DT, "bessel_terms": n_p,
                   "l2": "inputs larger than L2 (8 vector blocks x 134 MB)",
                   "parallelism": f"replicas x{world} (independent random vectors)"},
        "roofline": roofline,
        "paper_equivalent_site_updates_per_s": paper_value,
        "paper_equivalent_note": "N R ((M - 1) + 4 (N_p - 1)) per correlation time, the recursion steps of "
                                 "Algorithms 3, 5-7 as printed, over the same time",
        "gpu_launches": int(cnt["kpm_launches"] + cnt["evolve_launches"] + cnt["other_launches"]),
        "phase_ms": {"kpm": cnt["kpm_ms"], "evolve": cnt["evolve_ms"]},
        "clocks": clk,
        "e2e": {"value": executed_work / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(phi_host.numel() * 16 / K),
                "d2h_bytes_per_step": int(out_host.numel() * 16 / K), "seconds": e2e_s},
        "sanity_bounded_moments": ok,
        "sigma": sigma,
    }
    if c64 is not None:
        line["c64"] = c64
    if world == 1 and not args.no_cpu_baseline and CONFIG_NAME == DEFAULT_WORKLOAD:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_batched(args):
    """16 uneven zigzag ribbons (widths 8..64 chains, lengths 1k..16k cells, Anderson
    W = 0.5..2 eV), 64 vectors each, M = 2000 DOS moments, all in one persistent,
    graph-captured launch.  One step = one kg_batched_dos_moments call."""
    import torch
    import paper_1307_0288_gb300 as kg

    rank, world = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1)
    torch.cuda.set_device(_env_int("LOCAL_RANK", 0))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    rv, mm = 64, 2000
    ws = ki.ribbon_set_16(n_vec=rv)
    from paper_1307_0288_gb300 import replicas
    for w in ws:
        w.vector_seed = replicas.rank_vector_seed(1000, rank, rv)
    hs = [kg.from_workload(w) for w in ws]
    phis = [torch.from_numpy(w.vectors(rv)).to("cuda") for w in ws]
    n_sites = sum(w.n_sites for w in ws)
    out = torch.zeros((len(ws), rv, mm), dtype=torch.complex128, device="cuda")
    fp64_peak = fp64_peak_tflops(kg)
    for _ in range(args.warmup):
        kg.batched_dos_moments(hs, phis, mm, out=out)
    tune = kg.batched_tuning()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    e0.record()
    for _ in range(args.steps):
        kg.batched_dos_moments(hs, phis, mm, out=out)
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    ms = e0.elapsed_time(e1)
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    # end to end from pinned host inputs to host moments
    phis_h = [p.cpu().pin_memory() for p in phis]
    out_h = torch.zeros((len(ws), rv, mm), dtype=torch.complex128).pin_memory()
    t0 = time.perf_counter()
    kg.batched_dos_moments(hs, phis_h, mm, out=out_h)
    e2e_s = time.perf_counter() - t0
    steps_per_call = (mm + 1) // 2   # first step + (M - 1) / 2 doubling steps
    work = float(n_sites) * rv * steps_per_call * args.steps * world
    paper_work = float(n_sites) * rv * (mm - 1) * args.steps * world
    step_ms = ms / args.steps / steps_per_call
    # Anderson disorder adds the on-site term e x: y = c (a + b + d) + e x - z costs 4 FMA per
    # real component, 8 DFMA = 16 flops per complex item
    flops = (KPM_FP64_FLOPS_PER_ITEM + 4) * n_sites * rv
    achieved = flops / (step_ms * 1e-3) / 1e12
    bytes_step = n_sites * (12 + 8 + 48 * rv)
    peaks = _peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    c = out.real
    ok = bool(torch.isfinite(c).all()) and bool((c.abs() <= c[..., :1] * (1 + 1e-9)).all())
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": work / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "value_counts": "executed (site, vector, recursion step) updates",
        "paper_equivalent_site_updates_per_s": paper_work / (ms * 1e-3),
        "config": {"workload": BATCHED_WORKLOAD, "instances": len(ws), "sites": n_sites,
                   "vectors_per_instance": rv, "moments": mm,
                   "l2": "inputs larger than L2 (2 x 6.9 GB vector blocks)",
                   "parallelism": f"replicas x{world} (independent random vectors)"},
        "roofline": {"bound": "alu", "kernel": "batched_kpm_kernel<64,RB> (persistent FP64 doubling KPM)",
                     "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp64_peak, "traffic": None,
                     "peak_source": "measured in-run (kg_fp64_fma_rate)",
                     "avg_step_ms": step_ms,
                     "hbm": {"achieved_gbs": bytes_step / (step_ms * 1e-3) / 1e9, "peak_gbs": hbm_peak}},
        "autotune": tune,
        "gpu_launches": 2 * args.steps,
        "clocks": clk,
        "e2e": {"value": float(n_sites) * rv * steps_per_call / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(sum(p.numel() for p in phis_h) * 16),
                "d2h_bytes_per_step": int(out_h.numel() * 16), "seconds": e2e_s},
        "sanity_bounded_moments": ok,
    }
    print(json.dumps(line), flush=True)


def run_surrogate(args):
    """Surrogate MLP (3 -> 4 x 256 GELU -> 1, BF16 tensor-core kernels): batch-1M
    inference, one step = one forward over 1,048,576 inputs; also the time of one Adam
    training step on 65,536 samples."""
    import torch
    import paper_1307_0288_gb300 as kg
    from paper_1307_0288_gb300 import surrogate

    torch.cuda.set_device(_env_int("LOCAL_RANK", 0))
    n = 1 << 20
    net = kg.Mlp(surrogate.init_params(1))
    g = torch.Generator(device="cuda").manual_seed(5)
    x = (torch.rand((n, 3), generator=g, device="cuda") * 2 - 1).contiguous()
    y = torch.zeros(n, dtype=torch.float32, device="cuda")
    # the inputs (12.6 MB) and outputs (4.2 MB) would stay in L2 from one forward to the
    # next: a 256 MB write between timed forwards (outside their events) flushes it
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        net.forward(x, out=y)
    launches0 = net.launches()
    net.timing_enable(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(torch.cuda.current_device())
    torch.cuda.synchronize()
    clocks.start()
    for e0, e1 in ev:
        flush.zero_()
        e0.record()
        net.forward(x, out=y)
        e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = sum(e0.elapsed_time(e1) for e0, e1 in ev)
    tm = net.timing_read()
    net.timing_enable(False)
    launches = net.launches() - launches0
    flop_sample = 2 * (3 * 256 + 3 * 256 * 256 + 256)
    # end to end: host inputs and outputs
    xh = x.cpu().pin_memory()
    yh = torch.zeros(n, dtype=torch.float32).pin_memory()
    t0 = time.perf_counter()
    net.forward(xh, out=yh)
    e2e_s = time.perf_counter() - t0
    # one training step (forward, backward, Adam) on 65,536 samples
    xt = x[:65536].contiguous()
    tt = torch.sin(2 * xt[:, 0]) + xt[:, 1] * xt[:, 2]
    for _ in range(3):
        net.train_step(xt, tt, 1e-4)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(10):
        net.train_step(xt, tt, 1e-4)
    torch.cuda.synchronize()
    train_s = (time.perf_counter() - t0) / 10
    peaks = _peaks()
    peak = peaks.get("bf16_tflops", 1900.0)
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    achieved = tm["gemm_flop"] / (tm["gemm_ms"] * 1e-3) / 1e12
    # One fused kernel runs the whole network per 128-row tile with the activations in
    # shared memory and TMEM: HBM carries only the inputs (12 B/row) and outputs (4 B/row),
    # and the weights come from L2, so the three 256 x 256 tensor-core layers bound it.
    fused_bytes = (n * 16 + 3 * 256 * 256 * 2) * args.steps
    achieved_gbs = fused_bytes / (tm["gemm_ms"] * 1e-3) / 1e9
    line = {
        "metric": "surrogate sigma(E,t) predictions/s", "value": n * args.steps / (ms * 1e-3),
        "unit": "samples/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16", "data": "synthetic",
        "config": {"workload": SURROGATE_WORKLOAD, "batch": n, "hidden": [256] * 4,
                   "l2": "L2 flushed between timed forwards (256 MB write outside the timed events); "
                         "activations stay in shared memory and TMEM"},
        "roofline": {"bound": "tensor",
                     "kernel": "mlp_fused_kernel (tcgen05 BF16, all layers per 128-row tile, 1M rows)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None, "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)"
                     if "bf16_tflops" in peaks else "fallback",
                     "hbm": {"algorithmic_bytes_per_step": fused_bytes / args.steps, "achieved_gbs": achieved_gbs,
                             "peak_gbs": hbm_peak, "frac": achieved_gbs / hbm_peak},
                     "fused_kernel_ms_per_step": tm["gemm_ms"] / args.steps,
                     "fused_kernel_share_of_step": tm["gemm_ms"] / ms},
        "model_tflops": flop_sample * n * args.steps / (ms * 1e-3) / 1e12,
        "train_step_ms_65536": train_s * 1e3,
        "gpu_launches": launches,
        "clocks": clk,
        "e2e": {"value": n / e2e_s, "unit": "samples/s", "h2d_bytes_per_step": n * 12,
                "d2h_bytes_per_step": n * 4, "seconds": e2e_s},
    }
    print(json.dumps(line), flush=True)


def run_small(args):
    """The small VAC case (4096-site sheet, 1 % vacancies, one vector, M = 512, 10
    correlation times of dt = hbar/gamma0, sigma^GK on 201 energies): one step = one whole
    run.  Latency-bound: every launch covers only 4096 site-vectors."""
    import torch
    import paper_1307_0288_gb300 as kg

    torch.cuda.set_device(_env_int("LOCAL_RANK", 0))
    m, nc, dt = 512, 10, 1.0
    w = ki.sheet_cells(32, 32, vacancy_conc=0.01, n_vec=1)
    stream = torch.cuda.Stream()
    h = kg.from_workload(w, stream=stream)
    n_p = len(kg.bessel_series(h.emax_ev * dt / w.gamma0_ev, TOL))
    phi_host = torch.from_numpy(w.vectors(1)).pin_memory()
    phi = phi_host.to("cuda")
    out = torch.zeros((1, nc, m), dtype=torch.complex128, device="cuda")
    en = np.linspace(-3 * w.gamma0_ev, 3 * w.gamma0_ev, 201)
    t_fs = dt * kg.HBAR_EV_FS / w.gamma0_ev

    def one_run(dst):
        kg.vac(h, phi, m, nc, dt, bessel_tol=TOL, out=dst)

    fp64_peak = fp64_peak_tflops(kg)

    for _ in range(args.warmup):
        one_run(out)
    torch.cuda.synchronize()
    kg.timing_enable(h, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    e0.record(stream)
    for _ in range(args.steps):
        one_run(out)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    cnt = kg.timing_read(h)
    kg.timing_enable(h, False)
    # sigma^GK(E, t) on the host from the last run's moments (Eqs. 6, 31)
    t0 = time.perf_counter()
    dens = kg.kpm_sum(out.cpu().numpy()[0].real, en, h.emax_ev, h.area_nm2)
    kg.conductivity(kg.KG_SIGMA_GK, dens, t_fs)
    sums_s = time.perf_counter() - t0
    # end to end: host input and output through the same call
    out_host = torch.zeros((1, nc, m), dtype=torch.complex128).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    kg.vac(h, phi_host, m, nc, dt, bessel_tol=TOL, out=out_host)
    e2e_s = time.perf_counter() - t0
    # paper-counted work of one run: per time, M - 1 KPM steps; per time step, two chains
    # of N_p - 1 Chebyshev-Bessel terms (Algorithm 2)
    paper_work = float(w.n_sites) * (nc * (m - 1) + (nc - 1) * 2 * (n_p - 1))
    per_run_s = ms * 1e-3 / args.steps
    work = (cnt["kpm_site_steps"] + cnt["evolve_site_steps"]) / args.steps   # executed, per run
    # dominant kernel: the cluster KPM loop (vectors in shared memory, 6 DFMA = 12 FP64 flops per
    # site-vector step); its CUDA-event phase time covers the moment loops of the timed runs
    kpm_flop = 12.0 * cnt["kpm_site_steps"]
    achieved_tflops = kpm_flop / (cnt["kpm_ms"] * 1e-3) / 1e12 if cnt["kpm_ms"] > 0 else 0.0
    line = {
        "metric": METRIC, "value": work / per_run_s, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "value_counts": "executed (site, vector, recursion step) updates",
        "paper_equivalent_site_updates_per_s": paper_work / per_run_s,
        "config": {"workload": SMALL_WORKLOAD, "sites": w.n_sites, "vacancies": len(w.vacancies),
                   "vectors": 1, "moments": m, "times": nc, "energies": 201, "bessel_terms": n_p,
                   "us_per_run": per_run_s * 1e6, "host_sums_us": sums_s * 1e6,
                   "kpm_us_per_step": cnt["kpm_ms"] * 1e3 / max(cnt["kpm_site_steps"] / w.n_sites, 1.0),
                   "l2": "working set 0.3 MB stays in L2 (vectors of the moment loop in shared memory); "
                         "one step = one whole run"},
        "roofline": {"bound": "alu", "kernel": "kpm_cluster_kernel<double,1> (VAC KPM steps, up to 256 per "
                                              "16-CTA cluster launch, vectors in shared memory)",
                     "achieved": achieved_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": achieved_tflops / fp64_peak, "traffic": None,
                     "peak_source": "measured in-run (kg_fp64_fma_rate)",
                     "note": "latency-bound: one recursion step over 4096 site-vectors takes about 1 us "
                             "(cluster barrier, distributed shared memory gathers, FP64 chain)"},
        "gpu_launches": int(cnt["kpm_launches"] + cnt["evolve_launches"] + cnt["other_launches"]),
        "clocks": clk,
        "e2e": {"value": work / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(phi_host.numel() * 16),
                "d2h_bytes_per_step": int(out_host.numel() * 16), "seconds": e2e_s},
    }
    if not args.no_cpu_baseline:
        import oracle
        ho = oracle.from_workload(w)
        t0 = time.perf_counter()
        oracle.vac_moments(ho, w.vectors(1)[:, 0], m, nc, dt)
        sec = time.perf_counter() - t0
        # the oracle runs Algorithms 2, 5 and 6 as printed: its executed work is the paper count
        line["cpu_baseline"] = {"value": paper_work / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"the whole run (VAC, 10 times, M = 512) in the oracle, one host "
                                          f"thread: {sec:.2f} s"}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + [BATCHED_WORKLOAD, SURROGATE_WORKLOAD, SMALL_WORKLOAD],
                    default=DEFAULT_WORKLOAD)
    args = ap.parse_args()
    global CELLS, VAC, R, M, DT, PREC, CONFIG_NAME
    if args.workload == BATCHED_WORKLOAD:
        return run_batched(args)
    if args.workload == SMALL_WORKLOAD:
        return run_small(args)
    if args.workload == SURROGATE_WORKLOAD:
        return run_surrogate(args)
    CELLS, VAC, R, M, DT, PREC = WORKLOADS[args.workload]
    CONFIG_NAME = args.workload
    if args.warmup < 1 or args.steps < 1:
        raise SystemExit("--steps and --warmup must be >= 1")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
