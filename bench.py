"""Benchmark: batched Helmholtz solves with the additive sweeping preconditioner.

Workload (one step): the 2D n=1023 problem at omega = 128 pi (16 points per
wavelength), 16 random smoothed horizontal velocity layers, PML 20 points,
layers of b = 4 columns, 32 Gaussian point sources -- factor all 3m-2 = 736
layer subproblems in complex64 (Algorithm 1, plus the dense trace-transfer
maps of the two sweeps) and solve all 32 right-hand sides to a relative FP64
residual of 1e-6 with right-preconditioned FGMRES(40) (Algorithm 2 as the
preconditioner).  Metric: solves per second (right-hand sides solved per
second of step time), whole job over all ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl asp|reference]

N > 1 runs under torchrun, one independent replica per GPU (the path has no
cross-GPU exchange: replicas only).  ``--impl reference`` times the CPU FP64
oracle (test infrastructure) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "solves/s (2D n=1023, omega=128pi, 32 RHS, to 1e-6 FP64 residual)"
UNIT = "solves/s"
WORKLOAD = {"workload": "2d_helmholtz_n1023_layered_omega128pi_pml20_b4_32rhs", "n": 1023,
            "omega": "128*pi", "pml": 20, "b": 4, "nrhs": 32, "velocity": "16 random layers, smoothed 3h",
            "factor_precision": "complex64", "krylov": "FGMRES(40) FP64", "tol": 1e-6,
            "l2": "no flush needed: factors 11.5 GB + transfer maps 4.1 GB exceed the 129 MB L2"}
PHASES = ["factor", "tmap", "embed", "chain", "fill", "elementwise", "matvec", "krylov", "schur3d", "tdiag"]
METRIC_3D = "solves/s (3D n=95, omega=48pi, 1 RHS, to 1e-6 FP64 residual)"
WORKLOAD_3D = {"workload": "3d_helmholtz_n95_bump_omega48pi_pml8_b4_1rhs", "n": 95, "omega": "48*pi", "pml": 8,
               "b": 4, "nrhs": 1, "velocity": "1 + 0.3 Gaussian bump at the centre",
               "factor_precision": "complex64", "krylov": "FGMRES(40) FP64", "tol": 1e-6,
               "l2": "no flush needed: slab factors 76 GB exceed the 129 MB L2"}


def algorithmic3d(n, gamma, b):
    """Algorithmic work of the 3D slab factor: every slab has n dense blocks of
    size nb = n*w, each inverted by Gauss-Jordan (nb^3 complex multiply-adds =
    8 nb^3 real flops); an apply reads every stored block twice (forward and
    backward substitution) in complex64."""
    m, wM, wR, wL, _ = _layer_widths(n, gamma, b)
    nbs = [n * w for w in wM + wR + wL]
    flops = 8.0 * n * sum(nb ** 3 for nb in nbs)
    w_bytes = 8.0 * n * sum(nb * ((nb + 3) // 4 * 4) for nb in nbs)
    # the rank-256 updates (tensor cores): per outer block [C0, C0+K), every
    # row and the nb - K columns outside it, K complex multiply-adds each
    schur = 0.0
    for nb in nbs:
        for C0 in range(0, nb, 256):
            K = min(256, nb - C0)
            schur += 8.0 * nb * (nb - K) * K
    return {"factor_flops": flops, "factor_bytes": w_bytes, "apply_bytes": 2 * w_bytes,
            "schur_flops": n * schur}


def algorithmic3d_nd(n, gamma, b):
    """Work of the nested-dissection slab factor (Section 4), from the library's
    host plan of the n x n column grid: per slab, the fronts' Gauss-Jordan steps
    (s steps over an ns x ns front: s*ns^2 complex multiply-adds, 8 real flops
    each) and the stored factor entries ([X; L] and P), read once each by an
    apply's forward and backward passes in complex64."""
    import ctypes
    from paper_1504_04058_gb300 import _lib
    lib = _lib.load()
    m, wM, wR, wL, _ = _layer_widths(n, gamma, b)
    flops = 0.0
    entries = 0.0
    for w in wM + wR + wL:
        st = (ctypes.c_longlong * 9)()
        _lib.check(lib.asp_nd_plan_check(n, w, st, 9), "asp_nd_plan_check")
        entries += st[3]
        flops += 8.0 * st[8]
    return {"factor_flops": flops, "factor_bytes": 8.0 * entries, "apply_bytes": 8.0 * entries}


def dist_max(x: float, device=None) -> float:
    """Maximum of a per-rank value over all ranks (the step time the job is
    judged by); the value itself when there is no process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, nrhs: int, ms: float) -> float:
    """Right-hand sides solved per second by the whole job: every rank runs an
    independent replica (weak scaling), timed by the slowest rank."""
    return world * nrhs / (ms * 1e-3)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self, device_index: int = 0):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9 or not parts[0].isdigit() or int(parts[0]) != device_index:
                continue
            rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": sorted(reasons)}


def _layer_widths(n, gamma, b, gamma_a=None, widths=None):
    """Layer count and padded subproblem widths: layers of the given physical
    widths (default: b columns, the last one taking the remainder of the
    P = n + 2 - 2*gamma physical columns), padded by gamma_a - 1 auxiliary-PML
    columns on their inner sides (the first layer's grid starts at column 1,
    the last one's ends at column n).  wT: the R and L subproblems that have a
    transfer map (p = 2..m-1)."""
    ga = gamma if not gamma_a else gamma_a
    P = n + 2 - 2 * gamma
    if widths is None:
        m = P // b
        widths = [b] * (m - 1) + [b + P - m * b]
    m = len(widths)
    alpha, beta, a = [], [], gamma
    for p, x in enumerate(widths, start=1):
        alpha.append(a)
        beta.append(a + x - 1 if p < m else n + 1 - gamma)
        a += x
    m_lo = [1 if p == 0 else alpha[p] - ga + 1 for p in range(m)]
    m_hi = [n if p == m - 1 else beta[p] + ga - 1 for p in range(m)]
    wM = [m_hi[p] - m_lo[p] + 1 for p in range(m)]
    wR = [m_hi[p] - alpha[p] + 1 for p in range(1, m)]
    wL = [beta[p] - m_lo[p] + 1 for p in range(0, m - 1)]
    wT = [m_hi[p] - alpha[p] + 1 for p in range(1, m - 1)]  # R maps; the L maps match for equal widths
    return m, wM, wR, wL, wT


def _map_widths(n, gamma, b, gamma_a=None, widths=None):
    """Padded widths of every subproblem with a transfer map: H_p^R and H_p^L
    for p = 2..m-1."""
    m, wM, wR, wL, wT = _layer_widths(n, gamma, b, gamma_a, widths)
    return wR[:m - 2] + wL[1:m - 1]


def tc_maps(n, gamma, b, precision="c64", gamma_a=None, widths=None):
    """True when the library builds the transfer maps on the tensor cores
    (complex64 factors, every sweep subproblem at most 32 columns wide)."""
    m, wM, wR, wL, wT = _layer_widths(n, gamma, b, gamma_a, widths)
    return precision in ("c64", "c64sym") and m >= 3 and max(wR + wL) <= 32


def algorithmic(n, gamma, b, nrhs, esz, gamma_a=None, tc=False, widths=None):
    """Algorithmic bytes and flops per launch of each phase: a banded solve
    reads its L and U band once, n*w*(2w+1) entries, and does 8*(2w+1) real
    flops per entry row per right-hand side.  A transfer map T_p has n
    columns and is written once (n*n entries).  Built by solves (tc False),
    column r's forward pass starts at its own block (n - r steps of w^2
    complex MACs) and its backward pass takes all n: 1.5*n^2*w^2 complex MACs
    per map.  Built from the diagonal blocks of the inverse (tc True), each
    column runs one chain of r block steps from its diagonal block, for the
    upper and (by symmetry) the lower triangle: n(n-1) w^2 complex MACs per
    map, plus the diagonal-block recursion (tdiag), two w x w x w complex
    products per block."""
    m, wM, wR, wL, _ = _layer_widths(n, gamma, b, gamma_a, widths)
    wT = _map_widths(n, gamma, b, gamma_a, widths)  # 2(m-2) maps, R then L
    band = lambda ws: sum(n * w * (2 * w + 1) for w in ws)  # noqa: E731
    N = n * n
    vec = N * nrhs * esz
    out = {}
    out["embed"] = {"bytes": band(wM) * esz + 2 * vec, "flops": 8.0 * nrhs * band(wM)}
    out["fill"] = {"bytes": (band(wR) + band(wL)) * esz + 2 * vec, "flops": 8.0 * nrhs * (band(wR) + band(wL))}
    if tc:
        out["tmap"] = {"bytes": band(wT) * esz + len(wT) * n * n * esz + len(wT) * n * 2 * 32 * esz,
                       "flops": 8.0 * n * (n - 1) * sum(w * w for w in wT)}
        out["tdiag"] = {"bytes": band(wT) * esz + len(wT) * n * 2 * 32 * esz,
                        "flops": 8.0 * 2 * (n - 1) * sum(w ** 3 for w in wT)}
    else:
        out["tmap"] = {"bytes": band(wT) * esz + len(wT) * n * n * esz,
                       "flops": 8.0 * 1.5 * n * n * sum(w * w for w in wT)}
    out["chain"] = {"bytes": len(wT) * n * n * esz, "flops": 8.0 * nrhs * len(wT) * n * n}
    out["factor"] = {"bytes": (band(wM) + band(wR) + band(wL)) * esz,
                     "flops": 8.0 * n * sum(w ** 3 for w in wM + wR + wL)}
    out["matvec"] = {"bytes": 2 * N * nrhs * 16 + N * 8, "flops": 8.0 * 5 * N * nrhs}
    return out


def symmetric_band_bytes(n, gamma, b, esz, gamma_a=None, widths=None):
    """Bytes of every subproblem's symmetric factorization (Section 3.1,
    practical remark 4): L of LDL^T (w sub-diagonals) and D, n*w*(w+1) entries
    per subproblem of padded width w."""
    m, wM, wR, wL, _ = _layer_widths(n, gamma, b, gamma_a, widths)
    return sum(n * w * (w + 1) for w in wM + wR + wL) * esz


def stored_factor_bytes(n, gamma, b, esz, gamma_a=None, widths=None, packed=True):
    """Bytes of the factor blocks this library stores: per subproblem n blocks,
    each the packed upper triangle of the symmetric W_k Delta (w(w+1)/2
    entries, padded to even) for complex64, else w x w_pad."""
    m, wM, wR, wL, _ = _layer_widths(n, gamma, b, gamma_a, widths)
    if packed:
        return sum(n * ((w * (w + 1) // 2 + 1) // 2 * 2) for w in wM + wR + wL) * esz
    return sum(n * w * (w + (w % 2)) for w in wM + wR + wL) * esz


def _traffic_from_profile(kernel_phase):
    """dram bytes per launch (ncu, the n=1023 workload) from the committed
    summary, if it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "btsolve_n1023_traffic.txt")
    try:
        kv = {}
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
    except OSError:
        return None
    name, key = ("chain.cu", "chain_sha256_16") if kernel_phase == "chain" else ("btsolve.cuh", "btsolve_sha256_16")
    src = os.path.join(ROOT, "paper_1504_04058_gb300", "csrc", name)
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if kv.get(key) != sha:
        return None
    v = kv.get(f"{kernel_phase}_dram_bytes_per_launch")
    return float(v) if v else None


def run_asp(args, rank, world):
    import numpy as np
    import torch

    import paper_1504_04058_gb300 as asp
    import workloads as W

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    restart = 40
    if args.workload == "n1023":
        P = W.problem_2d_n1023_layered(nrhs=32, seed=1504 + rank, source=args.source)
    elif args.workload == "n95_3d":
        P = W.problem_3d_n95_bump()
    elif args.workload == "n47_3d_slab":  # one 3D slab (m = 1), blocks of 47*47 unknowns: profiling case
        P = W.small_problem(3, 47, 12 * math.pi, 6, 37, "bump", nrhs=1)
    elif args.workload == "n255x32":  # the n=1023 workload's layer widths (PML 20, b = 4) on 4.2 GB: profiler captures
        P = W.small_problem(2, 255, 32 * math.pi, 20, 4, "layered", nrhs=32, seed=1504 + rank)
        restart = 4
    elif args.workload == "n255x1":  # the same with one right-hand side, for captures of the 1-RHS layer solves
        P = W.small_problem(2, 255, 32 * math.pi, 20, 4, "layered", nrhs=1, seed=1504 + rank)
        restart = 4
    else:  # smaller case of the same kernels, for profiler captures
        P = W.small_problem(2, 511, 64 * math.pi, 16, 4, "layered", nrhs=32, seed=1504 + rank)
        restart = 16
    pml_aux = args.pml_aux if args.pml_aux else (P.pml_aux or 0)
    prm = asp.make_params(P.n, P.omega, P.pml, P.b, pml_aux=pml_aux, C=P.C, precision=args.precision,
                          max_rhs=P.nrhs, restart=restart, dim=P.dim,
                          slab_solver=args.slab_solver if P.dim == 3 else "block")
    widths = None
    if args.layer_widths:  # "BMIN:BMAX": widths chosen from the velocity by the library
        bmin, bmax = (int(x) for x in args.layer_widths.split(":"))
        widths = asp.layer_widths_from_velocity(prm, P.c, bmin, bmax)
    h = asp.asp_setup(P.c, prm, widths=widths)
    f_host = torch.from_numpy(P.f).pin_memory()
    f = f_host.to(dev)
    u = torch.empty_like(f)
    stream = torch.cuda.current_stream()

    def step():
        h.factor()
        _, info = h.gmres_solve(f, u, tol=P.tol, maxit=200)
        return info

    for _ in range(args.warmup):
        info = step()
    tuned = None
    if P.dim == 2 and not args.no_autotune:
        # launch shapes of the layer solves, chosen by timing on these factors
        tuned = {str(nr): h.autotune(nr) for nr in sorted({P.nrhs, 1})}
        info = step()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    h.take_launch_count()
    h.set_phase_timing(True)
    h.phase_times()
    clocks = ClockSampler()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    its = []
    for _ in range(args.steps):
        info = step()
        its.append(max(i["iterations"] for i in info))
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop(dev.index)
    phases = h.phase_times()
    h.set_phase_timing(False)
    launches = h.take_launch_count()
    ms = dist_max(ms, dev)
    if world > 1:
        torch.distributed.barrier()
    conv = all(i["converged"] for i in info)
    worst_res = max(i["rel_res_true"] for i in info)

    # ---- factor-resident solve rate (serving: factors cached, solve only)
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    h.gmres_solve(f, u, tol=P.tol, maxit=200)
    s1.record(stream)
    torch.cuda.synchronize()
    solve_ms = s0.elapsed_time(s1)

    # ---- factor alone (both internal streams joined on the caller's stream)
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    h.factor()
    g1.record(stream)
    torch.cuda.synchronize()
    factor_ms = g0.elapsed_time(g1)

    # ---- one preconditioner apply on its own (factors resident), at one
    # right-hand side (where the apply streams its factors from HBM) and at the
    # workload's count
    apply_runs = []
    if P.dim == 2:
        for nr in sorted({1, P.nrhs}):
            r_in = f[..., :nr].contiguous()
            z_out = torch.empty_like(r_in)
            for _ in range(2):
                h.apply_preconditioner(r_in, z_out)
            torch.cuda.synchronize()
            h.set_phase_timing(True)
            h.phase_times()
            reps = 5
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(reps):
                h.apply_preconditioner(r_in, z_out)
            a1.record(stream)
            torch.cuda.synchronize()
            ph = h.phase_times()
            h.set_phase_timing(False)
            apply_runs.append((nr, a0.elapsed_time(a1) / reps,
                               {k: round(ph[k][0] / reps, 3) for k in ("embed", "chain", "fill", "elementwise")}))

    # ---- end to end through the public API with host buffers.  The factor does
    # not read the right-hand sides, so a copy stream uploads them (after the
    # previous step's solution has been downloaded there) while the factor runs;
    # the solve waits for the upload.
    u_host = torch.empty_like(f_host).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    copy_stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    x0.record(stream)
    copy_stream.wait_event(x0)
    for _ in range(e2e_steps):
        with torch.cuda.stream(copy_stream):
            f.copy_(f_host, non_blocking=True)
        uploaded = torch.cuda.Event()
        uploaded.record(copy_stream)
        h.factor()
        stream.wait_event(uploaded)
        h.gmres_solve(f, u, tol=P.tol, maxit=200)
        solved = torch.cuda.Event()
        solved.record(stream)
        copy_stream.wait_event(solved)
        with torch.cuda.stream(copy_stream):
            u_host.copy_(u, non_blocking=True)
    stream.wait_stream(copy_stream)
    x1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = x0.elapsed_time(x1) / e2e_steps
    e2e_ms = dist_max(e2e_ms, dev)
    nbytes = P.f.size * 16

    # ---- roofline of the dominant kernel (live CUDA-event phase times)
    peaks, peak_kind = _peaks()
    roof_more = None
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12  # TFLOP/s at max clock
    phase_ms = {p: round(phases[p][0] / args.steps, 3) for p in PHASES}
    value = whole_job_rate(world, P.nrhs, ms)
    if P.dim == 3 and args.slab_solver == "nd":
        alg3 = algorithmic3d_nd(P.n, P.pml, P.b)
        fl = alg3["factor_flops"] / (factor_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": fl, "peak": fp32_peak, "unit": "TFLOP/s", "frac": fl / fp32_peak,
                "kernel": "nested-dissection slab factor (assembly, extend-add, blocked Gauss-Jordan on the fronts' "
                          "fully summed columns, CUDA cores; all launches of the factor)",
                "peak_source": "SMs x 128 FP32 lanes x 2 flops x max SM clock (derived)",
                "traffic": None, "factor_ms": factor_ms, "algorithmic_flops": alg3["factor_flops"],
                "factor_bytes": alg3["factor_bytes"]}
        apply_ms = (phases["embed"][0] + phases["fill"][0]) / max(phases["embed"][1], 1)
        roof["hbm_view"] = {"kernel": "3D slab solves of one apply (nested-dissection fronts)",
                            "algorithmic_bytes": alg3["apply_bytes"], "ms_per_apply": apply_ms,
                            "GBps": alg3["apply_bytes"] / (apply_ms * 1e-3) / 1e9,
                            "frac_of_measured_hbm": alg3["apply_bytes"] / (apply_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]}
        config = (dict(WORKLOAD_3D, parallelism=f"replicas x{world}", slab_solver="nested dissection",
                       l2="no flush needed: slab factors exceed the 129 MB L2")
                  if args.workload == "n95_3d" else
                  {"workload": "3d_helmholtz_n47_one_slab_omega12pi_pml6_b37 (profiling case)",
                   "slab_solver": "nested dissection"})
        metric = METRIC_3D
    elif P.dim == 3:
        alg3 = algorithmic3d(P.n, P.pml, P.b)
        # dominant kernel: the tensor-core rank-256 Schur update (tcgen05, split TF32)
        tf32_peak = peaks["bf16_tflops"] * 0.5  # nominal dense tf32 : bf16 ratio (1.1 : 2.25 PFLOP/s)
        sch_ms, sch_n = phases["schur3d"]
        sch_avg = sch_ms / max(sch_n, 1)
        flops_per_launch = alg3["schur_flops"] * args.steps / max(sch_n, 1)
        ach = flops_per_launch / (sch_avg * 1e-3) / 1e12 if sch_n else 0.0
        roof = {"bound": "tensor", "achieved": ach, "peak": tf32_peak, "unit": "TFLOP/s", "frac": ach / tf32_peak,
                "kernel": "tc_update_persistent_kernel: complex64 rank-256 Schur update of the slab factor on tcgen05 "
                          "(split TF32, 3 tensor products per useful product; achieved counts useful flops)",
                "peak_source": f"bf16_tflops ({peak_kind}) x 0.5 nominal tf32/bf16 ratio",
                "traffic": None, "avg_launch_ms": sch_avg, "launches_per_step": sch_n / args.steps,
                "algorithmic_flops_per_launch": flops_per_launch,
                "whole_factor": {"algorithmic_flops": alg3["factor_flops"], "ms": factor_ms,
                                 "TFLOPs": alg3["factor_flops"] / (factor_ms * 1e-3) / 1e12,
                                 "frac_of_fp32_alu_peak": alg3["factor_flops"] / (factor_ms * 1e-3) / 1e12 / fp32_peak}}
        apply_ms = (phases["embed"][0] + phases["fill"][0]) / max(phases["embed"][1], 1)
        roof["hbm_view"] = {"kernel": "3D slab solves of one apply", "algorithmic_bytes": alg3["apply_bytes"],
                            "ms_per_apply": apply_ms,
                            "GBps": alg3["apply_bytes"] / (apply_ms * 1e-3) / 1e9,
                            "frac_of_measured_hbm": alg3["apply_bytes"] / (apply_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]}
        config = (dict(WORKLOAD_3D, parallelism=f"replicas x{world}") if args.workload == "n95_3d" else
                  {"workload": "3d_helmholtz_n47_one_slab_omega12pi_pml6_b37 (profiling case)"})
        metric = METRIC_3D
    else:
        tcm = tc_maps(P.n, P.pml, P.b, args.precision, pml_aux, widths)
        alg = algorithmic(P.n, P.pml, P.b, P.nrhs, 8, pml_aux, tc=tcm, widths=widths)
        tf32_peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]) * 0.5

        def roofline_of(ph):
            """Roofline entry of one phase's kernel from its live CUDA-event times
            (total over the timed steps and launch count)."""
            tot_ms, nl = phases[ph]
            avg_ms = tot_ms / max(nl, 1)
            if ph == "tmap" and tcm:
                # tensor-core maps: useful flops (the complex products of the
                # chains) against the dense TF32 peak; the split-precision
                # scheme executes three tensor products per useful one
                ach = alg[ph]["flops"] / (avg_ms * 1e-3) / 1e12
                r = {"bound": "tensor", "achieved": ach, "peak": tf32_peak, "unit": "TFLOP/s",
                     "frac": ach / tf32_peak, "kernel": "tmap_tc_kernel (transfer maps on tcgen05, split TF32)",
                     "peak_source": f"bf16_tflops_sustained ({peak_kind}) x 0.5 nominal tf32/bf16 ratio",
                     "executed_tensor_frac": 3 * ach / tf32_peak}
            elif ph in ("embed", "fill", "tmap", "factor", "tdiag"):
                ach = alg[ph]["flops"] / (avg_ms * 1e-3) / 1e12
                kern = {"embed": "btsolve_kernel (M-solves)", "fill": "btsolve_kernel (sweep fills)",
                        "tmap": "btsolve_kernel (transfer maps by solves)", "factor": "btfactor_kernel",
                        "tdiag": "gdiag_kernel"}[ph]
                r = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": ach / fp32_peak, "kernel": kern,
                     "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 flops x max SM clock (derived; no measured FP32 "
                                    "peak is available)"}
            else:
                ach = alg[ph]["bytes"] / (avg_ms * 1e-3) / 1e9
                r = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": ach / peaks["hbm_gbs"], "kernel": ph, "peak_source": f"hbm_gbs ({peak_kind})"}
            # DRAM bytes per launch from the committed capture of the n=1023 workload (default
            # layers, complex64), if taken on this source
            headline = (args.workload == "n1023" and args.precision == "c64" and not pml_aux and widths is None)
            r["traffic"] = _traffic_from_profile(ph) if headline and ph in ("embed", "fill", "chain") else None
            r["avg_launch_ms"] = avg_ms
            r["launches_per_step"] = nl / args.steps
            r["hbm_view"] = {"algorithmic_bytes": alg[ph]["bytes"],
                             "GBps": alg[ph]["bytes"] / (avg_ms * 1e-3) / 1e9,
                             "frac_of_measured_hbm": alg[ph]["bytes"] / (avg_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]}
            return r

        # The dominant kernel is the one with the most device time in the step.
        # The factor's two launches (M-subproblems on the internal stream, R/L
        # on the caller's) run at the same time, so their event times overlap
        # and their sum is not device time; it is ranked by its longer launch.
        def device_ms(ph):
            tot, nl = phases[ph]
            return tot / max(nl / max(args.steps, 1), 1.0) if ph == "factor" else tot
        dom = max((p for p in PHASES if p in alg), key=device_ms)
        roof = roofline_of(dom)
        roof["selection"] = ("largest device time per step among the phases (the factor's concurrent stream launches "
                             "counted as one)")
        others = [p for p in ("tmap", "factor", "fill", "embed", "chain") if p in alg and p != dom and phases[p][1]]
        roof_more = {p: roofline_of(p) for p in others}
        config = (dict(WORKLOAD, parallelism=f"replicas x{world}") if args.workload == "n1023" else
                  {"workload": "2d_helmholtz_n255_layered_omega32pi_pml20_b4_32rhs (profiling case)"}
                  if args.workload == "n255x32" else
                  {"workload": "2d_helmholtz_n255_layered_omega32pi_pml20_b4_1rhs (profiling case)"}
                  if args.workload == "n255x1" else
                  {"workload": "2d_helmholtz_n511_layered_omega64pi_pml16_b4_32rhs (profiling case)"})
        metric = METRIC
    if args.source == "packet":
        config = dict(config, sources="Gaussian wave packets, one wavelength wide, seeded centres and directions")
    if widths is not None:
        config = dict(config, layer_widths=f"from the velocity, {args.layer_widths.replace(':', '..')} columns",
                      layers=len(widths), width_histogram={str(x): widths.count(x) for x in sorted(set(widths))})
    if args.pml_aux:
        config = dict(config, pml_aux=args.pml_aux,
                      variant="thinner auxiliary PML inside the domain (the boundary PML keeps its width)")
    precond_apply = None
    if apply_runs:
        alg2 = algorithmic(P.n, P.pml, P.b, 1, 8, pml_aux, tc=tcm, widths=widths)
        packed = args.precision == "c64sym" and P.dim == 2
        lu_bytes = alg2["factor"]["bytes"]                     # nonsymmetric banded L and U, once (complex64)
        sym_bytes = symmetric_band_bytes(P.n, P.pml, P.b, 8, pml_aux, widths)
        band_bytes = sym_bytes if packed else lu_bytes
        stored = stored_factor_bytes(P.n, P.pml, P.b, 8, pml_aux, widths, packed)
        design_bytes = stored + alg2["chain"]["bytes"]         # what this design reads: its factors + the maps
        precond_apply = []
        for nr, a_ms, ph in apply_runs:
            vec = 3 * P.n * P.n * nr * 16                      # r in, z out, and the complex64 copy of r
            # per phase: the banded layer solves (M-solves: the M factors; fills: the R and L factors,
            # each band read once as the paper's solves read it) and the sweep chain (the transfer maps
            # this design reads), each against its own phase time
            algn = algorithmic(P.n, P.pml, P.b, nr, 8, pml_aux, tc=tcm, widths=widths)
            phase_hbm = {}
            for phk in ("embed", "fill", "chain"):
                byt = algn[phk]["bytes"] if phk == "chain" else algn[phk]["bytes"] - 2 * P.n * P.n * nr * 8
                t_ms = ph.get(phk, 0.0)
                phase_hbm[phk] = {"bytes": byt, "ms": t_ms,
                                  "frac_of_measured_hbm": byt / (t_ms * 1e-3) / 1e9 / peaks["hbm_gbs"] if t_ms else None}
            ls_bytes = phase_hbm["embed"]["bytes"] + phase_hbm["fill"]["bytes"]
            ls_ms = ph.get("embed", 0.0) + ph.get("fill", 0.0)
            phase_hbm["layer_solves"] = {"bytes": ls_bytes, "ms": ls_ms,
                                         "frac_of_measured_hbm": ls_bytes / (ls_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]
                                         if ls_ms else None}
            precond_apply.append({
                "nrhs": nr, "ms": a_ms, "phase_ms": ph, "phase_hbm": phase_hbm,
                "algorithmic_bytes": band_bytes + vec,
                "GBps": (band_bytes + vec) / (a_ms * 1e-3) / 1e9,
                "frac_of_measured_hbm": (band_bytes + vec) / (a_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                "nonsymmetric_band_bytes": lu_bytes + vec,
                "design_bytes": design_bytes + vec,
                "design_GBps": (design_bytes + vec) / (a_ms * 1e-3) / 1e9,
                "note": ("algorithmic bytes: every layer subproblem's symmetric factorization once (Section 3.1, "
                         "practical remark 4: L of LDL^T and D, n*w*(w+1) entries per subproblem), the storage "
                         "this build's complex64 path uses; nonsymmetric: the banded L and U, n*w*(2w+1); design "
                         "bytes: the packed blocks this design reads plus the transfer maps of the sweep chain"
                         if packed else
                         "algorithmic bytes: the banded L and U factors of every layer subproblem, once, as the "
                         "paper's apply reads them; design bytes add the transfer maps this implementation's sweep "
                         "chain reads")})
    line = {
        "metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": f"{args.precision} factors / f64 krylov", "data": "synthetic",
        "config": config,
        "iterations_max": max(its), "converged": conv, "worst_rel_res_true": worst_res,
        "solve_only_solves_per_s": world * P.nrhs / (solve_ms * 1e-3),
        "factor_ms": factor_ms,
        "phase_ms_per_step": phase_ms,
        "e2e": {"value": whole_job_rate(world, P.nrhs, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes, "ms_per_step": e2e_ms},
        "gpu_launches": launches,
        "autotune": tuned,
        "roofline": roof,
        "roofline_other_kernels": roof_more,
        "precond_apply": precond_apply,
        "clocks": clk,
    }
    if args.workload == "n1023" and args.precision in ("c64", "c64sym") and not args.no_fp64_path:
        # the plain FP64 path on the same problem and GPU: complex128 factors
        # and applies inside the same FP64 FGMRES, one warm-up and one timed
        # step; the mixed path's solutions are compared with its solutions
        u64 = u.clone()
        h.destroy()
        prm128 = asp.make_params(P.n, P.omega, P.pml, P.b, pml_aux=pml_aux, C=P.C, precision="c128",
                                 max_rhs=P.nrhs, restart=restart, dim=P.dim)
        h = asp.asp_setup(P.c, prm128, widths=widths)
        h.factor()
        if not args.no_autotune:
            h.autotune(P.nrhs)
        h.gmres_solve(f, u, tol=P.tol, maxit=200)
        torch.cuda.synchronize()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        h.factor()
        q_mid = torch.cuda.Event(enable_timing=True)
        q_mid.record(stream)
        _, info128 = h.gmres_solve(f, u, tol=P.tol, maxit=200)
        q1.record(stream)
        torch.cuda.synchronize()
        ms128 = q0.elapsed_time(q1)
        d = (u64 - u).abs().amax(dim=(0, 1)) / u.abs().amax(dim=(0, 1))
        line["fp64_path"] = {
            "value": whole_job_rate(world, P.nrhs, ms128), "unit": UNIT, "ms_per_step": ms128,
            "factor_ms": q0.elapsed_time(q_mid), "iterations_max": max(i["iterations"] for i in info128),
            "worst_rel_res_true": max(i["rel_res_true"] for i in info128),
            "mixed_speedup": value / whole_job_rate(world, P.nrhs, ms128),
            "mixed_vs_fp64_max_rel_diff": float(d.max()),
            "note": "complex128 factors and applies, same problem, same FGMRES(40) to 1e-6, one timed step; "
                    "mixed_vs_fp64_max_rel_diff: per right-hand side, max |u_c64 - u_c128| / max |u_c128| "
                    "(two tolerance-stopped solutions)"}
    h.destroy()
    return line


ORACLE_SAMPLER = r"""
import json, os, sys, time
sys.path.insert(0, %r)
import numpy as np
import workloads as W
from oracle import operator, partition, subproblems
steps, its = %d, %d
P = W.problem_2d_n1023_layered(nrhs=1)
part = partition.make_partition(P.n, P.pml, P.b)
m = part.m
A = operator.helmholtz_matrix(2, P.n, P.omega, P.c, P.pml, P.C)
x = P.f[..., 0].reshape(-1)
rng = np.random.default_rng(0)
for step in range(steps):
    # one subproblem of each kind per step, rotating over the layers
    t_fac, t_sol = {}, {}
    for kind, lo, hi in (("M", 1, m), ("R", 2, m), ("L", 1, m - 1)):
        p = lo + (step * 37) %% (hi - lo + 1)
        t0 = time.perf_counter()
        F = subproblems.factor_subproblem(2, P.n, P.omega, P.c, P.pml, P.C, part, p, kind)
        t1 = time.perf_counter()
        F.solve(rng.standard_normal((F.w, F.T)) + 0j)
        t2 = time.perf_counter()
        t_fac[kind], t_sol[kind] = t1 - t0, t2 - t1
        del F
    t0 = time.perf_counter(); A @ x; t_mv = time.perf_counter() - t0
    # Krylov vector work of the oracle's FGMRES: modified Gram-Schmidt takes
    # j+1 dot products and axpys at iteration j; time its+1 of them on
    # N-vectors and scale to sum_{j=1..its} (j+1) per right-hand side
    v = np.asarray(P.f[..., 0].reshape(-1), dtype=np.complex128)
    w = v * (1 + 0.5j)
    t0 = time.perf_counter()
    for _ in range(its + 1):
        hij = np.vdot(v, w)
        w = w - hij * v
    t_gs = (time.perf_counter() - t0) * (sum(j + 1 for j in range(1, its + 1)) / (its + 1))
    print(json.dumps({"step": step, "fac": t_fac, "sol": t_sol, "matvec": t_mv, "gs_per_rhs": t_gs,
                      "layers": m}), flush=True)
"""


def oracle_samples(steps: int, iterations: int, threads: int = 1, timeout: float = 900.0):
    """Run the oracle as it stands on `steps` bounded samples of the n=1023
    workload in a child process (numpy/LAPACK limited to `threads` threads).
    Each sample factors and solves one layer subproblem of each kind (M, R, L;
    the layer index rotates from sample to sample), runs one sparse matvec, and
    times the Gram-Schmidt vector work of `iterations` FGMRES iterations.
    Returns (per-sample records, wall seconds of each sample, error)."""
    code = ORACLE_SAMPLER % (ROOT, steps, iterations)
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    recs, walls = [], []
    proc = subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                            text=True, env=env)
    t_last = time.perf_counter()
    deadline = t_last + timeout
    for line in proc.stdout:
        now = time.perf_counter()
        if line.startswith("{"):
            recs.append(json.loads(line))
            walls.append(now - t_last)
            t_last = now
        if now > deadline:
            proc.kill()
            break
    err = proc.stderr.read()
    proc.wait()
    if proc.returncode not in (0, None) and not recs:
        return [], [], err[-300:]
    return recs, walls, None


def oracle_batch_seconds(rec: dict, iterations: int, nrhs: int = 32) -> float:
    """One 32-RHS batch of the oracle extrapolated from one sample: factor all
    3m-2 subproblems, then per right-hand side `iterations` applies (m M-solves
    and m-1 solves of each sweep kind) and matvecs plus its Gram-Schmidt work."""
    m = rec["layers"]
    f, s = rec["fac"], rec["sol"]
    setup = m * f["M"] + (m - 1) * (f["R"] + f["L"])
    apply1 = m * s["M"] + (m - 1) * (s["R"] + s["L"])
    return setup + nrhs * (iterations * (apply1 + rec["matvec"]) + rec["gs_per_rhs"])


def oracle_iterations():
    """The oracle's own FGMRES iteration count on the n=1023 benchmark problem
    (tests/golden/oracle_iterations_n1023.txt, written by the oracle-only script
    beside it); None if the file is absent."""
    path = os.path.join(ROOT, "tests", "golden", "oracle_iterations_n1023.txt")
    try:
        its = [int(ln.split()[1]) for ln in open(path) if ln.strip() and not ln.startswith("#")]
    except OSError:
        return None
    return max(its) if its else None


def cpu_baseline_sample(iterations: int, samples: int = 8):
    """The oracle on one host thread, `samples` bounded samples (about 1-2 s
    each), each extrapolated to one 32-RHS batch; the median is reported."""
    recs, walls, err = oracle_samples(samples, iterations, threads=1)
    if not recs:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": err}
    t_batch = statistics.median(oracle_batch_seconds(r, iterations) for r in recs)
    return {"value": 32 / t_batch, "unit": UNIT, "cores": 1, "kind": "oracle",
            "value_kind": "extrapolated from bounded samples",
            "sample": (f"{len(recs)} samples, each: oracle factor + solve of one layer subproblem of each kind "
                       f"(M, R, L; 3 of the 736), one sparse matvec and the Gram-Schmidt vector work of "
                       f"{iterations} FGMRES iterations at n=1023, extrapolated to one 32-RHS batch "
                       f"(factor all 736, {iterations} applies + matvecs + Krylov work per right-hand side); "
                       f"median over samples"),
            "sample_wall_s": sum(walls), "extrapolated_batch_s": t_batch}


def cpu_baseline_all_cores(iterations: int):
    """The oracle as it stands on every host core: all 736 layer subproblems
    are factored and solved once each, one subproblem per worker process
    (numpy/LAPACK single-threaded in each), in a child process that never
    touches CUDA.  Measured: the wall time of the parallel factorizations, of
    the parallel M-solves, and each R/L solve.  Scaled to one 32-RHS batch:
    factor wall + 32 * iterations * (M-solve wall + the longer of the two
    sequential sweeps + one matvec) -- Algorithm 2 parallelizes the M-solves,
    while each sweep stays a chain of dependent solves."""
    code = r"""
import json, os, sys, time
sys.path.insert(0, %r)
import multiprocessing as mp
import numpy as np
import workloads as W
from oracle import operator, partition, subproblems
P = W.problem_2d_n1023_layered(nrhs=1)
part = partition.make_partition(P.n, P.pml, P.b)
m = part.m

def job(t):
    kind, p = t
    rng = np.random.default_rng(p)
    t0 = time.perf_counter()
    F = subproblems.factor_subproblem(2, P.n, P.omega, P.c, P.pml, P.C, part, p, kind)
    t1 = time.perf_counter()
    F.solve(rng.standard_normal((F.w, F.T)) + 0j)
    return kind, t1 - t0, time.perf_counter() - t1

def fac_only(t):
    kind, p = t
    subproblems.factor_subproblem(2, P.n, P.omega, P.c, P.pml, P.C, part, p, kind)
    return 0

if __name__ == "__main__":
    cores = os.cpu_count() or 1
    tasks = [("M", p) for p in range(1, m + 1)] + [("R", p) for p in range(2, m + 1)] + \
            [("L", p) for p in range(1, m)]
    with mp.get_context("fork").Pool(cores) as pool:
        t0 = time.perf_counter(); pool.map(fac_only, tasks, chunksize=1); fac_wall = time.perf_counter() - t0
        res = pool.map(job, tasks, chunksize=1)
    mres = [r for r in res if r[0] == "M"]
    # M-solves in parallel: their total over the cores (each solve is independent)
    m_wall = sum(r[2] for r in mres) / cores
    sweep = max(sum(r[2] for r in res if r[0] == "R"), sum(r[2] for r in res if r[0] == "L"))
    A = operator.helmholtz_matrix(2, P.n, P.omega, P.c, P.pml, P.C)
    x = P.f[..., 0].reshape(-1)
    t0 = time.perf_counter(); A @ x; t_mv = time.perf_counter() - t0
    its = %d
    v = np.asarray(x, dtype=np.complex128); w = v * (1 + 0.5j)
    t0 = time.perf_counter()
    for _ in range(its + 1):
        hij = np.vdot(v, w); w = w - hij * v
    t_gs = (time.perf_counter() - t0) * (sum(j + 1 for j in range(1, its + 1)) / (its + 1))
    print(json.dumps({"cores": cores, "factor_wall_s": fac_wall, "msolve_wall_s_per_rhs": m_wall,
                      "sweep_s_per_rhs": sweep, "matvec_s_per_rhs": t_mv, "gs_s_per_rhs": t_gs,
                      "subproblems": len(tasks)}))
""" % (ROOT, iterations)
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    fd, path = tempfile.mkstemp(suffix=".py")
    with os.fdopen(fd, "w") as fh:
        fh.write(code)
    t0 = time.perf_counter()
    try:
        r = subprocess.run([sys.executable, path], capture_output=True, text=True, env=env, timeout=900)
    finally:
        os.unlink(path)
    wall = time.perf_counter() - t0
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "kind": "oracle", "error": r.stderr[-300:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    nrhs = 32
    t_batch = d["factor_wall_s"] + nrhs * (iterations * (d["msolve_wall_s_per_rhs"] + d["sweep_s_per_rhs"] +
                                                           d["matvec_s_per_rhs"]) + d["gs_s_per_rhs"])
    return {"value": nrhs / t_batch, "unit": UNIT, "cores": d["cores"], "kind": "oracle",
            "sample": (f"every one of the {d['subproblems']} layer subproblems factored and solved once on "
                       f"{d['cores']} worker processes (1 thread each), plus one sparse matvec at n=1023; scaled to "
                       f"one 32-RHS batch with {iterations} FGMRES iterations (M-solves parallel, sweeps sequential) "
                       f"plus the Gram-Schmidt vector work of those iterations on one core"),
            "sample_wall_s": wall, "extrapolated_batch_s": t_batch, **d}


def run_reference(args):
    """The oracle arm: the CPU FP64 oracle as it stands on one host thread.
    Every step (warm-up and timed) is one bounded sample of the n=1023 workload
    (oracle_samples: one layer subproblem of each kind factored and solved, one
    matvec, the Krylov vector work), extrapolated to one 32-RHS batch with the
    oracle's own iteration count.  `value` is the median extrapolated rate over
    the timed steps; `ms_per_step` is the measured wall time of one sample."""
    its = oracle_iterations()
    its_note = "the oracle's own count (tests/golden/oracle_iterations_n1023.txt)"
    if its is None:
        its, its_note = 13, "13 (the oracle's count file is absent; the GPU path's count)"
    recs, walls, err = oracle_samples(args.warmup + args.steps, its, threads=1)
    timed = recs[args.warmup:]
    twalls = walls[args.warmup:]
    if not timed:
        return {"impl": "reference", "unavailable": f"oracle sampler failed: {err}"}
    t_batch = statistics.median(oracle_batch_seconds(r, its) for r in timed)
    value = 32 / t_batch
    ms = statistics.mean(twalls) * 1e3
    sample = (f"each step one bounded sample: oracle factor + solve of one layer subproblem of each kind (M, R, L; "
              f"3 of the 736, rotating), one sparse matvec and the Gram-Schmidt vector work of {its} FGMRES "
              f"iterations at n=1023; value extrapolated to one 32-RHS batch with {its} iterations ({its_note}); "
              f"median over {len(timed)} timed samples")
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": len(timed),
            "warmup": min(args.warmup, len(recs)), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(WORKLOAD, parallelism="cpu oracle, 1 thread"),
            "impl": "reference", "value_kind": "extrapolated from bounded samples",
            "extrapolated_batch_s": t_batch, "oracle_iterations": its,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["asp", "reference"], default="asp")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", choices=["c64", "c64sym", "c128"], default="c64",
                    help="layer factors and preconditioner applies in complex64 (mixed path, the headline), "
                         "complex64 with packed symmetric factors (half the factor memory), or complex128 (the "
                         "plain FP64 path); FGMRES is FP64 either way")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes of the layer solves (no asp_autotune before timing)")
    ap.add_argument("--no-fp64-path", action="store_true",
                    help="skip the complex128 comparison step after the complex64 headline")
    ap.add_argument("--source", choices=["point", "packet"], default="point",
                    help="right-hand sides of the n=1023 workload: Gaussian point sources or wave packets")
    ap.add_argument("--layer-widths", default="",
                    help="BMIN:BMAX -- layer widths chosen from the velocity (at least BMIN columns, up to BMAX "
                         "where it jumps heavily) instead of uniform layers of b columns")
    ap.add_argument("--slab-solver", choices=["block", "nd"], default="block",
                    help="3D workloads: block elimination over the x2 planes, or nested dissection (Section 4)")
    ap.add_argument("--pml-aux", type=int, default=0,
                    help="width of the auxiliary PMLs between layers (default: the boundary PML width)")
    ap.add_argument("--workload", choices=["n1023", "n511x32", "n255x32", "n255x1", "n95_3d", "n47_3d_slab"], default="n1023",
                    help="n511x32: the same kernels on a 2D n=511 problem with 32 RHS (profiling); "
                         "n255x32: the n=1023 workload's layer widths (PML 20, b = 4) at n=255, 4.2 GB (profiling); "
                         "n255x1: the same with one RHS (profiling); "
                         "n95_3d: the 3D slab path on the n=95 bump problem (1 RHS); "
                         "n47_3d_slab: one 3D slab with 2209-unknown blocks, 2.1 GB (profiling)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl")
    from paper_1504_04058_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    line = run_asp(args, rank, world)
    if rank == 0:
        if args.workload in ("n95_3d", "n47_3d_slab"):
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": "not run: one banded LU of a single 95^3 slab subproblem "
                                              "(162450 rows, half-bandwidth 1710) is minutes of CPU work"}
        elif not args.no_cpu_baseline:
            its_o = oracle_iterations() or line["iterations_max"]
            line["cpu_baseline"] = cpu_baseline_sample(its_o)
            line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(its_o)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
