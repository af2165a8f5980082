"""Benchmark: butterfly FIO apply on one GB300 (or N independent replicas).

Workload (one "step" = one fio_apply of the whole path: initialization,
recursion in p, switch, recursion in x, termination):
  N = 1024, q = 9, ellipse phase [2, 1, 16, 1] (eq. ex1 with the constants scaled by 1/16),
  32 right-hand sides of complex64 white noise (seeds 0..31), FP32 form, s = 3, e = 2.
The FP64 form (1 RHS, same N and q) is timed beside it.  The JSON line reports
outputs/s = N^2 * nrhs / time, the rel-L2 error against the FP64 direct sum on
512 seeded x, per-kernel times and the dominant kernel's roofline, the same
metric end to end through host buffers, and the CPU oracle timed on the host.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torchrun; every rank runs an independent replica (the
butterfly of one operator does not shard without an all-to-all; replicas only).
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

METRIC = "FIO outputs/s (N²·RHS/s) at N=1024 q=9, FP32 vs FP64 form; rel-L2 err"
N, Q, NRHS, S, E = 1024, 9, 32, 3, 2
PARAMS = (2.0, 1.0, 16.0, 1.0)
NSAMPLE = 512
FP32_PEAK_NOTE = "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (max SM clock)"
FP32_PEAK = 152 * 128 * 2 * 2.070e9


def _tf32_peak_tflops() -> float:
    """TF32 dense peak: the measured bf16 burst figure of MEASURED_PEAKS.json times the nominal
    TF32 / BF16 ratio (1.1 / 2.25 PFLOP/s); the recipe's fallback 1.9 PFLOP/s bf16 if absent."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as fh:
            bf16 = float(json.load(fh)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        bf16 = 1900.0
    return bf16 * 1.1 / 2.25


TF32_PEAK_FROM_BF16 = _tf32_peak_tflops()


def workload_config(precision="f32", nrhs=NRHS):
    return {"workload": "2D butterfly FIO apply N=%d q=%d ellipse[2,1,16,1] %d RHS %s form s=%d e=%d"
                        % (N, Q, nrhs, precision.upper(), S, E),
            "N": N, "q": Q, "nrhs": nrhs, "precision": precision, "s": S, "e": E, "phase": "ellipse/16",
            "l2": "inputs larger than L2: state 87 GB per level, no flush needed"}


# ------------------------------------------------------------------ helpers


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# DRAM bytes (read + write) per launch at the N=1024, q=9, 32-RHS workload, from ncu captures of
# the current kernels on smaller cases (inputs larger than L2), scaled by pairs x RHS.
MEASURED_TRAFFIC = {"switch": 171.0e9, "trans_p": 173.1e9, "trans_x": 173.1e9, "init": 86.7e9, "term": 87.2e9}


def kernel_flops_bytes(kind: str, info, nrhs: int) -> tuple[float, float]:
    """Algorithmic FP32 flops and HBM bytes of ONE launch of a kernel kind.

    Per pair (A,B) and RHS: translations 24q^3 + 30q^2 flops (6q^3 complex x real
    MACs of the dimension-wise Lagrange sums, 5q^2 complex modulations); switch
    8q^4 (a q^2 x q^2 complex matrix-vector product); termination
    4Mq^2 + 4M^2 q + 6(M^2 + q^2) with M = 2^s; initialization 4q^2 + 8 per
    source, box A and RHS.  Bytes: the state read and written once (complex,
    8 B in FP32) plus f or u.  Phase evaluations are not counted here."""
    q, M = info.q, 1 << info.s
    P = info.pairs_per_level
    eb = 8 if info.precision == 1 else 16
    blk = P * nrhs * q * q * eb
    NN = info.N * info.N
    if kind.startswith("trans"):
        return P * nrhs * (24 * q ** 3 + 30 * q ** 2), 2 * blk
    if kind.startswith("switch"):
        return P * nrhs * 8 * q ** 4, 2 * blk
    if kind.startswith("term"):
        return P * nrhs * (4 * M * q * q + 4 * M * M * q + 6 * (M * M + q * q)), blk + NN * nrhs * eb
    if kind.startswith("init"):
        return (4 ** info.l0) * NN * nrhs * (4 * q * q + 8), blk + NN * nrhs * eb
    return 0.0, 0.0


def _tensor_switch(kind: str, switch_impl: int) -> bool:
    return kind.startswith("switch") and switch_impl in (1, 3, 4, 5, 6)


def kernel_report(prof: dict, info, steps: int, switch_impl: int, tf32_peak=None) -> tuple[dict, dict]:
    """Per-kernel breakdown of the timed applies and the dominant kernel's roofline.

    prof: {kernel kind: (launches, total ms)} over `steps` applies of the headline plan (`info`
    its PlanInfo).  Each kernel's roofline time is the larger of its algorithmic work at the
    peak of the pipe it runs on (the FP32 FMA peak, or for a tensor-core switch the TF32 peak:
    8 q^4 flops per pair and RHS, the split-TF32 products counted once) and its algorithmic
    HBM bytes at the measured HBM bandwidth; `bound` names the larger, and frac = roofline time
    / measured time (equivalently achieved / peak in the bound's unit).  tf32_peak (flop/s):
    the measured tensor-core TF32 rate (fio_peak_probe), else the bf16 figure of
    MEASURED_PEAKS.json times the nominal TF32/BF16 ratio."""
    p_tf32 = tf32_peak if tf32_peak else TF32_PEAK_FROM_BF16 * 1e12
    tf32_src = ("tcgen05.mma kind::tf32 M=128 N=256 measured by fio_peak_probe (of measured)" if tf32_peak
                else "measured bf16 burst x nominal TF32/BF16 1.1/2.25 (of measured)")
    bw = _hbm_peak_gbs() * 1e9

    def roof_of(k, avg_ms):
        fl, by = kernel_flops_bytes(k, info, NRHS)
        tc = _tensor_switch(k, switch_impl)
        peak = p_tf32 if tc else FP32_PEAK
        t_c, t_m = fl / peak, by / bw
        hbm = t_m > t_c
        sec = avg_ms * 1e-3
        return {"bound": "hbm" if hbm else ("tensor" if tc else "alu"),
                "achieved": (by / sec / 1e9) if hbm else (fl / sec / 1e12),
                "peak": (bw / 1e9) if hbm else (peak / 1e12), "unit": "GB/s" if hbm else "TFLOP/s",
                "frac": max(t_c, t_m) / sec, "t_compute_ms": t_c * 1e3, "t_hbm_ms": t_m * 1e3,
                "pipe": "tf32 tensor" if tc else "fp32 fma", "fl": fl, "by": by}

    kernels = {}
    for k, (n, ms) in prof.items():
        avg = ms / n
        r = roof_of(k, avg)
        kernels[k] = {"launches": n, "ms_per_launch": round(avg, 3), "share": None, "bound": r["bound"],
                      "frac": round(r["frac"], 3), "tflops": round(r["fl"] / (avg * 1e-3) / 1e12, 2),
                      "gbs": round(r["by"] / (avg * 1e-3) / 1e9, 1), "pipe": r["pipe"]}
    tot = sum(v["ms_per_launch"] * v["launches"] for v in kernels.values())
    for v in kernels.values():
        v["share"] = round(v["ms_per_launch"] * v["launches"] / tot, 3)
    dom = max(kernels, key=lambda k: kernels[k]["share"])
    dom_ms = prof[dom][1] / prof[dom][0]
    r = roof_of(dom, dom_ms)
    roof = {"kernel": dom, "bound": r["bound"], "achieved": r["achieved"], "peak": r["peak"], "unit": r["unit"],
            "frac": r["frac"],
            "traffic": MEASURED_TRAFFIC.get(dom) if (info.N, info.q, NRHS) == (1024, 9, 32) else None,
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the same kernel on a smaller "
                              "case, scaled by pairs x RHS",
            "peak_source": ("MEASURED_PEAKS.json hbm_gbs (of measured)" if r["bound"] == "hbm"
                            else tf32_src if r["pipe"] == "tf32 tensor" else FP32_PEAK_NOTE + " (derived, not measured)"),
            "t_compute_ms": r["t_compute_ms"], "t_hbm_ms": r["t_hbm_ms"],
            "algorithmic_flops_per_launch": r["fl"], "algorithmic_bytes_per_launch": r["by"],
            "compute_pipe": r["pipe"], "compute_achieved_tflops": r["fl"] / (dom_ms * 1e-3) / 1e12,
            "hbm_achieved_gbs": r["by"] / (dom_ms * 1e-3) / 1e9}
    return kernels, roof


def _hbm_peak_gbs() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def apply_roofline(info, nrhs: int, ms_apply: float, probes: dict) -> dict:
    """The whole apply against its roofline time
        T_roof = max(B_min / BW, F32 / P_fp32, F64 / P_fp64, 2E / P_mufu, F_tc / P_tf32)
    with this plan's algorithmic counts (P = 2^e N^2 pairs per level, R RHS, M = 2^s):
      F32  FP32 flops of the initialization, every translation level and the termination
           (kernel_flops_bytes; the switch is not in it: it runs on the tensor cores);
      F_tc the switch's complex MACs, 8 q^4 flops per pair and RHS, split-TF32 counted once;
      E    phase evaluations e^{2 pi i theta}: q^4 per switch pair, 5 q^2 per pair of every
           translation level, 4^s N^2 + q^2 P in the initialization, (q^2 + M^2) P in the
           termination, each one sine and one cosine (2E special-function operations);
      F64  FP64 flops: none in this build's FP32 form (its phases run in double-float on the
           FP32 pipe); with FP64 phases at ~10 FP64 flops per evaluation the term is
           reported separately as t_fp64_phases_ms;
      B_min f in, u out and one state round trip at the switch: 2 N^2 R 8 + 2 P R q^2 8 bytes.
    apply_frac = T_roof / t_apply."""
    q, M, N, P, R = info.q, 1 << info.s, info.N, info.pairs_per_level, nrhs
    ntrans = (info.lm - info.l0) + (info.l1 - info.lm)
    f_init = kernel_flops_bytes("init", info, R)[0]
    f_tr = kernel_flops_bytes("trans", info, R)[0]
    f_term = kernel_flops_bytes("term", info, R)[0]
    F32 = f_init + ntrans * f_tr + f_term
    Ftc = 8 * q ** 4 * P * R
    E = q ** 4 * P + ntrans * 5 * q * q * P + (4 ** info.s) * N * N + q * q * P + (q * q + M * M) * P
    B = 2 * N * N * R * 8 + 2 * P * R * q * q * 8
    p32 = FP32_PEAK
    p64 = probes.get("fp64") if isinstance(probes.get("fp64"), float) else 1.06e12
    pmufu = probes.get("sfu") if isinstance(probes.get("sfu"), float) else 4.9e12
    t = probes.get("mma_tf32_n256")
    ptf32 = t if isinstance(t, float) else TF32_PEAK_FROM_BF16 * 1e12
    bw = _hbm_peak_gbs() * 1e9
    terms = {"hbm_ms": B / bw * 1e3, "fp32_ms": F32 / p32 * 1e3, "tf32_ms": Ftc / ptf32 * 1e3,
             "mufu_ms": 2 * E / pmufu * 1e3, "fp64_ms": 0.0}
    t_roof = max(terms.values())
    t64 = 10.0 * E / p64 * 1e3
    return {"formula": "max(B_min/BW, F32/P_fp32, F64/P_fp64, 2E/P_mufu, F_tc/P_tf32)",
            "F32": F32, "F_tc": Ftc, "E": E, "B_min": B, "F64": 0.0,
            "terms_ms": {k: round(v, 2) for k, v in terms.items()}, "t_roof_ms": round(t_roof, 2),
            "t_apply_ms": round(ms_apply, 2), "apply_frac": round(t_roof / ms_apply, 4),
            "t_fp64_phases_ms": round(t64, 1),
            "apply_frac_with_fp64_phases": round(max(t_roof, t64) / ms_apply, 4),
            "peaks": {"fp32_tflops": round(p32 / 1e12, 2), "fp32_source": "derived (152 x 128 x 2 x 2.07 GHz)",
                      "tf32_tflops": round(ptf32 / 1e12, 1),
                      "tf32_source": ("tcgen05 kind::tf32 N=256 by fio_peak_probe (of measured)" if isinstance(t, float)
                                      else "measured bf16 x 1.1/2.25 (of measured)"),
                      "hbm_gbs": round(bw / 1e9, 1), "hbm_source": "MEASURED_PEAKS.json (of measured)",
                      "mufu_per_s": pmufu, "fp64_flops": p64, "mufu_fp64_source": "fio_peak_probe on this GPU"}}


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest x over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, ms_max: float, world: int) -> float:
    """Units processed by all ranks per second, timed by the slowest rank."""
    return units_per_rank * world / (ms_max * 1e-3)


def time_steps(fn, steps, warmup, torch):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def cpu_baseline(f0: np.ndarray, nsample: int):
    """The FP64 CPU oracle as it stands: the direct sum of eq. dfio on a seeded
    sample of x of RHS 0 of the workload, all host threads.  Returns the timing
    record and the sampled reference values (used for the rel-L2 errors)."""
    from oracle import oracle as O
    from paper_0809_0719_gb300.inputs import sample_indices

    xi = sample_indices(N, nsample, 1000)
    t0 = time.perf_counter()
    ref = O.direct(N, O.ELLIPSE, list(PARAMS), f0, xi)
    dt = time.perf_counter() - t0
    rec = {"value": nsample / dt, "unit": "outputs/s", "cores": O.threads(), "kind": "oracle",
           "sample": "FP64 direct sum (eq. dfio) at %d seeded x of RHS 0 of the N=%d workload, %.1f s wall"
                     % (nsample, N, dt)}
    return rec, xi, ref


def cpu_butterfly_baseline():
    """The FP64 CPU butterfly of the oracle (the paper's algorithm, step by step, dense 2D
    Lagrange matrices), one RHS of the workload's phase, q, s and e, on all host threads and
    on one.  The full N = 1024 runs for tens of minutes, so the bounded samples are N = 256
    (all threads) and N = 128 (one thread); outputs/s = N^2 / wall time."""
    from oracle import oracle as O
    from paper_0809_0719_gb300.inputs import gaussian_sources

    nthreads = O.threads()
    rec = {"kind": "oracle", "q": Q, "s": S, "e": E, "nrhs": 1, "nproc": os.cpu_count()}
    for key, n, th in (("all_cores", 256, nthreads), ("one_core", 128, 1)):
        O.set_threads(th)
        f = gaussian_sources(n, 0)
        t0 = time.perf_counter()
        O.butterfly(n, Q, O.ELLIPSE, list(PARAMS), f, s=S, e=E)
        dt = time.perf_counter() - t0
        rec[key] = {"N": n, "cores": th, "seconds": round(dt, 2), "value": n * n / dt, "unit": "outputs/s"}
    O.set_threads(nthreads)
    return rec


def rel_err(u, xi, ref):
    a = u.reshape(-1)[xi].astype(np.complex128)
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


# ------------------------------------------------------------------ arms


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle, as it stands, on this host's cores."""
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_0809_0719_gb300.inputs import gaussian_sources, sample_indices

    O.build()
    f0 = gaussian_sources(N, 0)
    nsample = 128
    times = []
    for it in range(args.warmup + args.steps):
        xi = sample_indices(N, nsample, 2000 + it)
        t0 = time.perf_counter()
        O.direct(N, O.ELLIPSE, list(PARAMS), f0, xi)
        if it >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    v = nsample / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "outputs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(),
            "cpu_baseline": {"value": v, "unit": "outputs/s", "cores": O.threads(), "kind": "oracle",
                             "sample": "FP64 direct sum at %d seeded x per step of RHS 0, N=%d" % (nsample, N)},
            "e2e": {"value": v, "unit": "outputs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, dist):
    import torch

    from paper_0809_0719_gb300 import fio
    from paper_0809_0719_gb300.inputs import gaussian_batch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def tmax(x):
        return max_over_ranks(x, dist, dev)

    F = gaussian_batch(N, range(NRHS))
    # ---- FP32 form, 32 RHS (the headline)
    plan = fio.Plan(N, Q, "ellipse", PARAMS, "f32", nrhs_max=NRHS, s=S, e=E)
    f = torch.from_numpy(F).to(torch.complex64).to(dev)
    u = torch.empty_like(f)
    step = lambda: plan.apply(f, out=u)
    for _ in range(args.warmup):
        step()
    barrier()
    plan.profile(True)
    with ClockSampler(local) as clk:
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            step()
        b.record()
        barrier()
    plan.profile(False)
    ms32 = tmax(a.elapsed_time(b) / args.steps)
    prof = plan.profile_read()
    launches_per_step = plan.kernel_launches(NRHS)
    switch_impl = plan.info.switch_impl
    trans_rs = (plan.info.trans_rs, plan.info.trans_rs_x)
    sw_tile = plan.info.switch_rhs_tile
    u32 = u[0].cpu().numpy()
    # the adjoint apply (backward of the differentiable apply) on the same plan, outside the timed region
    fbar = torch.empty_like(f)
    ms_adj = tmax(time_steps(lambda: plan.adjoint(u, out=fbar), max(1, args.steps), max(3, args.warmup), torch))
    # dot test at this size: <g, B f> against <B^H g, f> over all 32 RHS, g = the seeds 100..131
    gdot = torch.from_numpy(gaussian_batch(N, range(100, 100 + NRHS))).to(torch.complex64).to(dev)
    plan.apply(f, out=u)
    plan.adjoint(gdot, out=fbar)
    g64, bf = gdot.to(torch.complex128).flatten(), u.to(torch.complex128).flatten()
    da = torch.vdot(g64, bf)
    db = torch.vdot(fbar.to(torch.complex128).flatten(), f.to(torch.complex128).flatten())
    dot = {"rel_to_inner_product": abs(da - db).item() / abs(da).item(),
           "rel_to_norms": abs(da - db).item() / (g64.norm() * bf.norm()).item()}
    del fbar, gdot, g64, bf

    # ---- end to end through host buffers (pinned), copies inside the timed region
    fh = torch.from_numpy(F).to(torch.complex64).pin_memory()
    uh = torch.empty_like(fh).pin_memory()
    e2e_step = lambda: plan.apply_host(fh, uh)
    for _ in range(max(1, args.warmup // 2)):
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    barrier()
    e2e_ms = tmax((time.perf_counter() - t0) * 1e3 / args.steps)
    info = plan.info
    # ---- variable amplitude (eq. allfio): 4 separated terms x 8 inputs = the plan's 32 RHS
    nt, na = 4, NRHS // 4
    ga = torch.ones(nt, N, N, dtype=torch.complex64, device=dev) * 0.5
    ha = torch.ones(nt, N, N, dtype=torch.complex64, device=dev) * 0.5
    fa = f[:na].contiguous()
    ua = torch.empty_like(fa)
    ms_amp = tmax(time_steps(lambda: plan.apply_amplitude(fa, ga, ha, out=ua), max(1, args.steps),
                             max(3, args.warmup), torch))
    del ga, ha, fa, ua
    plan.close()
    del f, u, fh, uh
    torch.cuda.empty_cache()

    # ---- FP64 form, 1 RHS, same N and q
    plan64 = fio.Plan(N, Q, "ellipse", PARAMS, "f64", nrhs_max=1, s=S, e=E)
    f64 = torch.from_numpy(F[:1]).to(dev)
    u64 = torch.empty_like(f64)
    # a side measurement (5 s per apply): a few timed applies after one warm-up
    ms64 = tmax(time_steps(lambda: plan64.apply(f64, out=u64), max(1, min(3, args.steps // 2)), 1, torch))
    u64h = u64[0].cpu().numpy()
    plan64.close()
    del f64, u64
    torch.cuda.empty_cache()

    # ---- the wave propagator as a sum of two FIOs (every rank: replicas)
    wave = run_wave(args, dev, tmax, world)

    # ---- the three-dimensional butterfly (every rank: replicas)
    b3 = run_3d(args, dev, tmax, world, with_errors=rank == 0)

    # ---- the uneven batch of plans (every rank: replicas)
    ub = run_uneven_batch(args, dev, with_errors=rank == 0) if args.batch else None

    if rank != 0:
        return
    out32 = whole_job_rate(N * N * NRHS, ms32, world)
    out64 = whole_job_rate(N * N, ms64, world)

    probes = {}
    for kind in ("fp32", "fp64", "sfu", "mma_tf32_n64", "mma_tf32_n256", "mma_bf16_n256"):
        try:
            probes[kind] = fio.peak_probe(kind)
        except Exception as ex:  # measurement aid only
            probes[kind] = str(ex)
    tf32 = probes.get("mma_tf32_n256")
    kernels, roof = kernel_report(prof, info, args.steps, switch_impl,
                                  tf32_peak=tf32 if isinstance(tf32, float) else None)
    roof["apply"] = apply_roofline(info, NRHS, ms32, probes)

    base, xi, ref = cpu_baseline(F[0], NSAMPLE)
    base["butterfly"] = cpu_butterfly_baseline()
    err32 = rel_err(u32, xi, ref)
    err64 = rel_err(u64h, xi, ref)
    line = {
        "metric": METRIC, "value": out32, "unit": "outputs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (white-noise complex64 sources, seeds 0..31)",
        "config": dict(workload_config(), parallelism="replicas" if world > 1 else "single GPU"),
        "e2e": {"value": whole_job_rate(N * N * NRHS, e2e_ms, world), "unit": "outputs/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": N * N * NRHS * 8, "d2h_bytes_per_step": N * N * NRHS * 8,
                "api": "fio_apply_host (pinned host buffers)"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
        "cpu_baseline": base,
        "switch_kernel": ["fp32_fma", "tcgen05_tf32_smem_a", "fp32_fma_warp_specialised",
                          "tcgen05_tf32_tmem_a", "tcgen05_tf32_tmem_a_wide_n", "tcgen05_tf32x3_tmem_a",
                          "tcgen05_tf32x3_tmem_a_wide_n"][switch_impl] + " (plan autotuner)",
        "translation_rhs_subtile": trans_rs, "switch_rhs_tile": sw_tile,
        "peak_probes": probes,
        "uneven_batch": ub,
        "wave": wave,
        "butterfly_3d": b3,
        "amplitude": {"value": whole_job_rate(N * N * na, ms_amp, world), "unit": "outputs/s", "ms_per_step": ms_amp,
                      "what": "fio_apply_amplitude: %d inputs x %d separated amplitude terms (eq. allfio) as one "
                              "32-RHS butterfly" % (na, nt)},
        "kernels": kernels,
        "roofline": roof,
        # accuracy last, so that the end of the line carries it
        "adjoint": {"value": whole_job_rate(N * N * NRHS, ms_adj, world), "unit": "outputs/s", "ms_per_step": ms_adj,
                    "what": "fio_apply_adjoint on the same plan (32 RHS)"},
        "fp64_form": {"value": out64, "unit": "outputs/s", "ms_per_step": ms64, "nrhs": 1, "dtype": "f64",
                      "rel_l2_err": err64},
        "speedup_f32_vs_f64_form": out32 / out64,
        "dot_test": dot,
        "rel_l2_err": err32,
        "accuracy_bar": "FP32 err <= max(2 x FP64-form err, 1e-5) on 512 seeded x vs the FP64 direct sum",
        "accuracy_bar_met": err32 <= max(2 * err64, 1e-5),
    }
    print(json.dumps(line), flush=True)


WAVE_N = 512
WAVE_TIMES = (0.25, 0.5, 0.75, 1.0)


def run_wave(args, dev, tmax, world):
    """fio_apply_wave_series: u(t) = (B_+t f + B_-t f)/2 with the circle phases x.k +- c(x)|k|t,
    c(x) = (3 + sin 2 pi x1 sin 2 pi x2)/20, at four times t from ONE plan (Sec. 1), N = WAVE_N,
    q = 9, 32 RHS, FP32 form: 8 butterflies per step on one plan's tables and state.  Reports
    outputs/s (times x N^2 x RHS per second) and the device memory against one plan per phase.
    A failure is reported in the result instead of raised, so the headline line is printed
    whatever happens here."""
    import torch

    from paper_0809_0719_gb300 import fio
    from paper_0809_0719_gb300.inputs import gaussian_batch

    n = WAVE_N
    plan = None
    try:
        plan = fio.Plan(n, Q, "circle", (3.0, 1.0, 20.0, 1.0), "f32", nrhs_max=NRHS, s=S, e=E)
        f = torch.from_numpy(gaussian_batch(n, range(NRHS))).to(torch.complex64).to(dev)
        u = torch.empty((len(WAVE_TIMES),) + tuple(f.shape), dtype=f.dtype, device=dev)
        ms = tmax(time_steps(lambda: fio.apply_wave_series(plan, WAVE_TIMES, f, out=u), max(1, args.steps // 2),
                             max(3, args.warmup), torch))
        plan.check()
        one = plan.info.table_bytes + plan.info.state_bytes + n * n * NRHS * 8
        del f, u
        return {"workload": "wave propagator u(t) = (B+t f + B-t f)/2, phases x.k +- c(x)|k|t, c = (3 + sin sin)/20, "
                            "t in %s, N=%d q=%d %d RHS, FP32 form" % (list(WAVE_TIMES), n, Q, NRHS),
                "value": whole_job_rate(n * n * NRHS * len(WAVE_TIMES), ms, world), "unit": "outputs/s",
                "ms_per_step": ms, "api": "fio_apply_wave_series (one plan's tables and state for all phases)",
                "device_bytes": one, "device_bytes_one_plan_per_phase": 2 * len(WAVE_TIMES) * (one - n * n * NRHS * 8)}
    except Exception as ex:  # reported, not raised
        return {"error": "%s: %s" % (type(ex).__name__, ex)}
    finally:
        if plan is not None:
            plan.close()
        torch.cuda.empty_cache()


N3, Q3, E3 = 64, 7, 1
EX3 = (3.0, 1.0, 4.0, 1.0)


def run_3d(args, dev, tmax, world, with_errors=True):
    """The three-dimensional butterfly (fio3_apply, FP64) on Table 3's workload: N = 64, q = 7,
    the phase of eq. ex3 (c(x) = (3 + sin sin sin)/4), white-noise sources, one RHS, e = 1,
    s = 3.  Outputs/s = N^3 / time; the error is eq. err on 64 seeded x against the oracle's
    3D direct sum (the reference values of the CPU-baseline leg).  A failure is reported in
    the result instead of raised."""
    import torch

    from paper_0809_0719_gb300 import fio

    plan = None
    try:
        plan = fio.Plan3(N3, Q3, "sphere", EX3, nrhs_max=1, s=3, e=E3)
        rng = np.random.default_rng(0)
        F = rng.standard_normal((N3, N3, N3)) + 1j * rng.standard_normal((N3, N3, N3))
        f = torch.from_numpy(F[None]).to(dev)
        u = torch.empty_like(f)
        ms = tmax(time_steps(lambda: plan.apply(f, out=u), 1, 1, torch))
        rec = {"workload": "3D butterfly N=%d q=%d eq. ex3, e=%d s=3, 1 RHS, FP64 form (Table 3)" % (N3, Q3, E3),
               "value": whole_job_rate(N3 ** 3, ms, world), "unit": "outputs/s", "ms_per_step": ms,
               "api": "fio3_apply", "paper_table3_eps_a": 3.32e-3}
        if with_errors:
            from oracle import oracle as O

            xi = np.sort(np.random.default_rng(1000).choice(N3 ** 3, 64, replace=False)).astype(np.int64)
            t0 = time.perf_counter()
            ref = O.direct3(N3, O.SPHERE, list(EX3), F, xi)
            dt = time.perf_counter() - t0
            a = u.cpu().numpy().reshape(-1)[xi]
            rec["rel_l2_err"] = float(np.linalg.norm(a - ref) / np.linalg.norm(ref))
            rec["cpu_direct_sum"] = {"value": 64 / dt, "unit": "outputs/s", "cores": O.threads(),
                                     "sample": "FP64 3D direct sum at 64 seeded x"}
        del f, u
        return rec
    except Exception as ex:  # reported, not raised
        return {"error": "%s: %s" % (type(ex).__name__, ex)}
    finally:
        if plan is not None:
            plan.close()
        torch.cuda.empty_cache()


def run_uneven_batch(args, dev, with_errors=True):
    """The uneven batch: 96 FP32 plans (N in {64, 128, 256, 512} drawn with seed 4,
    q in {5, 7, 9}, 1-8 RHS, ellipse / c(x)|k| phases alternating) applied through
    fio_batch_apply (one persistent launch per step and q-group, CUDA graph,
    autotuned grids).  Returns aggregate outputs/s, per-kernel-kind times from one
    eager profiled pass, and each plan's rel-L2 error (RHS 0) against the FP64-form
    butterfly of the same plan parameters."""
    import torch

    from paper_0809_0719_gb300 import fio
    from paper_0809_0719_gb300.inputs import uneven_batch_sources, uneven_batch_specs

    specs = uneven_batch_specs()
    t0 = time.perf_counter()
    plans = [fio.Plan(sp["N"], sp["q"], sp["phase"], sp["params"], "f32", nrhs_max=sp["nrhs"]) for sp in specs]
    batch = fio.Batch(plans, [sp["nrhs"] for sp in specs], tune=True)
    setup_s = time.perf_counter() - t0
    xs = [torch.from_numpy(uneven_batch_sources(sp, i)).to(torch.complex64) for i, sp in enumerate(specs)]
    x = batch.pack([t.to(dev) for t in xs])
    y = torch.empty_like(x)
    ms = time_steps(lambda: batch.apply(x, out=y), args.steps, args.warmup, torch)
    outputs = batch.offsets[-1]
    prof = batch.profile(x)
    rec = {"workload": "96 FP32 plans, N from {64,128,256,512} (seed 4), q from {5,7,9}, 1-8 RHS, "
                       "ellipse[2,1,16,1] / circle[3,1,20,1] alternating, s=3 e=2",
           "value": outputs / (ms * 1e-3), "unit": "outputs/s", "ms_per_step": ms, "outputs_per_step": outputs,
           "plans": len(specs), "groups": batch.info.ngroups, "launches_per_step": batch.info.launches_fwd + 1,
           "graph": "one CUDA graph per apply, groups on %s branches"
                    % ("parallel" if batch.info.parallel_groups else "serial"),
           "setup_s": setup_s, "tune_ms": batch.info.tune_ms,
           "kernels": {k: {"launches": n, "ms": t} for k, (n, t) in prof.items()}}
    ys = [t[0].cpu().numpy() for t in batch.unpack(y)]
    batch.close()
    for p in plans:
        p.close()
    del x, y
    torch.cuda.empty_cache()
    if with_errors:
        errs = []
        for i, sp in enumerate(specs):
            p64 = fio.Plan(sp["N"], sp["q"], sp["phase"], sp["params"], "f64", nrhs_max=1)
            u = p64.apply(xs[i][:1].to(torch.complex128).to(dev))[0].cpu().numpy()
            p64.close()
            errs.append(float(np.linalg.norm(ys[i] - u) / np.linalg.norm(u)))
        rec["rel_l2_err_vs_fp64_butterfly"] = {"max": max(errs), "median": statistics.median(errs),
                                               "plans": len(errs)}
    return rec


def run_small(args):
    """--case small: only the timed applies of a small FP32 plan (default N=256, q=9,
    16 RHS: 5.4 GB of state), forward then adjoint; the case the ncu captures use."""
    import torch

    from paper_0809_0719_gb300 import fio
    from paper_0809_0719_gb300.inputs import gaussian_batch

    n, r = args.small_n, args.small_nrhs
    plan = fio.Plan(n, Q, "ellipse", PARAMS, "f32", nrhs_max=r, s=S, e=E)
    if args.switch_impl >= 0 or args.trans_rs > 0 or args.trans_rs_x > 0:
        plan.set_tuning(args.switch_impl, -1, args.trans_rs if args.trans_rs > 0 else -1,
                        args.trans_rs_x if args.trans_rs_x > 0 else -1)
    f = torch.from_numpy(gaussian_batch(n, range(r))).to(torch.complex64).cuda()
    u = torch.empty_like(f)
    ms = time_steps(lambda: plan.apply(f, out=u), args.steps, args.warmup, torch)
    msa = time_steps(lambda: plan.adjoint(u, out=f), args.steps, args.warmup, torch)
    plan.profile(True)
    plan.apply(f, out=u)
    plan.adjoint(u, out=f)
    prof = plan.profile_read()
    plan.profile(False)
    print(json.dumps({"case": "small", "N": n, "q": Q, "nrhs": r, "switch_impl": plan.info.switch_impl,
                      "trans_rs": plan.info.trans_rs, "trans_rs_x": plan.info.trans_rs_x, "ms_forward": ms, "ms_adjoint": msa,
                      "kernels_ms": {k: round(t / c, 3) for k, (c, t) in prof.items()},
                      "launches_per_apply": plan.kernel_launches(r)}), flush=True)
    plan.close()


def run_eq_sweep(args):
    """--case eq: the cost of the accuracy knobs.  For the angular refinement e in {1, 2, 3} and
    q in {7, 9, 11} (s = 3, ellipse [2, 1, 16, 1], N = --small-n): the FP32 apply time of 32 RHS
    (CUDA events, the plan's autotuned kernels) and the relative l2 error of RHS 0 on 512 seeded x
    against the FP64 direct sum of eq. dfio (fio_direct), for the FP32 form and the FP64 form."""
    import torch

    from paper_0809_0719_gb300 import fio
    from paper_0809_0719_gb300.inputs import gaussian_batch, sample_indices

    n, r = args.small_n, NRHS
    F = gaussian_batch(n, range(r)).astype(np.complex64)
    f = torch.from_numpy(F).cuda()
    xi = torch.from_numpy(sample_indices(n, NSAMPLE, 1000)).cuda()
    rows = []
    ref = None
    for e in (1, 2, 3):
        for q in (7, 9, 11):
            plan = fio.Plan(n, q, "ellipse", PARAMS, "f32", nrhs_max=r, s=S, e=e)
            if ref is None:  # the direct sum does not depend on the plan's q and e
                ref = plan.direct(f[:1], xi)[0].cpu().numpy()  # FP64 sums of the complex64 inputs
            u = torch.empty_like(f)
            ms = time_steps(lambda: plan.apply(f, out=u), args.steps, args.warmup, torch)
            err32 = float(np.linalg.norm(u[0].reshape(-1)[xi].cpu().numpy() - ref) / np.linalg.norm(ref))
            plan.close()
            p64 = fio.Plan(n, q, "ellipse", PARAMS, "f64", nrhs_max=1, s=S, e=e)
            u64 = p64.apply(f[:1].to(torch.complex128))
            err64 = float(np.linalg.norm(u64[0].reshape(-1)[xi].cpu().numpy() - ref) / np.linalg.norm(ref))
            p64.close()
            rows.append({"e": e, "q": q, "ms_f32_32rhs": round(ms, 3), "rel_l2_err_f32": err32,
                         "rel_l2_err_f64": err64})
            torch.cuda.empty_cache()
    print(json.dumps({"case": "eq", "N": n, "nrhs": r, "s": S, "phase": "ellipse [2,1,16,1]", "rows": rows}),
          flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--case", default="full", choices=["full", "small", "batch", "eq"],
                    help="small: N=256 q=9 16-RHS applies only (for profiler captures); batch: the uneven batch "
                         "only; eq: apply time and error over e in {1,2,3} x q in {7,9,11} at N=--small-n")
    ap.add_argument("--no-batch", dest="batch", action="store_false", help="skip the uneven-batch measurement")
    ap.add_argument("--small-n", type=int, default=256, help="--case small: N")
    ap.add_argument("--small-nrhs", type=int, default=16, help="--case small: right-hand sides")
    ap.add_argument("--switch-impl", type=int, default=-1,
                    help="--case small: force the FP32 switch kernel (fio_plan_set_tuning), -1 = autotuner")
    ap.add_argument("--trans-rs", type=int, default=0,
                    help="--case small: force the FP32 translation kernel (2, 4, 8 RHS subtiles; 32, 33 "
                         "register-tiled), 0 = autotuner")
    ap.add_argument("--trans-rs-x", type=int, default=0,
                    help="--case small: force the x-shape translation kernel (2, 4, 8; 32 register-tiled)")
    args = ap.parse_args()
    if args.case == "small":
        run_small(args)
        return
    if args.case == "eq":
        run_eq_sweep(args)
        return
    if args.case == "batch":
        import torch

        print(json.dumps({"case": "batch", **run_uneven_batch(args, torch.device("cuda", 0), with_errors=False)}),
              flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
