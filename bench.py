#!/usr/bin/env python3
"""Benchmark of the quasistatic LSPR boundary-element hot path on GB300.

Metric: wavelength solves per second (lambda-solves/s) at sigma_ext error <= 1e-4
relative to the plain FP64 solve; the matvec rate (G-interactions/s: one
(target, source Gauss node, wavelength) evaluation of G and dG/dn on complex
data) is reported alongside.

One step = the whole hot path for one batch of synthetic input: mesh upload and
panel/near-singular precompute, Morton sort + octree + interaction lists, FP64
right-hand side, GMRES with the treecode matvec, dipole and sigma_ext.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload sphere20480]
  python bench.py --impl reference ...   (the CPU oracle on a bounded sample)

Multi-GPU: wavelengths and geometries are independent, so N ranks run N
independent replicas of the step (weak scaling, no data-path collective); the
barrier and max-over-ranks timing use torch.distributed.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1812_10722_gb300 import inputs as I  # noqa: E402

WORKLOADS = {
    # 20480-panel silver sphere, single wavelength 380 nm, FP32 treecode GMRES with refinement to 1e-6; the
    # treecode parameters (theta, P, Ncrit) are autotuned under the sigma_ext <= 1e-4 bound of the metric
    "sphere20480": dict(sub=5, R=10.0, lam=[380.0], mode="tree_fp32", tol=1e-6, theta=0.5, P=6, Ncrit=300,
                        K=4, K_fine=19, N_k=9, restart=50, refine=True, autotune=True),
    # the same at the literal P=6, theta=0.5, Ncrit=300 (sigma_ext deviates 7e-4 from the FP64 oracle there)
    "sphere20480_p6": dict(sub=5, R=10.0, lam=[380.0], mode="tree_fp32", tol=1e-6, theta=0.5, P=6, Ncrit=300,
                           K=4, K_fine=19, N_k=9, restart=50, refine=True),
    # the plain FP64 treecode, one wavelength at a time (baseline of the mixed-precision form)
    "sphere20480_fp64": dict(sub=5, R=10.0, lam=[380.0], mode="tree_fp64", tol=1e-6, theta=0.5, P=6, Ncrit=300,
                             K=4, K_fine=19, N_k=9, restart=50, refine=False, autotune=True),
    # 1280-panel sphere, direct FP64 matvec, GMRES 1e-8
    "sphere1280": dict(sub=3, R=10.0, lam=[380.0], mode="direct_fp64", tol=1e-8, theta=0.5, P=6, Ncrit=300,
                       K=4, K_fine=19, N_k=9, restart=100, refine=False),
    # 20480-panel sphere, 16 wavelengths over 350-420 nm in one batched solve
    "sphere20480_sweep16": dict(sub=5, R=10.0, lam=list(I.wavelengths(350, 420, 16)), mode="tree_fp32", tol=1e-6,
                                theta=0.5, P=6, Ncrit=300, K=4, K_fine=19, N_k=9, restart=50, refine=True,
                                autotune=True),
    # sensor-analyte: 81920-panel sphere plus two 32768-panel protein-like analytes (eps 2.25) at 1 nm on
    # +-z, 32 wavelengths over 370-400 nm in one batched solve; the resonance shift against the bare sphere
    "sensor_c4": dict(sub=6, R=10.0, lam=list(I.wavelengths(370, 400, 32)), mode="tree_fp32", tol=1e-6,
                      theta=0.5, P=6, Ncrit=300, K=4, K_fine=19, N_k=9, restart=50, refine=True, autotune=True,
                      analytes=(("+z", 1.0), ("-z", 1.0)), analyte_sub=6, eps_analyte=2.25, tune_lams=1),
    # 81920-panel sphere, 64 wavelengths over 350-420 nm in one batched solve
    "sphere81920_sweep64": dict(sub=6, R=10.0, lam=list(I.wavelengths(350, 420, 64)), mode="tree_fp32", tol=1e-6,
                                theta=0.5, P=6, Ncrit=300, K=4, K_fine=19, N_k=9, restart=50, refine=True,
                                autotune=True),
}


def tuning_wavelengths(lam: np.ndarray, count: int = 4) -> np.ndarray:
    """Wavelengths the autotuner checks: the one nearest the sphere's dipole resonance
    (smallest |eps + 2 eps_m|, where the solve amplifies operator errors most) and, with
    count 4, three more spread over the sweep."""
    lam = np.asarray(lam, float)
    k = int(np.argmin(np.abs(I.drude_eps(lam) + 2 * I.EPS_WATER)))
    if count == 1:
        return lam[k:k + 1]
    if len(lam) <= 4:
        return lam
    pick = {k, 0, len(lam) // 2, len(lam) - 1}
    return lam[sorted(pick)]


def workload_geometry(wl):
    """(verts, tris, surf or None) of a workload: the sphere, or the sphere plus analytes."""
    if wl.get("analytes"):
        return I.sensor_geometry(wl["sub"], wl["R"], wl["analytes"], wl["analyte_sub"])
    v, t = I.icosphere(wl["sub"], wl["R"])
    return v, t, None


def workload_eps(wl, lam):
    """[B] or [B, S] permittivities: Drude silver for the sphere, eps_analyte for analytes."""
    e = I.drude_eps(np.asarray(lam, float))
    if not wl.get("analytes"):
        return e
    S = 1 + len(wl["analytes"])
    out = np.full((len(e), S), complex(wl["eps_analyte"]), np.complex128)
    out[:, 0] = e
    return out


def resonance_peak(lam, sigma):
    """Wavelength of the largest sigma_ext from a parabola through the 3 samples around it."""
    k = int(np.clip(np.argmax(sigma), 1, len(sigma) - 2))
    a, b, _ = np.polyfit(lam[k - 1:k + 2], sigma[k - 1:k + 2], 2)
    return float(-b / (2 * a))


L2_BYTES = 129 * 2 ** 20
P2P_GEN_FLOPS = 16      # per (target, source) pair, generation of G and dG/dn (FMA = 2 flops)
P2P_FP32_INSTR = 16     # FP32-pipe instructions per pair
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64
TF32_PER_BF16 = 1.1 / 2.25  # nominal dense tensor rates, TF32 over BF16
# DRAM bytes (read + write) per launch of the current kernels, from the ncu captures summarised in
# profiles/{p2p,m2p,p2m}_fp32_sphere20480.md (dram__bytes.sum.per_second x gpu__time_duration.sum), keyed by
# workload, kernel and treecode parameters (theta, P, Ncrit); None where no capture matches
# (the P2P entry was dropped when its contraction became packed FFMA2: the kernel changed since the
# capture, so its traffic is unknown until the next one)
NCU_TRAFFIC = {("sphere20480", "m2p", 0.4, 5, 256): 2.410e6, ("sphere20480", "p2m", 0.4, 5, 256): 5.097e6}


def m2p_flops(P: int, B: int = 1) -> int:
    """Flops per (target, box) M2P evaluation: the coefficient recurrence (once, whatever B)
    plus the 4-channel dot with the moments of each of the B right-hand sides (FMA = 2)."""
    terms = [(a, b, n - a - b) for n in range(P + 1) for a in range(n, -1, -1) for b in range(n - a, -1, -1)]
    f = 3 + 5 + 1   # R components, r^2, 1/r^2
    for k in terms[1:]:
        m1 = sum(1 for d in range(3) if k[d] >= 1)
        m2 = sum(1 for d in range(3) if k[d] >= 2)
        f += 2 * m1 + m2 + 3
    return f + 8 * len(terms) * B


def p2p_flops(B: int = 1) -> int:
    """Flops per (target, source) pair: G and dG/dn generated once (16), then two kernels
    times 2 real channels of each right-hand side (8 B)."""
    return P2P_GEN_FLOPS + 8 * B


def fp32_peak_tflops(mhz: float) -> float:
    # 152 SMs x 128 FP32 lanes x 2 flops (FMA) per clock
    return 152 * 128 * 2 * mhz * 1e6 / 1e12


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "fallback": True}


# ----------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ our GPU arm
def run_ours(args, wl, rank, world, local_rank):
    import torch
    from paper_1812_10722_gb300 import lspr
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    verts, tris, surf = workload_geometry(wl)
    lam = np.asarray(wl["lam"], float)
    eps = workload_eps(wl, lam)
    em = I.EPS_WATER
    B = len(lam)
    v_d = torch.as_tensor(verts, device=dev)
    t_d = torch.as_tensor(tris, device=dev)
    s_d = None if surf is None else torch.as_tensor(surf, device=dev)
    stream = torch.cuda.current_stream(dev)
    ctx = lspr.Context(local_rank, stream.cuda_stream)
    if args.no_tc:
        ctx.set_tensor_cores(False)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    tune = None
    if wl.get("autotune") and wl["mode"].startswith("tree"):
        # once per geometry, before the timed region: treecode parameters under the sigma_ext bound
        ctx.mesh_upload(v_d, t_d, wl["K"], wl["K_fine"], wl["N_k"], surf_id=s_d)
        lt = tuning_wavelengths(lam, wl.get("tune_lams", 4))
        t0 = time.perf_counter()
        tune = ctx.autotune(workload_eps(wl, lt), em, lt, target_rel_err=1e-4, tol=min(wl["tol"], 1e-8),
                            restart=wl["restart"], mode=wl["mode"], refine=1 if wl["refine"] else 0,
                            coarse=len(tris) > 50000)
        tune["seconds"] = round(time.perf_counter() - t0, 2)
        tune["wavelengths"] = [float(x) for x in lt]
        wl["theta"], wl["P"], wl["Ncrit"] = tune["theta"], tune["P"], tune["Ncrit"]

    def step(host: bool):
        if host:
            ctx.mesh_upload(verts, tris, wl["K"], wl["K_fine"], wl["N_k"], surf_id=surf)
        else:
            ctx.mesh_upload(v_d, t_d, wl["K"], wl["K_fine"], wl["N_k"], surf_id=s_d)
        if wl["mode"].startswith("tree"):
            ctx.tree_build(wl["theta"], wl["P"], wl["Ncrit"])
        return ctx.solve(eps, em, lam, tol=wl["tol"], restart=wl["restart"], maxiter=2000, mode=wl["mode"],
                         refine=wl["refine"])

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step(False)
    barrier()
    # ---- timed region: inputs resident in HBM, L2 flushed between steps
    sampler = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else local_rank)
    sampler.start()
    n0 = ctx_launches(ctx)
    total_ms = 0.0
    iters = []
    mvs = []   # operator applications x right-hand sides per step (GMRES, residuals, right-hand side)
    sig = None
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = step(False)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        iters.append(int(r.iterations.max()))
        mvs.append(int(r.matvecs))
        sig = r.sigma_ext
    launches = ctx_launches(ctx) - n0
    clocks = sampler.stop()
    graph_stats = ctx.graph_stats()
    barrier()
    # ---- instrumented replay of the timed steps: CUDA events around every kernel on the
    # stream it runs on.  Events cannot sit inside the graph loops of the Arnoldi cycles, so
    # timing switches the solver to host-driven cycles; the kernels and inputs are the same.
    ctx.set_timing(True)
    replay_ms = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(False)
        e1.record(stream)
        e1.synchronize()
        replay_ms += e0.elapsed_time(e1)
    ktime = ctx.timing()
    ctx.set_timing(False)
    barrier()
    info = ctx.info()
    t_max = total_ms
    if world > 1:
        tt = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_max = float(tt.item())
    value = B * args.steps * world / (t_max / 1e3)

    # ---- accuracy: the same step with the plain FP64 treecode (same P, theta) and the oracle's stored value
    acc = {}
    if wl["mode"] == "tree_fp32":
        # large batches: the wavelength nearest the resonance (the FP64 treecode is ~30x slower)
        ka = [int(np.argmin(np.abs(I.drude_eps(lam) + 2 * em)))] if B > 4 else list(range(B))
        r64 = ctx.solve(eps[ka], em, lam[ka], tol=min(wl["tol"], 1e-8), restart=wl["restart"], maxiter=2000,
                        mode="tree_fp64")
        acc["sigma_rel_err_vs_fp64_treecode"] = float(np.max(np.abs(sig[ka] - r64.sigma_ext) / r64.sigma_ext))
        acc["checked_wavelengths_nm"] = [float(lam[k]) for k in ka]
    if wl.get("analytes"):
        # resonance shift: the same sweep on the bare sphere, peaks from parabolic fits
        vb, tb = I.icosphere(wl["sub"], wl["R"])
        ctx.mesh_upload(vb, tb, wl["K"], wl["K_fine"], wl["N_k"])
        ctx.tree_build(wl["theta"], wl["P"], wl["Ncrit"])
        rb = ctx.solve(I.drude_eps(lam), em, lam, tol=wl["tol"], restart=wl["restart"], maxiter=2000,
                       mode=wl["mode"], refine=wl["refine"])
        acc["resonance"] = {"peak_nm": resonance_peak(lam, sig), "bare_sphere_peak_nm": resonance_peak(lam, rb.sigma_ext),
                            "shift_nm": resonance_peak(lam, sig) - resonance_peak(lam, rb.sigma_ext),
                            "peak_sigma_nm2": float(np.max(sig)), "bare_peak_sigma_nm2": float(np.max(rb.sigma_ext))}
    gold = os.path.join(ROOT, "tests", "golden", f"sphere{info['n_panels']}_l380.json")
    if B == 1 and lam[0] == 380.0 and os.path.exists(gold):
        with open(gold) as f:
            g = json.load(f)
        acc["sigma_rel_err_vs_oracle"] = float(abs(sig[0] - g["sigma_ext_nm2"]) / g["sigma_ext_nm2"])

    # ---- end to end through the public API with host buffers
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = step(True)
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    if world > 1:
        tt = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(tt.item())
    h2d = verts.nbytes + tris.nbytes + eps.astype(np.complex128).nbytes + lam.nbytes + 24 + (
        0 if surf is None else surf.nbytes)
    d2h = B * (3 * 16 + 8)

    # ---- roofline of the dominant kernel (CUDA events around every launch in the timed region)
    peaks = load_peaks()
    mhz = (clocks or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    kernels = {}
    matvecs_per_step = None
    for name in ("p2p", "m2p", "p2m", "near_assembly", "gmres", "tree", "mesh", "p2p_fp64", "m2p_fp64", "p2m_fp64",
                 "weights", "p2p_ff", "m2p_ff", "p2m_ff"):
        ms, n = ktime[name]
        if n:
            kernels[name] = {"ms_total": round(ms, 4), "launches": n, "ms_per_launch": ms / n,
                             "share_of_step": round(ms / replay_ms, 4)}
    pairs = info["n_p2p_pairs"] if wl["mode"].startswith("tree") else info["n_panels"] * info["n_sources"]
    roof = None
    # dominant single kernel: the far-field evaluations (the "gmres" slot groups many small
    # vector kernels, and P2M's event time overlaps the concurrent P2P on the side stream)
    dom = max((k for k in kernels if k in ("p2p", "m2p", "p2p_fp64", "m2p_fp64", "p2p_ff", "m2p_ff")),
              key=lambda k: kernels[k]["ms_total"], default=None)
    fp32 = wl["mode"].endswith("fp32")
    peak_fp32 = fp32_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
    if "p2p" in kernels:
        k = kernels["p2p"]
        k["algorithmic_tflops"] = pairs * p2p_flops(B) / (k["ms_per_launch"] * 1e-3) / 1e12
        k["pairs_per_launch"] = pairs
    m2p_tc = B > 1 and fp32 and not args.no_tc   # the FP32 M2P of several right-hand sides runs on tcgen05
    if "m2p" in kernels:
        k = kernels["m2p"]
        k["algorithmic_tflops"] = info["n_m2p_pairs"] * kernel_targets(info) * m2p_flops(wl["P"], B) / (
            k["ms_per_launch"] * 1e-3) / 1e12
        k["path"] = "tcgen05 (TF32 hi/lo split, FP32 accumulation)" if m2p_tc else "FP32 pipe"
    for name, flops in (("p2p_fp64", True), ("m2p_fp64", None), ("p2p_ff", True), ("m2p_ff", None)):
        if name in kernels:
            k = kernels[name]
            work = pairs * p2p_flops(B) if flops else info["n_m2p_pairs"] * kernel_targets(info) * m2p_flops(wl["P"], B)
            k["algorithmic_tflops"] = work / (k["ms_per_launch"] * 1e-3) / 1e12
    if dom in ("p2p_fp64", "m2p_fp64"):
        a = kernels[dom]["algorithmic_tflops"]
        roof = {"bound": "alu", "kernel": dom, "achieved": round(a, 4), "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": round(a / FP64_PEAK_TFLOPS, 4), "traffic": NCU_TRAFFIC.get((args.workload, dom, wl["theta"], wl["P"], wl["Ncrit"])),
                "peak_note": "FP64 nominal 1.25 TFLOP/s (no measured FP64 peak)"}
    elif dom == "m2p" and m2p_tc:
        a = kernels[dom]["algorithmic_tflops"]
        pk = peaks.get("bf16_tflops_sustained", 1755.8) * TF32_PER_BF16
        roof = {"bound": "tensor", "kernel": dom, "achieved": round(a, 3), "peak": round(pk, 1), "unit": "TFLOP/s",
                "frac": round(a / pk, 4), "traffic": NCU_TRAFFIC.get((args.workload, dom, wl["theta"], wl["P"], wl["Ncrit"])),
                "peak_note": "measured sustained bf16 x nominal TF32/BF16 rate (1.1/2.25); achieved counts the "
                             "algorithmic contraction flops, not the split products"}
    elif dom in ("p2p", "m2p") and fp32:
        a = kernels[dom]["algorithmic_tflops"]
        roof = {"bound": "alu", "kernel": dom, "achieved": round(a, 3), "peak": round(peak_fp32, 2),
                "unit": "TFLOP/s", "frac": round(a / peak_fp32, 4), "traffic": NCU_TRAFFIC.get((args.workload, dom, wl["theta"], wl["P"], wl["Ncrit"])),
                "peak_note": "FP32 FMA peak 152 SM x 128 lanes x 2 flops x 2070 MHz (derived, no measured FP32 peak)"}
    elif dom in ("p2p_ff", "m2p_ff"):
        a = kernels[dom]["algorithmic_tflops"]
        roof = {"bound": "alu", "kernel": dom, "achieved": round(a, 4), "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s (FP64-equivalent)", "frac": round(a / FP64_PEAK_TFLOPS, 4), "traffic": NCU_TRAFFIC.get((args.workload, dom, wl["theta"], wl["P"], wl["Ncrit"])),
                "peak_note": "float-float kernel replacing FP64; peak is the nominal FP64 1.25 TFLOP/s"}
    elif dom is not None:
        roof = {"bound": "hbm", "kernel": dom, "achieved": None, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                "frac": None, "traffic": None, "peak_note": "of measured"}
    g_int = pairs * (sum(mvs) / len(mvs)) / (total_ms / args.steps / 1e3)

    out = {
        "metric": "lambda-solves/s at sigma_ext rel err <= 1e-4 vs plain FP64 (treecode GMRES)",
        "value": round(value, 4), "unit": "lambda-solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if fp32 else "f64",
        "data": "synthetic (icosphere, Drude silver in water)",
        "config": {"workload": args.workload, "panels": len(tris), "sources": len(tris) * wl["K"],
                   "surfaces": 1 if surf is None else int(surf.max()) + 1,
                   "analytes": None if surf is None else [list(a) for a in wl["analytes"]],
                   "wavelengths": B, "mode": wl["mode"], "theta": wl["theta"], "P": wl["P"], "Ncrit": wl["Ncrit"],
                   "K": wl["K"], "K_fine": wl["K_fine"], "N_k": wl["N_k"], "gmres_tol": wl["tol"],
                   "restart": wl["restart"], "l2": "flushed between steps (258 MiB write)",
                   "parallelism": f"replicas x{world}", "autotune": tune},
        "e2e": {"value": round(B * args.steps * world / e2e_s, 4), "unit": "lambda-solves/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "roofline": roof,
        "matvec_g_interactions_per_s": round(g_int / 1e9, 3),
        "gmres_iterations": iters[-1],
        "sigma_ext_nm2": float(sig[0]),
        "accuracy": acc,
        "kernels": kernels,
        "kernel_timing": {"how": "CUDA events around every launch, instrumented replay of the timed steps "
                                 "(host-driven Arnoldi cycles, same kernels and inputs)",
                          "replay_ms_per_step": round(replay_ms / args.steps, 3)},
        "arnoldi_graphs": graph_stats,
        "tree": {"boxes": info["n_boxes"], "p2p_pairs_per_matvec": info["n_p2p_pairs"],
                 "m2p_box_target_blocks": info["n_m2p_pairs"], "near_entries": info["n_near"]},
        "clocks": clocks,
    }
    ctx.close()
    return out, iters


def kernel_targets(info) -> int:
    return 64   # targets per interaction block


def ctx_launches(ctx) -> int:
    return ctx.launch_count()


# --------------------------------------------------------- oracle (CPU) timings
def oracle_sample(wl, iters_hint: int, reps: int = 1):
    """Time the oracle's matrix-free matvec at full size and extrapolate one
    lambda-solve as (GMRES iterations + 2) matvecs (explicit residual and RHS)."""
    import oracle
    verts, tris, surf = workload_geometry(wl)
    n = len(tris)
    if n > 40000:
        # too large for a full product in the time budget: the matrix entries of a block of
        # rows (the product's cost), scaled to all n rows
        rows = 256
        t0 = time.perf_counter()
        oracle.entries(verts, tris, K=wl["K"], K_fine=wl["K_fine"], rows=(0, rows))
        t_mv = (time.perf_counter() - t0) * n / rows
        return t_mv, (iters_hint + 2) * t_mv, f"the oracle's matrix entries of {rows} of {n} rows, scaled to a product"
    s = I.drude_eps(wl["lam"][0]) / I.EPS_WATER
    x = I.random_complex(2 * n, seed=0)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.matvec(verts, tris, x, s, K=wl["K"], K_fine=wl["K_fine"])
        times.append(time.perf_counter() - t0)
    t_mv = float(np.median(times))
    t_solve = (iters_hint + 2) * t_mv
    return t_mv, t_solve, "one full-size oracle matvec"


def oracle_iterations_hint(wl):
    gold = os.path.join(ROOT, "tests", "golden", f"sphere{len(I.icosphere(wl['sub'], wl['R'])[1])}_l380.json")
    try:
        with open(gold) as f:
            return int(json.load(f)["gmres_iterations"])
    except OSError:
        return 30


def run_reference(args, wl):
    import oracle
    oracle.build()
    it = oracle_iterations_hint(wl)
    for _ in range(args.warmup):
        oracle_sample(wl, it)
    t = 0.0
    for _ in range(args.steps):
        t_mv, t_solve, sample = oracle_sample(wl, it)
        t += t_solve
    value = len(wl["lam"]) * args.steps / t if len(wl["lam"]) == 1 else args.steps / t
    cores = os.cpu_count()
    return {
        "impl": "reference", "metric": "lambda-solves/s at sigma_ext rel err <= 1e-4 vs plain FP64 (treecode GMRES)",
        "value": value, "unit": "lambda-solves/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (icosphere, Drude silver in water)",
        "config": {"workload": args.workload, "panels": len(workload_geometry(wl)[1]),
                   "wavelengths": 1, "mode": "oracle direct FP64 (plain CPU)"},
        "cpu_baseline": {"value": value, "unit": "lambda-solves/s", "cores": cores, "kind": "oracle",
                         "sample": f"{sample} per step, lambda-solve extrapolated as "
                                   f"({it} GMRES iterations + 2) matvecs"},
        "e2e": {"value": value, "unit": "lambda-solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_matvecs(args, wl):
    """K bare matvecs of the workload's mode on a seeded random vector (profiling aid)."""
    import torch
    from paper_1812_10722_gb300 import lspr
    verts, tris = I.icosphere(wl["sub"], wl["R"])
    n = len(tris)
    lam = np.asarray(wl["lam"], float)
    s = I.drude_eps(lam) / I.EPS_WATER   # one product over the workload's B right-hand sides
    ctx = lspr.Context(0, torch.cuda.current_stream().cuda_stream)
    if args.no_tc:
        ctx.set_tensor_cores(False)
    ctx.mesh_upload(verts, tris, wl["K"], wl["K_fine"], wl["N_k"])
    mode = args.matvec_mode or wl["mode"]
    if mode.startswith("tree"):
        ctx.tree_build(wl["theta"], wl["P"], wl["Ncrit"])
    x = torch.as_tensor(I.random_complex(2 * n, seed=0, batch=len(lam)) if len(lam) > 1
                        else I.random_complex(2 * n, seed=0), device="cuda")
    if len(lam) == 1:
        s = complex(s[0])
    ctx.matvec(x, s, mode)
    torch.cuda.synchronize()
    ctx.set_timing(True)
    t0 = time.perf_counter()
    for _ in range(args.matvecs):
        y = ctx.matvec(x, s, mode)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.matvecs
    out = {"workload": args.workload, "mode": mode, "matvecs": args.matvecs, "ms_per_matvec": 1e3 * dt,
           "kernels_ms": {k: v for k, v in ctx.timing().items() if v[1]}, "info": ctx.info(),
           "checksum": float(torch.linalg.vector_norm(y).item())}
    ctx.close()
    return out


def run_profile(args, wl):
    """Profiling aid: W untimed steps, then K steps inside an NVTX range "timed" (for
    ncu --nvtx --nvtx-include timed/), nothing else; the treecode parameters come from
    --tree (no autotuning)."""
    import torch
    from paper_1812_10722_gb300 import lspr
    verts, tris = I.icosphere(wl["sub"], wl["R"])
    lam = np.asarray(wl["lam"], float)
    eps = I.drude_eps(lam)
    v_d = torch.as_tensor(verts, device="cuda")
    t_d = torch.as_tensor(tris, device="cuda")
    stream = torch.cuda.current_stream()
    ctx = lspr.Context(0, stream.cuda_stream)
    if args.no_graphs:
        ctx.set_graphs(False)   # ncu does not profile the kernels inside a graph's loop
    if args.no_tc:
        ctx.set_tensor_cores(False)

    def step():
        ctx.mesh_upload(v_d, t_d, wl["K"], wl["K_fine"], wl["N_k"])
        if wl["mode"].startswith("tree"):
            ctx.tree_build(wl["theta"], wl["P"], wl["Ncrit"])
        return ctx.solve(eps, I.EPS_WATER, lam, tol=wl["tol"], restart=wl["restart"], maxiter=2000,
                         mode=wl["mode"], refine=wl["refine"])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        r = step()
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    e1.synchronize()
    out = {"workload": args.workload, "tree": [wl["theta"], wl["P"], wl["Ncrit"]], "steps": args.steps,
           "ms_per_step": e0.elapsed_time(e1) / args.steps, "iterations": int(r.iterations.max()),
           "matvecs": int(r.matvecs), "launches": ctx.launch_count()}
    ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sphere20480", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--restart", type=int, default=None, help="override the workload's GMRES restart length")
    ap.add_argument("--matvecs", type=int, default=0, help="only run this many bare matvecs (profiling)")
    ap.add_argument("--matvec-mode", default=None, help="matvec mode for --matvecs (default: the workload's)")
    ap.add_argument("--tree", default=None, help="THETA,P,NCRIT: fixed treecode parameters (no autotuning)")
    ap.add_argument("--profile", action="store_true", help="only the steps, in an NVTX range 'timed' (profiling)")
    ap.add_argument("--no-graphs", action="store_true", help="host-driven Arnoldi cycles (profiling)")
    ap.add_argument("--no-tc", action="store_true", help="FP32 M2P on the CUDA cores, not tcgen05")
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.restart:
        wl["restart"] = args.restart
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.tree:
        th, P, nc = args.tree.split(",")
        wl.update(theta=float(th), P=int(P), Ncrit=int(nc), autotune=False)
    if args.matvecs:
        print(json.dumps(run_matvecs(args, wl)))
        return
    if args.profile:
        print(json.dumps(run_profile(args, wl)))
        return

    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args, wl)))
        return

    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    out, iters = run_ours(args, wl, rank, world, local_rank)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_mv, t_solve, sample = oracle_sample(wl, iters[-1])
        out["cpu_baseline"] = {"value": 1.0 / t_solve,
                               "unit": "lambda-solves/s", "cores": os.cpu_count(), "kind": "oracle",
                               "sample": f"{sample} ({t_mv:.2f} s) on the host cores; one "
                                         f"lambda-solve extrapolated as ({iters[-1]} GMRES iterations + 2) matvecs"}
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
