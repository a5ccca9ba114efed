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
    """Wavelength of the extinction peak (reciprocal-parabola vertex, sensitivity.peak_wavelength)."""
    from paper_1812_10722_gb300.sensitivity import peak_wavelength
    return peak_wavelength(lam, sigma)


METRIC = "lambda-solves/s at sigma_ext rel err <= 1e-4 vs plain FP64 (treecode GMRES)"
L2_BYTES = 129 * 2 ** 20
P2P_GEN_FLOPS = 18      # per (target, source) pair, generation of G and dG/dn: 3 sub, 3 FMA (r^2), 2 mul
                        # (r^-3), 3 FMA (n.d), 2 scale, with FMA = 2 flops; the rsqrt goes to the SFU
SFU_PER_CLK_SM = 16     # MUFU (rsqrt, reciprocal) results per clock per SM
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64
TF32_PER_BF16 = 1.1 / 2.25  # nominal dense tensor rates, TF32 over BF16
# DRAM bytes (read + write) per launch of the current kernels, from the ncu captures summarised in
# profiles/ (dram__bytes_read.sum + dram__bytes_write.sum of one launch), keyed by workload, kernel and
# treecode parameters (theta, P, Ncrit); None where no capture of the current kernel matches
NCU_TRAFFIC = {("sphere20480", "m2p", 0.4, 5, 256): 2.410e6,          # m2p_fp32_sphere20480.md
               ("sphere20480", "p2p", 0.4, 5, 256): 5.045e6,          # p2p1_fp32_sphere20480.md
               ("sphere81920_sweep64", "m2p", 0.4, 7, 512): 8.883e9,  # m2p_tc_sphere81920_sweep64.md
               ("sphere81920_sweep64", "p2p", 0.4, 7, 512): 9.805e8}  # p2p_tc_sphere81920_sweep64.md


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


def p2p_tc_bound(B: int, pairs: int, stages: int, peaks: dict, mhz: float) -> dict:
    """Time bound of one tensor-core P2P launch: the largest of its G and dG/dn generation on the
    FP32 pipe (the blocks' own pairs, once per unit of 64 right-hand sides), its rsqrt on the SFU,
    and its issued MMAs on the tensor pipe (per stage of 8 sources: M = 128 channels x N = 256
    targets x K = 8, for the single and the double layer, 3 products each above 32 right-hand
    sides in the unit, 2 at 32 or fewer)."""
    units = [min(64, B - b0) for b0 in range(0, B, 64)]
    gen = pairs * P2P_GEN_FLOPS * len(units)
    mufu = pairs * len(units)
    mma = sum(stages * 2 * (3 if nb > 32 else 2) * 2 * 128 * 256 * 8 for nb in units)
    fp32_peak = fp32_peak_tflops(mhz) * 1e12
    sfu_peak = SFU_PER_CLK_SM * 152 * mhz * 1e6
    tf32_peak = peaks.get("bf16_tflops_sustained", 1741.2) * TF32_PER_BF16 * 1e12
    t = {"fp32_generation": gen / fp32_peak, "sfu": mufu / sfu_peak, "tensor_mma": mma / tf32_peak}
    return {"terms_s": t, "bound_s": max(t.values()), "limiter": max(t, key=t.get), "mma_flops": mma,
            "generation_flops": gen, "mufu_ops": mufu, "tf32_peak_tflops": tf32_peak / 1e12,
            "fp32_peak_tflops": fp32_peak / 1e12, "sfu_peak_tops": sfu_peak / 1e12}


def tc_roofline(bnd: dict, t: float, kernel: str, traffic) -> dict:
    """Roofline entry of a tensor-core kernel from its max-of-three bound and launch time t (s)."""
    lim = bnd["limiter"]
    if lim == "tensor_mma":
        a, pk, unit, bound = bnd["mma_flops"] / t / 1e12, bnd["tf32_peak_tflops"], "TFLOP/s", "tensor"
    elif lim == "fp32_generation":
        a, pk, unit, bound = bnd["generation_flops"] / t / 1e12, bnd["fp32_peak_tflops"], "TFLOP/s", "alu"
    else:
        a, pk, unit, bound = bnd["mufu_ops"] / t / 1e12, bnd["sfu_peak_tops"], "Top/s", "alu"
    return {"bound": bound, "kernel": kernel, "achieved": round(a, 3), "peak": round(pk, 2), "unit": unit,
            "frac": round(bnd["bound_s"] / t, 4), "traffic": traffic,
            "bound_terms_ms": {x: round(1e3 * y, 4) for x, y in bnd["terms_s"].items()},
            "peak_note": "frac = max(generation flops / FP32 peak (152 SM x 128 x 2 x 2070 MHz, derived), rsqrt / "
                         "SFU peak (16 per clock per SM), issued TF32 MMA flops / TF32 peak (measured sustained "
                         "bf16 x nominal 1.1/2.25)) / the launch time; achieved and peak are the limiting term's"}


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest x over the ranks (the replicas' job time is the slowest rank's)."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_rate(B: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job lambda-solves/s: every rank solves its own B wavelengths per step."""
    return B * steps * world / seconds


def arnoldi_gb(n_panels: int, c: dict) -> float:
    """Basis traffic (GB) of the Arnoldi vector kernels from the device work counters
    (lspr_get_arnoldi_stats): 16 bytes per complex entry of vectors of 2N entries; per
    system-step 7 + 2 (j + 1) vectors, and 3 + 2 (j + 1) more for a second Gram-Schmidt pass."""
    vec = 16 * 2 * n_panels
    return vec * (7 * c["system_steps"] + 2 * c["vectors"] + 2 * c["vectors_second_pass"]
                  + 3 * c["system_steps_second_pass"]) / 1e9


def m2p_terms(P: int) -> int:
    """Taylor terms with |k| <= P."""
    return (P + 1) * (P + 2) * (P + 3) // 6


def p2p_flops(B: int = 1) -> int:
    """Flops per (target, source) pair: G and dG/dn generated once (18), then two kernels
    times 2 real channels of each right-hand side (8 B)."""
    return P2P_GEN_FLOPS + 8 * B


def m2p_tc_bound(P: int, B: int, group_box_pairs: int, peaks: dict, mhz: float) -> dict:
    """Time bound of one tensor-core M2P launch: the largest of its coefficient generation on the
    FP32 pipe (the recurrence for 256 targets per (group, box) and unit of 16, 32 or 64 right-hand
    sides), its reciprocal square roots on the SFU, and its issued MMAs on the tensor pipe
    (M = 128 channels x N = 256 targets x K = 8 per step; 3 MMAs per step for each A part of 32
    right-hand sides, 2 for units of 16; above 32 right-hand sides a unit carries two A parts
    against one set of coefficients)."""
    nt = (P + 1) * (P + 2) * (P + 3) // 6
    rc = 16 if B <= 16 else (32 if B <= 32 else 64)
    units = (B + rc - 1) // rc                      # coefficient generations per (group, box)
    parts = (B + min(rc, 32) - 1) // min(rc, 32)    # A parts of 32 (or 16) right-hand sides
    ksteps = sum((min(16, nt - kc) + 7) // 8 for kc in range(0, nt, 16))
    gen = group_box_pairs * units * 256 * (m2p_flops(P, 0))
    mufu = group_box_pairs * units * 256
    mma = group_box_pairs * parts * (2 if rc == 16 else 3) * 2 * 128 * 256 * 8 * ksteps
    fp32_peak = fp32_peak_tflops(mhz) * 1e12
    sfu_peak = SFU_PER_CLK_SM * 152 * mhz * 1e6
    tf32_peak = peaks.get("bf16_tflops_sustained", 1741.2) * TF32_PER_BF16 * 1e12
    t = {"fp32_generation": gen / fp32_peak, "sfu": mufu / sfu_peak, "tensor_mma": mma / tf32_peak}
    return {"terms_s": t, "bound_s": max(t.values()), "limiter": max(t, key=t.get), "mma_flops": mma,
            "generation_flops": gen, "mufu_ops": mufu, "tf32_peak_tflops": tf32_peak / 1e12,
            "fp32_peak_tflops": fp32_peak / 1e12, "sfu_peak_tops": sfu_peak / 1e12}


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
    elif args.tc is not None:
        ctx.set_tensor_cores(args.tc)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    tune = None
    if wl.get("autotune") and wl["mode"].startswith("tree"):
        # once per geometry, before the timed region: treecode parameters under the sigma_ext bound
        ctx.mesh_upload(v_d, t_d, wl["K"], wl["K_fine"], wl["N_k"], surf_id=s_d)
        lt = tuning_wavelengths(lam, wl.get("tune_lams", 4))
        t0 = time.perf_counter()
        # a batch: candidates costed from product times at the batch's size, then the restart
        # length and the P2P path timed with full solves of the batch
        tune = ctx.autotune(workload_eps(wl, lt), em, lt, target_rel_err=1e-4, tol=min(wl["tol"], 1e-8),
                            restart=wl["restart"], mode=wl["mode"], refine=1 if wl["refine"] else 0,
                            coarse=len(tris) > 50000, time_rhs=B if B > 1 else 0)
        wl["theta"], wl["P"], wl["Ncrit"] = tune["theta"], tune["P"], tune["Ncrit"]
        if B > 1 and wl["mode"] == "tree_fp32" and args.tc is None and not args.no_tc:
            tune["solver"] = ctx.tune_solver(eps, em, lam, restarts=(30, 50, 80), tol=wl["tol"], maxiter=2000,
                                             mode=wl["mode"], refine=1 if wl["refine"] else 0)
            wl["restart"] = tune["solver"]["restart"]
        tune["seconds"] = round(time.perf_counter() - t0, 2)
        tune["wavelengths"] = [float(x) for x in lt]
        if args.no_tc:
            ctx.set_tensor_cores(False)
        elif args.tc is not None:
            ctx.set_tensor_cores(args.tc)

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
    arn0 = ctx.arnoldi_stats()
    ctx.set_timing(True)
    replay_ms = 0.0
    replay_steps = min(args.steps, 3)   # the per-kernel table needs a few steps, not all
    for _ in range(replay_steps):
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
    krhs = ctx.timing_rhs()
    ctx_tc = ctx.tc_info()
    arn1 = ctx.arnoldi_stats()
    arn = {k: arn1[k] - arn0[k] for k in arn0}
    # ---- the far-field kernels at the full batch: inside the solves converged wavelengths are
    # packed out, so a replayed launch carries anywhere from B down to 1 right-hand sides; the
    # roofline of a kernel is taken on 3 bare products of all B (seeded random right-hand sides,
    # the last tree of the replay), each launch timed with CUDA events on its stream
    ctx.set_timing(False)
    ctx.set_timing(True)
    xfull = torch.as_tensor(I.random_complex(2 * len(tris), seed=1, batch=B) if B > 1
                            else I.random_complex(2 * len(tris), seed=1), device=dev)
    sfull = eps / em if B > 1 else complex(eps[0] / em)
    for _ in range(3):
        ctx.matvec(xfull, sfull, wl["mode"])
    torch.cuda.synchronize(dev)
    kfull = ctx.timing()
    del xfull
    ctx.set_timing(False)
    barrier()
    info = ctx.info()
    t_max = max_over_ranks(total_ms, world, dev)
    value = replica_rate(B, args.steps, world, t_max / 1e3)

    # ---- accuracy and the plain baseline: the FP64 treecode (same tree) one wavelength at a time at
    # the checked wavelengths (all of them for B <= 4; else the one nearest the resonance, both ends
    # and the middle), each solve timed with CUDA events; the mixed-precision sigma_ext and the FP64
    # one against each other and against the oracle's stored solves
    acc = {}
    base = None
    if wl["mode"] == "tree_fp32":
        ka = [int(np.where(lam == x)[0][0]) for x in tuning_wavelengths(lam)] if B > 4 else list(range(B))
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        ctx.mesh_upload(v_d, t_d, wl["K"], wl["K_fine"], wl["N_k"], surf_id=s_d)
        ctx.tree_build(wl["theta"], wl["P"], wl["Ncrit"])
        g1.record(stream)
        g1.synchronize()
        t_geom = g0.elapsed_time(g1)
        ctx.solve(eps[ka[:1]], em, lam[ka[:1]], tol=wl["tol"], restart=wl["restart"], maxiter=2000, mode="tree_fp64")
        sig64, t64, it64 = [], [], []
        for k in ka:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r64 = ctx.solve(eps[k:k + 1], em, lam[k:k + 1], tol=wl["tol"], restart=wl["restart"], maxiter=2000,
                            mode="tree_fp64")
            e1.record(stream)
            e1.synchronize()
            t64.append(e0.elapsed_time(e1))
            sig64.append(float(r64.sigma_ext[0]))
            it64.append(int(r64.iterations[0]))
        sig64 = np.asarray(sig64)
        acc["sigma_rel_err_vs_fp64_treecode"] = float(np.max(np.abs(sig[ka] - sig64) / sig64))
        acc["checked_wavelengths_nm"] = [float(lam[k]) for k in ka]
        t_sweep = t_geom + B / len(ka) * sum(t64)
        base = {"value": round(1e3 * B / t_sweep, 4), "unit": "lambda-solves/s",
                "ms_per_sweep": round(t_sweep, 2), "extrapolated": B > len(ka),
                "ratio": round(value / (1e3 * B / t_sweep), 3),
                "sample": f"plain FP64 treecode GMRES (theta {wl['theta']}, P {wl['P']}, Ncrit {wl['Ncrit']}, tol "
                          f"{wl['tol']}, restart {wl['restart']}, no refinement), one wavelength at a time: "
                          f"{len(ka)} of the {B} wavelengths ({acc['checked_wavelengths_nm']}) solved and timed "
                          f"with CUDA events ({[round(x, 1) for x in t64]} ms, {it64} Arnoldi steps); the sweep = "
                          f"one mesh upload and tree build ({t_geom:.1f} ms) + {B}/{len(ka)} x their sum",
                "sigma_ext_nm2": [float(x) for x in sig64]}
    gname = os.path.join(ROOT, "tests", "golden", f"{args.workload}.json")
    gold1 = os.path.join(ROOT, "tests", "golden", f"sphere{info['n_panels']}_l380.json")
    if os.path.exists(gname):
        with open(gname) as f:
            g = json.load(f)
        idx = [int(np.argmin(np.abs(lam - x))) for x in g["lambda_nm"]]
        ref = np.asarray(g["sigma_ext_nm2"])
        err = np.abs(sig[idx] - ref) / ref
        acc["oracle"] = {"lambda_nm": [float(lam[k]) for k in idx], "sigma_rel_err": [float(e) for e in err],
                         "max_rel_err": float(err.max()), "within_1e-4": bool(err.max() <= 1e-4),
                         "resonance_lambda_nm": float(lam[g["resonance_index"]]),
                         "golden": f"tests/golden/{args.workload}.json (oracle, direct FP64, tol 1e-8)"}
        if base is not None:
            s64 = dict(zip(acc["checked_wavelengths_nm"], base["sigma_ext_nm2"]))
            e64 = [abs(s64[float(lam[k])] - r) / r for k, r in zip(idx, ref) if float(lam[k]) in s64]
            if e64:
                base["sigma_max_rel_err_vs_oracle"] = float(max(e64))
        acc["sigma_rel_err_vs_oracle"] = float(err.max())
    elif B == 1 and lam[0] == 380.0 and os.path.exists(gold1):
        with open(gold1) as f:
            g = json.load(f)
        acc["sigma_rel_err_vs_oracle"] = float(abs(sig[0] - g["sigma_ext_nm2"]) / g["sigma_ext_nm2"])
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
    dev_errors = ctx.device_errors()

    # ---- end to end through the public API with host buffers
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = step(True)
    torch.cuda.synchronize(dev)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    h2d = verts.nbytes + tris.nbytes + eps.astype(np.complex128).nbytes + lam.nbytes + 24 + (
        0 if surf is None else surf.nbytes)
    d2h = B * (3 * 16 + 8)

    # ---- roofline of the dominant kernel: CUDA events around every launch of the instrumented
    # replay, in which the far-field kernels run one after another on one stream (no overlap);
    # algorithmic work counted from the right-hand sides each timed launch carried
    peaks = load_peaks()
    mhz = peaks.get("sm_max_mhz", 2070.0)
    kernels = {}
    for name in ("p2p", "m2p", "p2m", "near_assembly", "gmres", "tree", "mesh", "p2p_fp64", "m2p_fp64", "p2m_fp64",
                 "weights", "p2p_ff", "m2p_ff", "p2m_ff"):
        ms, n = ktime[name]
        if n:
            kernels[name] = {"ms_total": round(ms, 4), "launches": n, "ms_per_launch": ms / n,
                             "share_of_step": round(ms / replay_ms, 4)}
            if krhs[name]:
                kernels[name]["rhs_per_launch"] = round(krhs[name] / n, 3)
    pairs = info["n_p2p_pairs"] if wl["mode"].startswith("tree") else info["n_panels"] * info["n_sources"]
    tgt_box = info["n_m2p_pairs"] * kernel_targets(info)
    fp32 = wl["mode"].endswith("fp32")
    peak_fp32 = fp32_peak_tflops(mhz)
    m2p_tc = B > 1 and fp32 and not args.no_tc and (args.tc is None or args.tc & 1)   # M2P of several RHS on tcgen05
    p2p_tc = B > 1 and fp32 and not args.no_tc and ctx_tc["p2p_stages"] > 0           # P2P of several RHS on tcgen05

    def work(name):
        """Algorithmic flops of all timed launches of a far-field slot."""
        n, r = kernels[name]["launches"], krhs[name]
        if name.startswith("p2p"):
            return pairs * (P2P_GEN_FLOPS * n + 8 * r)
        if name.startswith("m2p"):
            return tgt_box * (m2p_flops(wl["P"], 0) * n + 8 * m2p_terms(wl["P"]) * r)
        return None

    for name in ("p2p", "m2p", "p2p_fp64", "m2p_fp64", "p2p_ff", "m2p_ff"):
        if name in kernels and krhs[name]:
            k = kernels[name]
            k["algorithmic_tflops"] = work(name) / (k["ms_total"] * 1e-3) / 1e12
    if "p2p" in kernels:
        kernels["p2p"]["pairs_per_launch"] = pairs
        kernels["p2p"]["path"] = "tcgen05 (TF32 hi/lo split, FP32 accumulation)" if p2p_tc else "FP32 pipe"
    if "m2p" in kernels:
        kernels["m2p"]["path"] = "tcgen05 (TF32 hi/lo split, FP32 accumulation)" if m2p_tc else "FP32 pipe"
    if "gmres" in kernels and arn["system_steps"]:
        # basis traffic of the Arnoldi vector kernels (16 bytes per complex entry of 2N): per
        # system-step 3 vectors (v_j, z, w read) + 2 (j + 3) for the first Gram-Schmidt pass
        # (w converted in place, the j + 1 basis vectors read twice, w written), and 2 (j + 1) + 3
        # for a second pass; the cycles' update (once per restart) is not counted
        gb = arnoldi_gb(len(tris), arn)
        k = kernels["gmres"]
        k["algorithmic_gb"] = round(gb, 3)
        k["achieved_gbs"] = round(gb / (k["ms_total"] * 1e-3), 1)
        k["hbm_frac"] = round(k["achieved_gbs"] / peaks.get("hbm_gbs", 6800.0), 4)
        k["arnoldi_counters"] = arn
    full = {}   # per-launch times of the far-field kernels at all B right-hand sides
    for name in ("p2p", "m2p", "p2m", "near_assembly", "weights", "p2p_fp64", "m2p_fp64", "p2m_fp64"):
        ms, n = kfull.get(name, (0.0, 0))
        if n:
            full[name] = {"ms_per_launch": round(ms / n, 4), "launches": n, "rhs": B}
    for name in ("p2p", "m2p"):
        if name in full:
            n = full[name]["launches"]
            w = (pairs * p2p_flops(B) if name == "p2p" else tgt_box * m2p_flops(wl["P"], B))
            full[name]["algorithmic_tflops"] = round(w / (full[name]["ms_per_launch"] * 1e-3) / 1e12, 3)
    roof = None
    dom = max((k for k in kernels if k in ("p2p", "m2p", "p2p_fp64", "m2p_fp64", "p2p_ff", "m2p_ff")),
              key=lambda k: kernels[k]["ms_total"], default=None)
    traffic = NCU_TRAFFIC.get((args.workload, dom, wl["theta"], wl["P"], wl["Ncrit"])) if dom else None
    if dom in ("p2p_fp64", "m2p_fp64"):
        a = kernels[dom]["algorithmic_tflops"]
        roof = {"bound": "alu", "kernel": dom, "achieved": round(a, 4), "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": round(a / FP64_PEAK_TFLOPS, 4), "traffic": traffic,
                "peak_note": "FP64 nominal 1.25 TFLOP/s (no measured FP64 peak)"}
    elif dom == "m2p" and m2p_tc and "m2p" in full:
        # max(generation / FP32 peak, rsqrt / SFU peak, issued MMA flops / TF32 peak) per launch of
        # all B right-hand sides
        bnd = m2p_tc_bound(wl["P"], B, ctx_tc["m2p_group_boxes"], peaks, mhz)
        roof = tc_roofline(bnd, full["m2p"]["ms_per_launch"] * 1e-3, dom, traffic)
    elif dom == "p2p" and p2p_tc and "p2p" in full:
        bnd = p2p_tc_bound(B, pairs, ctx_tc["p2p_stages"], peaks, mhz)
        roof = tc_roofline(bnd, full["p2p"]["ms_per_launch"] * 1e-3, dom, traffic)
    elif dom in ("p2p", "m2p") and fp32 and dom in full:
        a = full[dom]["algorithmic_tflops"]
        roof = {"bound": "alu", "kernel": dom, "achieved": round(a, 3), "peak": round(peak_fp32, 2),
                "unit": "TFLOP/s", "frac": round(a / peak_fp32, 4), "traffic": traffic,
                "peak_note": "FP32 FMA peak 152 SM x 128 lanes x 2 flops x 2070 MHz (derived, no measured FP32 peak)"}
    elif dom in ("p2p_ff", "m2p_ff"):
        a = kernels[dom]["algorithmic_tflops"]
        roof = {"bound": "alu", "kernel": dom, "achieved": round(a, 4), "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s (FP64-equivalent)", "frac": round(a / FP64_PEAK_TFLOPS, 4), "traffic": traffic,
                "peak_note": "float-float kernel replacing FP64; peak is the nominal FP64 1.25 TFLOP/s"}
    # the other tensor-core kernel at the full batch, on the same max-of-three bound
    roof2 = None
    if roof is not None and roof.get("kernel") == "m2p" and p2p_tc and "p2p" in full:
        roof2 = tc_roofline(p2p_tc_bound(B, pairs, ctx_tc["p2p_stages"], peaks, mhz),
                            full["p2p"]["ms_per_launch"] * 1e-3, "p2p",
                            NCU_TRAFFIC.get((args.workload, "p2p", wl["theta"], wl["P"], wl["Ncrit"])))
        del roof2["peak_note"]
    g_int = pairs * (sum(mvs) / len(mvs)) / (total_ms / args.steps / 1e3)

    out = {
        "metric": METRIC,
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
        "e2e": {"value": round(replica_rate(B, args.steps, world, e2e_s), 4), "unit": "lambda-solves/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "roofline": roof,
        "roofline_p2p": roof2,
        "kernels_full_batch": full,
        "matvec_g_interactions_per_s": round(g_int / 1e9, 3),
        "gmres_iterations": iters[-1],
        "sigma_ext_nm2": float(sig[0]),
        "accuracy": acc,
        "baseline_fp64_treecode": base,
        "device_errors": dev_errors,
        "kernels": kernels,
        "kernel_timing": {"how": "CUDA events around every launch, instrumented replay of the first "
                                 f"{replay_steps} timed steps (far-field kernels one after another on one "
                                 "stream; Arnoldi cycles launched from the host instead of a graph loop: "
                                 "same kernels and inputs)",
                          "replay_ms_per_step": round(replay_ms / replay_steps, 3)},
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
def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def oracle_iterations(wl, n_panels: int):
    """The oracle's own GMRES step count for the workload, from its stored golden solves: the
    largest over the stored wavelengths (the lockstep solve of a sweep runs until its slowest
    wavelength converges).  Returns (steps, source)."""
    name = "sphere81920_sweep64.json" if n_panels == 81920 and len(wl["lam"]) > 1 else f"sphere{n_panels}_l380.json"
    try:
        with open(os.path.join(ROOT, "tests", "golden", name)) as f:
            its = json.load(f)["gmres_iterations"]
        return int(max(np.atleast_1d(its))), f"tests/golden/{name}"
    except (OSError, KeyError):
        return 40, "no stored oracle solve for this mesh: 40 assumed"


def oracle_block(wl, rows: int, nthreads: int = 0):
    """Time rows [0, rows) of the oracle's product with all the workload's right-hand sides (the
    entries of a row are evaluated once for all of them).  Returns (seconds, rows, n)."""
    import oracle
    verts, tris, surf = workload_geometry(wl)
    n = len(tris)
    rows = max(1, min(rows, n))
    lam = np.asarray(wl["lam"], float)
    if surf is not None:
        # several surfaces: the matrix entries of the block of rows (the product's cost)
        t0 = time.perf_counter()
        oracle.entries(verts, tris, K=wl["K"], K_fine=wl["K_fine"], rows=(0, rows))
        return time.perf_counter() - t0, rows, n
    s = I.drude_eps(lam) / I.EPS_WATER
    x = I.random_complex(2 * n, seed=0, batch=len(lam))
    t0 = time.perf_counter()
    oracle.matvec_rows(verts, tris, x, s, (0, rows), K=wl["K"], K_fine=wl["K_fine"], nthreads=nthreads)
    return time.perf_counter() - t0, rows, n


def oracle_rows_for(wl, seconds: float, nthreads: int = 0) -> int:
    """Rows of the oracle's product that take about `seconds` (calibrated on a small block)."""
    t, r, n = oracle_block(wl, 64, nthreads)
    return int(max(16, min(n, 64 * seconds / max(t, 1e-6))))


def oracle_rate(wl, t_block: float, rows: int, n: int, iters: int) -> float:
    """lambda-solves/s of the oracle's lockstep solve of the workload's B wavelengths, from the
    time of a block of rows of its B-right-hand-side product: (iterations + 3) products (first
    residual, one per Arnoldi step, final residual, the right-hand side's pass over V)."""
    t_prod = t_block * n / rows
    return len(wl["lam"]) / ((iters + 3) * t_prod)


def oracle_baseline(wl, n_panels: int, seconds: float = 12.0) -> dict:
    """The cpu_baseline of the GPU line: the oracle timed on all host cores and on one, on a
    bounded block of rows of its product, extrapolated to the workload's lambda-solves/s."""
    iters, src = oracle_iterations(wl, n_panels)
    rows = oracle_rows_for(wl, seconds)
    t_all, rows, n = oracle_block(wl, rows)
    if wl.get("analytes"):
        # several surfaces: the timed block is the matrix entries of the rows, which the oracle
        # evaluates on one thread
        v = oracle_rate(wl, t_all, rows, n, iters)
        return {"value": v, "unit": "lambda-solves/s", "cores": 1, "kind": "oracle", "single_thread_value": v,
                "cpu_model": cpu_model(), "extrapolated": True,
                "sample": f"matrix entries of rows 0..{rows} of {n} on one thread ({t_all:.2f} s), scaled to the "
                          f"whole matrix and to ({iters} + 3) products per lockstep solve; {iters} = {src}"}
    cores = os.cpu_count()
    rows1 = max(8, rows // max(1, cores))
    t_one, rows1, _ = oracle_block(wl, rows1, nthreads=1)
    v_all = oracle_rate(wl, t_all, rows, n, iters)
    v_one = oracle_rate(wl, t_one, rows1, n, iters)
    return {"value": v_all, "unit": "lambda-solves/s", "cores": cores, "kind": "oracle",
            "single_thread_value": v_one, "cpu_model": cpu_model(), "extrapolated": True,
            "sample": f"rows 0..{rows} of {n} of the oracle's {len(wl['lam'])}-right-hand-side product on "
                      f"{cores} threads ({t_all:.2f} s; {rows1} rows on one thread: {t_one:.2f} s), scaled to "
                      f"the whole product and to ({iters} + 3) products per lockstep solve; {iters} = the "
                      f"oracle's own step count ({src})"}


def run_reference(args, wl):
    """The oracle as it stands on the host cores: every step times one bounded block of rows of its
    B-right-hand-side product (about 4 s); the lambda-solve rate is extrapolated from it."""
    import oracle
    oracle.build()
    n = len(workload_geometry(wl)[1])
    iters, src = oracle_iterations(wl, n)
    rows = oracle_rows_for(wl, 4.0)
    for _ in range(args.warmup):
        oracle_block(wl, rows)
    ts = []
    for _ in range(args.steps):
        t, rows, n = oracle_block(wl, rows)
        ts.append(t)
    t_step = float(np.mean(ts))
    value = oracle_rate(wl, t_step, rows, n, iters)
    cores = os.cpu_count()
    sample = (f"each step: rows 0..{rows} of {n} of the oracle's {len(wl['lam'])}-right-hand-side product on "
              f"{cores} threads; value extrapolated to the whole product and to ({iters} + 3) products per "
              f"lockstep solve of the {len(wl['lam'])} wavelengths ({iters} = the oracle's own step count, {src})")
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "lambda-solves/s", "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (icosphere, Drude silver in water)",
        "extrapolated": True,
        "config": {"workload": args.workload, "panels": n, "wavelengths": len(wl["lam"]),
                   "mode": "oracle direct FP64 (plain CPU), lockstep GMRES"},
        "cpu_baseline": {"value": value, "unit": "lambda-solves/s", "cores": cores, "kind": "oracle",
                         "cpu_model": cpu_model(), "extrapolated": True, "sample": sample},
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
    elif args.tc is not None:
        ctx.set_tensor_cores(args.tc)
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
    if args.tc is not None:
        ctx.set_tensor_cores(args.tc)
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


def run_study(args):
    """Resonance-shift studies (builder runs, not the timed step): "sensitivity" = the 327680-panel
    sphere with six analytes at gaps of 0.5/1/2/4 nm on +-x, +-y, +-z, 32 wavelengths over
    370-400 nm each; "placement" = the 81920-panel sphere with two analytes at 1 nm on +-z, +-x
    or +-y.  Treecode parameters from the autotuner on the first geometry (one wavelength, the
    one nearest the resonance, coarse grid), or fixed by --tree."""
    import torch
    from paper_1812_10722_gb300 import lspr
    from paper_1812_10722_gb300 import sensitivity as SN
    lam = I.wavelengths(370, 400, 32)
    if args.study == "sensitivity":
        geoms = SN.gap_geometries([0.5, 1.0, 2.0, 4.0], sphere_sub=7)
        sub = 7
    else:
        geoms = SN.axis_geometries(1.0, sphere_sub=6)
        sub = 6
    ctx = lspr.Context(0, torch.cuda.current_stream().cuda_stream)
    if args.tc is not None:
        ctx.set_tensor_cores(args.tc)
    if args.tree:
        # fixed treecode parameters (--tree), no autotuning
        th, P, nc = args.tree.split(",")
        tree, tune = (float(th), int(P), int(nc)), None
    else:
        name0 = next(iter(geoms))
        v, t, surf = geoms[name0]
        S = int(surf.max()) + 1
        lt = tuning_wavelengths(lam, 1)
        e = np.full((1, S), 2.25 + 0j)
        e[:, 0] = I.drude_eps(lt)
        ctx.mesh_upload(v, t, surf_id=surf)
        t0 = time.perf_counter()
        tune = ctx.autotune(e, I.EPS_WATER, lt, target_rel_err=1e-4, tol=1e-8, restart=50, mode="tree_fp32",
                            refine=1, coarse=True)
        tune["seconds"] = round(time.perf_counter() - t0, 2)
        tree = (tune["theta"], tune["P"], tune["Ncrit"])
    t0 = time.perf_counter()
    res = SN.shift_study(ctx, geoms, lam, sub, tree=tree)
    out = {"study": args.study, "wavelengths": [float(lam[0]), float(lam[-1]), len(lam)], "tree": tree,
           "autotune": tune, "seconds": round(time.perf_counter() - t0, 1), "results": res,
           "device_errors": ctx.device_errors(), "tensor_cores": args.tc}
    ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sphere81920_sweep64", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--restart", type=int, default=None, help="override the workload's GMRES restart length")
    ap.add_argument("--matvecs", type=int, default=0, help="only run this many bare matvecs (profiling)")
    ap.add_argument("--matvec-mode", default=None, help="matvec mode for --matvecs (default: the workload's)")
    ap.add_argument("--tree", default=None, help="THETA,P,NCRIT: fixed treecode parameters (no autotuning)")
    ap.add_argument("--profile", action="store_true", help="only the steps, in an NVTX range 'timed' (profiling)")
    ap.add_argument("--no-graphs", action="store_true", help="host-driven Arnoldi cycles (profiling)")
    ap.add_argument("--no-tc", action="store_true", help="FP32 M2P on the CUDA cores, not tcgen05")
    ap.add_argument("--study", default=None, choices=["sensitivity", "placement"],
                    help="resonance-shift study instead of the timed step (builder runs)")
    ap.add_argument("--tc", type=int, default=None, help="tensor-core mask for several right-hand sides (1 M2P, 3 M2P+P2P)")
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
    if args.study:
        print(json.dumps(run_study(args)))
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
        out["cpu_baseline"] = oracle_baseline(wl, out["config"]["panels"])
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
