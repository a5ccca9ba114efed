"""The bench's workloads against the benchmark configurations (mesh sizes, wavelength grids,
media, tolerances) and its algorithmic work counts; CPU only, nothing is timed."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1812_10722_gb300 import inputs as I  # noqa: E402


def test_default_workload_is_the_batched_sweep():
    # the metric's configuration: 81920 panels, 64 wavelengths in one batched solve
    src = open(bench.__file__).read()
    assert 'add_argument("--workload", default="sphere81920_sweep64"' in src


def test_single_wavelength_workload_is_the_20480_panel_sphere():
    wl = bench.WORKLOADS["sphere20480"]
    v, t, surf = bench.workload_geometry(wl)
    assert len(t) == 20480 and surf is None
    r = np.linalg.norm(v, axis=1)
    assert np.allclose(r, 10.0)
    assert wl["lam"] == [380.0] and wl["tol"] == 1e-6 and wl["mode"] == "tree_fp32"
    assert (wl["K"], wl["K_fine"]) == (4, 19)


def test_sweep_workloads():
    w16 = bench.WORKLOADS["sphere20480_sweep16"]
    assert len(w16["lam"]) == 16 and w16["lam"][0] == 350.0 and w16["lam"][-1] == 420.0
    w64 = bench.WORKLOADS["sphere81920_sweep64"]
    lam = np.asarray(w64["lam"])
    assert len(lam) == 64 and lam[0] == 350.0 and lam[-1] == 420.0
    assert np.allclose(np.diff(lam), 70.0 / 63.0)          # uniform, endpoints included
    assert w64["sub"] == 6 and 20 * 4 ** w64["sub"] == 81920
    assert w64["tol"] == 1e-6 and w64["refine"]


def test_sensor_workload():
    wl = bench.WORKLOADS["sensor_c4"]
    lam = np.asarray(wl["lam"])
    assert len(lam) == 32 and lam[0] == 370.0 and lam[-1] == 400.0
    assert wl["eps_analyte"] == 2.25 and 20 * 4 ** wl["sub"] == 81920
    assert {a[1] for a in wl["analytes"]} == {1.0}          # 1 nm gaps on +-z
    eps = bench.workload_eps(wl, lam[:3])
    assert eps.shape == (3, 3)
    assert np.allclose(eps[:, 0], I.drude_eps(lam[:3])) and np.allclose(eps[:, 1:], 2.25)


def test_tuning_wavelengths_hold_the_resonance():
    lam = I.wavelengths(350, 420, 64)
    pick = bench.tuning_wavelengths(lam)
    k = np.argmin(np.abs(I.drude_eps(lam) + 2 * I.EPS_WATER))
    assert lam[k] in pick and lam[0] in pick and lam[-1] in pick and len(pick) <= 4
    assert list(bench.tuning_wavelengths(lam, 1)) == [lam[k]]
    assert list(bench.tuning_wavelengths(lam[:3])) == list(lam[:3])


def _terms(P):
    return [(a, b, n - a - b) for n in range(P + 1) for a in range(n, -1, -1) for b in range(n - a, -1, -1)]


@pytest.mark.parametrize("P", [1, 5, 6, 8])
def test_work_counts(P):
    nt = (P + 1) * (P + 2) * (P + 3) // 6
    assert len(_terms(P)) == nt
    # the contraction adds 4 channels x 2 flops per term and right-hand side
    assert bench.m2p_flops(P, 3) - bench.m2p_flops(P, 0) == 8 * nt * 3
    # the recurrence: each term beyond the first reads its lower neighbours along every axis with
    # a nonzero index (2 flops) and with an index >= 2 (1 flop), plus 3 to combine
    rec = sum(2 * sum(d >= 1 for d in k) + sum(d >= 2 for d in k) + 3 for k in _terms(P)[1:])
    assert bench.m2p_flops(P, 0) == 9 + rec
    # G and dG/dn once per pair (18 flops), then 2 kernels x 2 real channels x 2 flops per right-hand side
    assert bench.p2p_flops(16) == 18 + 8 * 16
    assert bench.m2p_terms(P) == nt


def test_tensor_core_m2p_bound():
    # the three terms of the bound scale as stated: generation and SFU once per unit (64
    # right-hand sides above 32: two A parts against one set of coefficients), MMAs with 3
    # products of 2 x 128 x 256 x 8 flops per K step of 8 terms and A part of 32
    pk = {"bf16_tflops_sustained": 1741.2}
    b = bench.m2p_tc_bound(7, 64, 1000, pk, 2070.0)
    nt = 120
    assert b["mufu_ops"] == 1000 * 256
    assert b["mma_flops"] == 1000 * 2 * 3 * 2 * 128 * 256 * 8 * (nt // 8)
    assert b["generation_flops"] == 1000 * 256 * bench.m2p_flops(7, 0)
    b32 = bench.m2p_tc_bound(7, 32, 1000, pk, 2070.0)
    assert b32["mufu_ops"] == 1000 * 256 and b32["mma_flops"] == b["mma_flops"] // 2
    assert b["bound_s"] == max(b["terms_s"].values())
    b16 = bench.m2p_tc_bound(7, 16, 1000, pk, 2070.0)
    assert b16["mma_flops"] == 1000 * 2 * 2 * 128 * 256 * 8 * (nt // 8)


def test_oracle_rate_model():
    wl = bench.WORKLOADS["sphere81920_sweep64"]
    # 64 wavelengths, a product timed on 1000 of 81920 rows in 2 s, 40 oracle steps
    v = bench.oracle_rate(wl, 2.0, 1000, 81920, 40)
    assert np.isclose(v, 64 / (43 * 2.0 * 81.92))


def test_arnoldi_traffic_model():
    # one system-step at j = 0 with a second pass: 7 + 2 vectors, then 3 + 2 more (14 vectors of
    # 2N complex entries of 16 bytes); the counters add linearly over steps
    c = {"system_steps": 1, "vectors": 1, "vectors_second_pass": 1, "system_steps_second_pass": 1}
    assert bench.arnoldi_gb(1000, c) == 14 * 16 * 2000 / 1e9
    c2 = {k: 3 * v for k, v in c.items()}
    assert abs(bench.arnoldi_gb(1000, c2) - 3 * bench.arnoldi_gb(1000, c)) < 1e-15
    # without the second pass: 7 + 2 (j + 1) vectors at j = 4
    c3 = {"system_steps": 1, "vectors": 5, "vectors_second_pass": 0, "system_steps_second_pass": 0}
    assert bench.arnoldi_gb(1000, c3) == 17 * 16 * 2000 / 1e9



def test_tensor_core_p2p_bound_and_roofline():
    # one unit of 64 right-hand sides: the kernel values and the rsqrt once per pair; per stage of
    # 8 sources, two layers x 3 products of 2 x 128 x 256 x 8 flops; a second unit of 6 right-hand
    # sides (70 in all) repeats the generation and issues 2 products per layer
    pk = {"bf16_tflops_sustained": 1741.2}
    pairs, stages = 10 ** 6, 500
    b = bench.p2p_tc_bound(64, pairs, stages, pk, 2070.0)
    assert b["mufu_ops"] == pairs
    assert b["generation_flops"] == pairs * bench.P2P_GEN_FLOPS
    assert b["mma_flops"] == stages * 2 * 3 * 2 * 128 * 256 * 8
    b70 = bench.p2p_tc_bound(70, pairs, stages, pk, 2070.0)
    assert b70["mufu_ops"] == 2 * pairs
    assert b70["mma_flops"] == b["mma_flops"] + stages * 2 * 2 * 2 * 128 * 256 * 8
    # the TF32 peak is the measured sustained bf16 rate x the nominal TF32 / BF16 ratio
    assert np.isclose(b["tf32_peak_tflops"], 1741.2 * bench.TF32_PER_BF16)
    # the roofline entry: frac = bound / launch time, achieved and peak from the limiting term
    assert b["limiter"] == "tensor_mma"
    r = bench.tc_roofline(b, 2 * b["bound_s"], "p2p", None)
    assert r["bound"] == "tensor" and r["frac"] == 0.5
    assert np.isclose(r["achieved"], 0.5 * r["peak"], rtol=1e-3)
