"""GPU: small instances run their moment recursion (Algorithm 5) as one cluster launch
per 256 steps instead of one launch per step.  The cluster kernel uses the per-step
kernels' grid, operations and reduction order, so its moments must equal the per-step
path's bit for bit (that path is checked against the oracle at 1e-10 elsewhere); one
case is also checked against the oracle directly.  Covered: the general (VAC) and the
doubling (DOS, MSD) recursion, on-site disorder, a ragged last CTA, one to three rings
of steps, clusters of 1, 8 and 16 CTAs (16 is above the portable size), complex64, and
a problem too large for one cluster (it keeps one launch per step).
"""
import math

import numpy as np
import pytest

import kg_inputs as ki
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1307_0288_gb300 as kg  # noqa: E402

RING = 256   # recursion steps per cluster launch


def _both(fn):
    """fn() with the cluster path (default) and with one launch per step."""
    try:
        kg.set_small_persistent(True)
        a = fn()
        kg.set_small_persistent(False)
        b = fn()
    finally:
        kg.set_small_persistent(True)
    return a, b


def _kpm_launches(h, fn):
    kg.timing_enable(h, True)
    fn()
    n = kg.timing_read(h)["kpm_launches"]
    kg.timing_enable(h, False)
    return n


def test_vac_small_sheet_bitwise_and_fewer_launches():
    """4096-site sheet, one vector (8 CTAs per step): the small VAC workload's shape."""
    w = ki.sheet_cells(32, 32, vacancy_conc=0.01)
    h = kg.from_workload(w)
    phi = w.vectors(1)
    m, nc = 512, 3
    a, b = _both(lambda: kg.vac(h, phi, m, nc, 1.0))
    assert np.array_equal(a, b)
    steps = m - 2
    kg.set_small_persistent(True)
    assert _kpm_launches(h, lambda: kg.vac(h, phi, m, nc, 1.0)) == nc * (1 + math.ceil(steps / RING))
    try:
        kg.set_small_persistent(False)
        assert _kpm_launches(h, lambda: kg.vac(h, phi, m, nc, 1.0)) == nc * (1 + steps)
    finally:
        kg.set_small_persistent(True)


@pytest.mark.parametrize("m", [3, 4, 5, 258, 259, 600])
def test_vac_ring_boundaries_bitwise(m):
    """Step counts around one ring (M - 2 = 1, 2, 3, 256, 257, 598) on a disordered
    ribbon with a ragged last CTA."""
    w = ki.zgnr(9, 70, anderson_w_ev=1.2, vacancy_conc=0.02, lattice_seed=31)   # 1260 sites
    h = kg.from_workload(w)
    phi = w.vectors(2)
    a, b = _both(lambda: kg.vac(h, phi, m, 2, 0.7))
    assert np.array_equal(a, b)


def test_vac_multi_ring_matches_oracle():
    """Three rings of steps (M = 600) against the oracle at the FP64 tolerance."""
    w = ki.sheet_cells(10, 9, vacancy_conc=0.03, anderson_w_ev=0.9, lattice_seed=32)   # 360 sites
    h = kg.from_workload(w)
    ho = oracle.from_workload(w)
    phi = w.vectors(1)
    got = kg.vac(h, phi, 600, 2, 1.0)
    want = oracle.vac_moments(ho, phi[:, 0], 600, 2, 1.0)
    err = np.max(np.abs(got[0] - want)) / np.max(np.abs(want))
    assert err < 1e-10


@pytest.mark.parametrize("r", [1, 2, 4])
def test_dos_and_msd_cluster_sizes_bitwise(r):
    """4096 sites with R = 1, 2, 4: clusters of 8 and 16 CTAs, and 32 CTAs (too many for
    one cluster: one launch per step, counted)."""
    w = ki.sheet_cells(32, 32, vacancy_conc=0.005, anderson_w_ev=0.5, lattice_seed=33)
    h = kg.from_workload(w)
    phi = w.vectors(r)
    a, b = _both(lambda: kg.dos_moments(h, phi, 1101))
    assert np.array_equal(a, b)
    a, b = _both(lambda: kg.msd(h, phi, 700, 2, 2.0))
    assert np.array_equal(a, b)
    steps = (1101 - 1) // 2
    got = _kpm_launches(h, lambda: kg.dos_moments(h, phi, 1101))
    assert got == (1 + math.ceil(steps / RING) if r <= 2 else 1 + steps)


def test_complex64_one_vector_bitwise():
    w = ki.zgnr(12, 60, anderson_w_ev=1.0, lattice_seed=34)
    h = kg.from_workload(w)
    phi = w.vectors(1)
    a, b = _both(lambda: kg.dos_moments(h, phi, 800, precision=kg.KG_C64))
    assert np.array_equal(a, b)
    a, b = _both(lambda: kg.vac(h, phi, 300, 2, 1.0, precision=kg.KG_C64))
    assert np.array_equal(a, b)
