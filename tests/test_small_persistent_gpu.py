"""GPU: small instances run their moment recursion (Algorithm 5) as one cluster launch
per chunk of up to 256 steps, vectors in the cluster's shared memory, instead of one
launch per step.  The recursion arithmetic is the per-step kernels'; the inner products
are summed in another order, so the moments must agree with the per-step path (itself
checked against the oracle at 1e-10 elsewhere) to 1e-12 in the norm
max|C_cluster - C_step| / max|C_step| per vector, and with the oracle at 1e-10.
Covered: the general (VAC) and the doubling (DOS, MSD) recursion, on-site disorder, a
ragged last CTA, chunk boundaries, one to several chunks, clusters of 1 to 16 CTAs (above
8 is the non-portable size), complex64, and a problem too large for one cluster (it
keeps one launch per step).
"""
import math

import numpy as np
import pytest

import kg_inputs as ki
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1307_0288_gb300 as kg  # noqa: E402

TOL_PATHS = 1e-12   # cluster path vs one launch per step (same vectors, other summation order)
TOL_ORACLE = 1e-10
MIN_CHUNK = 128     # steps per cluster launch at least, for the sizes below


def _rel(a, b):
    return max(float(np.max(np.abs(a[r] - b[r])) / np.max(np.abs(b[r]))) for r in range(len(b)))


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


def test_vac_small_sheet_matches_and_fewer_launches():
    """4096-site sheet, one vector: the small VAC workload (M = 512, 10 times), against
    the oracle, the per-step path, and the launch count."""
    w = ki.sheet_cells(32, 32, vacancy_conc=0.01)
    h = kg.from_workload(w)
    ho = oracle.from_workload(w)
    phi = w.vectors(1)
    m, nc = 512, 10
    a, b = _both(lambda: kg.vac(h, phi, m, nc, 1.0))
    assert _rel(a, b) < TOL_PATHS
    want = oracle.vac_moments(ho, phi[:, 0], m, nc, 1.0)
    assert _rel(a, want[None]) < TOL_ORACLE
    steps = m - 2
    kg.set_small_persistent(True)
    assert _kpm_launches(h, lambda: kg.vac(h, phi, m, nc, 1.0)) <= nc * (1 + math.ceil(steps / MIN_CHUNK))
    try:
        kg.set_small_persistent(False)
        assert _kpm_launches(h, lambda: kg.vac(h, phi, m, nc, 1.0)) == nc * (1 + steps)
    finally:
        kg.set_small_persistent(True)


@pytest.mark.parametrize("m", [3, 4, 5, 258, 259, 600])
def test_vac_chunk_boundaries(m):
    """Step counts around one chunk (M - 2 = 1, 2, 3, 256, 257, 598) on a disordered
    ribbon with a ragged last CTA."""
    w = ki.zgnr(9, 70, anderson_w_ev=1.2, vacancy_conc=0.02, lattice_seed=31)   # 1260 sites
    h = kg.from_workload(w)
    phi = w.vectors(2)
    a, b = _both(lambda: kg.vac(h, phi, m, 2, 0.7))
    assert _rel(a.reshape(2, -1), b.reshape(2, -1)) < TOL_PATHS


def test_vac_multi_ring_matches_oracle():
    """Several chunks of steps (M = 600) against the oracle at the FP64 tolerance."""
    w = ki.sheet_cells(10, 9, vacancy_conc=0.03, anderson_w_ev=0.9, lattice_seed=32)   # 360 sites
    h = kg.from_workload(w)
    ho = oracle.from_workload(w)
    phi = w.vectors(1)
    got = kg.vac(h, phi, 600, 2, 1.0)
    want = oracle.vac_moments(ho, phi[:, 0], 600, 2, 1.0)
    assert _rel(got, want[None]) < TOL_ORACLE


@pytest.mark.parametrize("r", [1, 2, 4])
def test_dos_and_msd_cluster_sizes(r):
    """4096 sites with R = 1, 2, 4: clusters of 16 CTAs (256 and 512 threads), and 4 x 4096
    site-vectors (too many for one cluster: one launch per step, counted)."""
    w = ki.sheet_cells(32, 32, vacancy_conc=0.005, anderson_w_ev=0.5, lattice_seed=33)
    h = kg.from_workload(w)
    ho = oracle.from_workload(w)
    phi = w.vectors(r)
    a, b = _both(lambda: kg.dos_moments(h, phi, 1101))
    assert _rel(a, b) < TOL_PATHS
    want = np.stack([oracle.kpm_moments(ho, phi[:, k], phi[:, k], 1101) for k in range(r)])
    assert _rel(a, want) < TOL_ORACLE
    a, b = _both(lambda: kg.msd(h, phi, 700, 2, 2.0))
    assert _rel(a[:, 1], b[:, 1]) < TOL_PATHS
    steps = (1101 - 1) // 2
    got = _kpm_launches(h, lambda: kg.dos_moments(h, phi, 1101))
    if r <= 2:
        assert got <= 1 + math.ceil(steps / MIN_CHUNK)
    else:
        assert got == 1 + steps


@pytest.mark.parametrize("r", [1, 4])
def test_complex64(r):
    """complex64 vectors (FP32 recursion, compensated sums): the cluster path agrees with
    the per-step path (paired kernels for R >= 2) to the FP32 sums' accuracy."""
    w = ki.zgnr(12, 60, anderson_w_ev=1.0, lattice_seed=34)
    h = kg.from_workload(w)
    phi = w.vectors(r)
    a, b = _both(lambda: kg.dos_moments(h, phi, 800, precision=kg.KG_C64))
    assert _rel(a, b) < 1e-9
    a, b = _both(lambda: kg.vac(h, phi, 300, 2, 1.0, precision=kg.KG_C64))
    assert _rel(a.reshape(r, -1), b.reshape(r, -1)) < 1e-9
