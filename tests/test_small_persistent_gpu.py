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


# ------------------------------------------------------------------ evolution series

def _evolve_both(h, dt, which, x):
    out = torch.empty_like(x)

    def run():
        kg.evolve(h, dt, which, x, out)
        return out.clone()

    return _both(run)


@pytest.mark.parametrize("r", [1, 4])
def test_evolve_series_cluster_is_bitwise_the_per_term_path(r):
    """The Chebyshev-Bessel series of U(+dt), U(-dt) and [X, U(dt)] (Algorithms 6-7) in one
    cluster launch equals the per-term launches bit for bit (same arithmetic, no
    reductions), on every lattice kind (transport along y uses the parity-dependent
    commutator factors), with vacancies and Anderson disorder, and against the oracle."""
    for w in [ki.sheet_cells(12, 9, vacancy_conc=0.03, anderson_w_ev=1.1, lattice_seed=35),
              ki.zgnr(10, 30, vacancy_conc=0.01, lattice_seed=36),
              ki.Workload(ki.AGNR, 11, 40, vacancy_conc=0.02, anderson_w_ev=0.6, lattice_seed=37),
              ki.Workload(ki.SHEET_OPEN_X, 14, 12, vacancy_conc=0.02, lattice_seed=38)]:
        h = kg.from_workload(w)
        ho = oracle.from_workload(w)
        phi = w.vectors(r)
        x = torch.from_numpy(np.ascontiguousarray(phi)).to("cuda")
        for dt in (0.41, 2.0, 9.0):
            tau = oracle.tau_of(ho, dt)
            for which, ref in [(kg.KG_U_FORWARD, lambda v: oracle.evolve(ho, v, tau, +1)),
                               (kg.KG_U_BACKWARD, lambda v: oracle.evolve(ho, v, tau, -1)),
                               (kg.KG_U_COMMUTATOR, lambda v: oracle.evolvex(ho, v, tau))]:
                a, b = _evolve_both(h, dt, which, x)
                assert torch.equal(a, b), (w.kind, dt, which)
                got = a.cpu().numpy()
                want = np.stack([ref(phi[:, k]) for k in range(r)], axis=1)
                assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < 1e-12, (w.kind, dt, which)


def test_evolve_series_long_series_falls_back_to_per_term():
    """A series longer than one cluster launch takes (dt = 40 hbar/gamma0, N_p above 96):
    the per-term launches, still equal to the oracle."""
    w = ki.sheet_cells(8, 8, vacancy_conc=0.02, lattice_seed=39)
    h = kg.from_workload(w)
    ho = oracle.from_workload(w)
    phi = w.vectors(1)
    x = torch.from_numpy(np.ascontiguousarray(phi)).to("cuda")
    assert len(kg.bessel_series(h.emax_ev * 40.0 / w.gamma0_ev, 1e-15)) > 97
    out = torch.empty_like(x)
    kg.timing_enable(h, True)
    kg.evolve(h, 40.0, kg.KG_U_FORWARD, x, out)
    n = kg.timing_read(h)["evolve_launches"]
    kg.timing_enable(h, False)
    assert n > 90
    want = oracle.evolve(ho, phi[:, 0], oracle.tau_of(ho, 40.0), +1)
    assert np.max(np.abs(out.cpu().numpy()[:, 0] - want)) / np.max(np.abs(want)) < 1e-12


@pytest.mark.parametrize("precision,tol", [(kg.KG_FP64, 0.0), (kg.KG_C64, 1e-9)])
def test_vac_and_msd_time_loops_one_series_launch_per_time_step(precision, tol):
    """VAC (two chains U(-dt)A, U(-dt)B) and MSD (U(dt)xi, U(dt)psi and the commutator
    chain) on the 4096-site sheet: one evolution launch per time step, and the moments of
    the cluster path equal to the per-step path (FP64: the propagated vectors are bitwise
    equal, the moments then differ only by the cluster KPM's summation order)."""
    w = ki.sheet_cells(32, 32, vacancy_conc=0.01)
    h = kg.from_workload(w)
    phi = w.vectors(1)
    nc = 6
    for fn in (kg.vac, kg.msd):
        counts = {}
        for cluster in (True, False):
            kg.set_small_persistent(cluster)
            kg.timing_enable(h, True)
            fn(h, phi, 200, nc, 1.0, precision=precision)
            counts[cluster] = kg.timing_read(h)
            kg.timing_enable(h, False)
        kg.set_small_persistent(True)
        assert counts[True]["evolve_launches"] == nc - 1, (fn.__name__, counts[True])
        # the unitarity norms of the nc - 1 steps come with the series launch (no inner-product
        # and reduction launches), and each moment loop's first step with its first cluster
        # launch (no separate first-step reduction): VAC has nc moment loops, MSD nc - 1
        loops = nc if fn is kg.vac else nc - 1
        assert counts[False]["other_launches"] - counts[True]["other_launches"] == 2 * (nc - 1) + loops, fn.__name__
        assert counts[True]["kpm_launches"] == loops * math.ceil((200 - 1 if fn is kg.vac else 100) / 256)
        a, b = _both(lambda: fn(h, phi, 200, nc, 1.0, precision=precision))
        assert _rel(a.reshape(1, -1), b.reshape(1, -1)) < max(tol, TOL_PATHS), fn.__name__
