"""Checkpoint / resume of the time loops and the host-side failure checks.

kg_msd_resume / kg_vac_resume carry the loop state (psi, xi) or (A, B) of Algorithms 2-3
across calls: chaining calls must reproduce one long run bit for bit, in both precisions.
A Bessel truncation far too loose breaks the unitarity of U(dt) (Eq. 36) and must be
reported as KG_ENUMERIC; a capped workspace allocator must give KG_ENOMEM and leave the
handle usable."""
import numpy as np
import pytest

import kg_inputs as ki

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1307_0288_gb300 as kg  # noqa: E402


@pytest.mark.parametrize("precision", [kg.KG_FP64, kg.KG_C64])
def test_msd_resume_reproduces_one_run(precision):
    w = ki.sheet_cells(48, 32, vacancy_conc=0.01, lattice_seed=5)
    h = kg.from_workload(w)
    phi = w.vectors(4)
    m, dt = 300, 2.0
    one = kg.msd(h, phi, m, 6, dt, precision=precision)             # t_0 .. t_5
    mu1, psi, xi = kg.msd_resume(h, phi, None, m, 2, dt, precision=precision)   # t_1, t_2
    mu2, psi, xi = kg.msd_resume(h, psi, xi, m, 3, dt, precision=precision)     # t_3 .. t_5
    assert np.array_equal(mu1, one[:, 1:3])
    assert np.array_equal(mu2, one[:, 3:6])
    # device buffers in and out
    psi_d = torch.from_numpy(psi).cuda()
    xi_d = torch.from_numpy(xi).cuda()
    mu3, psi3, xi3 = kg.msd_resume(h, psi_d, xi_d, m, 1, dt, precision=precision)
    full = kg.msd(h, phi, m, 7, dt, precision=precision)
    assert np.array_equal(mu3[:, 0], full[:, 6])


@pytest.mark.parametrize("precision", [kg.KG_FP64, kg.KG_C64])
def test_vac_resume_reproduces_one_run(precision):
    w = ki.zgnr(10, 96, anderson_w_ev=1.0, lattice_seed=6)
    h = kg.from_workload(w)
    phi = w.vectors(2)
    m, dt = 256, 1.0
    one = kg.vac(h, phi, m, 5, dt, precision=precision)              # t_0 .. t_4
    mu1, a, b = kg.vac_resume(h, phi, None, m, 1, dt, precision=precision)      # t_1
    mu2, a, b = kg.vac_resume(h, a, b, m, 3, dt, precision=precision)           # t_2 .. t_4
    assert np.array_equal(mu1, one[:, 1:2])
    assert np.array_equal(mu2, one[:, 2:5])


@pytest.mark.parametrize("cluster", [True, False])
def test_norm_drift_is_reported(cluster):
    """bessel_tol = 0.5 keeps only J_0 .. J_3 of U(dt) at tau = 3.15: far from unitary.
    Both ways of forming the norms: inside the small-instance series launch (cluster)
    and by separate inner-product launches (one launch per step)."""
    w = ki.sheet_cells(16, 16, vacancy_conc=0.02)
    h = kg.from_workload(w)
    phi = w.vectors(2)
    try:
        kg.set_small_persistent(cluster)
        for fn in (kg.msd, kg.vac):
            with pytest.raises(kg.KgError) as e:
                fn(h, phi, 64, 3, 1.0, bessel_tol=0.5)
            assert e.value.status == -5 and "norm drift" in str(e.value)
        assert np.all(np.isfinite(kg.msd(h, phi, 64, 3, 1.0)))
    finally:
        kg.set_small_persistent(True)


def test_allocation_cap_gives_enomem():
    w = ki.sheet_cells(32, 32)
    h = kg.from_workload(w)
    phi = w.vectors(4)
    ref = kg.dos_moments(h, phi, 100)
    h2 = kg.from_workload(w)
    kg.test_alloc_cap(1 << 16)
    try:
        with pytest.raises(kg.KgError) as e:
            kg.dos_moments(h2, phi, 100)
        assert e.value.status == -2
    finally:
        kg.test_alloc_cap(0)
    assert np.array_equal(kg.dos_moments(h2, phi, 100), ref)
