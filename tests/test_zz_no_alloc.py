"""The no-allocation DOS entry point (kg_dos_moments_noalloc) against the allocating
one (kg_dos_moments).

kg_dos_moments_noalloc is for callers that cannot call cudaMalloc (their device
memory belongs to a host framework's allocator, or they must not allocate once
serving): it keeps its scratch in one fixed device array instead.  This file is
collected last so that a stopping run has already run every other test; it passes
alone in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

import kg_inputs as ki

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1307_0288_gb300 as kg  # noqa: E402

TOL_MOMENTS = 1e-10   # same norm and tolerance as the oracle parity tests


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _noalloc(w, phi, m):
    idx = torch.from_numpy(kg.lattice_neighbors(w.kind, w.nx, w.ny, w.vacancies)).to("cuda")
    onsite = None
    if w.onsite is not None:
        onsite = torch.from_numpy(np.where(w.vacancy_mask() > 0, 0.0, w.onsite / w.emax_ev)).to("cuda")
    phi_dev = torch.from_numpy(np.ascontiguousarray(phi)).to("cuda")
    mu = torch.full((phi.shape[1], m), np.nan, dtype=torch.complex128, device="cuda")
    kg.dos_moments_noalloc(idx, onsite, w.n_sites, -w.gamma0_ev / w.emax_ev, phi_dev, mu)
    return mu.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls():
    """Two calls in a row with different sizes: the second must not see the first
    call's leftovers in the shared scratch array."""
    cases = [(ki.sheet_cells(40, 24, vacancy_conc=0.02, anderson_w_ev=1.0, lattice_seed=31), 4, 301),
             (ki.zgnr(9, 70, vacancy_conc=0.01, lattice_seed=32), 1, 64),
             (ki.sheet_cells(40, 24, vacancy_conc=0.02, anderson_w_ev=1.0, lattice_seed=31), 4, 301)]
    for w, r, m in cases:
        phi = w.vectors(r)
        h = kg.from_workload(w)
        ref = kg.dos_moments(h, phi, m)
        got = _noalloc(w, phi, m)
        assert np.all(np.isfinite(got))
        for k in range(r):
            assert _rel(got[k], ref[k]) < TOL_MOMENTS


def test_noalloc_rejects_problems_beyond_the_fixed_scratch():
    n = 2048 * 1024
    idx = torch.full((3, n), -1, dtype=torch.int32, device="cuda")
    phi = torch.zeros((n, 4), dtype=torch.complex128, device="cuda")
    mu = torch.zeros((4, 8), dtype=torch.complex128, device="cuda")
    with pytest.raises(kg.KgError) as e:
        kg.dos_moments_noalloc(idx, None, n, -2.7 / 8.505, phi, mu)
    assert e.value.status == -1 and "scratch" in str(e.value)


def test_noalloc_onsite_on_removed_sites_and_the_spectral_bound():
    """Raw Anderson energies left on the removed sites give the same moments when phi
    is zero there (the removed rows have no bonds, so they stay zero); on-site energies
    that push the spectrum of H~ outside [-1, 1] are refused with KG_EINVAL."""
    w = ki.sheet_cells(24, 16, vacancy_conc=0.03, anderson_w_ev=1.5, lattice_seed=33)
    phi = w.vectors(2)
    assert np.all(phi[w.vacancy_mask() > 0] == 0)
    h = kg.from_workload(w)
    ref = kg.dos_moments(h, phi, 200)
    idx = torch.from_numpy(kg.lattice_neighbors(w.kind, w.nx, w.ny, w.vacancies)).to("cuda")
    raw = torch.from_numpy(np.ascontiguousarray(w.onsite / w.emax_ev)).to("cuda")
    assert float(raw[torch.from_numpy(w.vacancy_mask() > 0).to("cuda")].abs().max()) > 0
    phi_dev = torch.from_numpy(np.ascontiguousarray(phi)).to("cuda")
    mu = torch.zeros((2, 200), dtype=torch.complex128, device="cuda")
    kg.dos_moments_noalloc(idx, raw, w.n_sites, -w.gamma0_ev / w.emax_ev, phi_dev, mu)
    got = mu.cpu().numpy()
    for k in range(2):
        assert _rel(got[k], ref[k]) < TOL_MOMENTS
    too_large = raw * 0 + 0.2   # 3 * 2.7 / E_max + 0.2 = 1.07 > 1
    with pytest.raises(kg.KgError) as e:
        kg.dos_moments_noalloc(idx, too_large, w.n_sites, -w.gamma0_ev / w.emax_ev, phi_dev, mu)
    assert e.value.status == -1 and "inside [-1, 1]" in str(e.value)
