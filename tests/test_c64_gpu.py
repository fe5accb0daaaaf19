"""Mixed precision (KG_C64): complex64 recursion vectors and FP32 recursion
arithmetic, with compensated FP32 per-thread inner products combined in FP64, and
FP64 Bessel/Jackson coefficients, moments and time integration.

Errors are stated against the FP64 oracle for the moments (norm: max |dC| / max |C|
per vector) and against the FP64 GPU path for sigma(E, t) (max over E and t of
|d sigma| / max |sigma|), the quantity the precision mode is held to (<= 1e-5).
"""
import numpy as np
import pytest

import kg_inputs as ki
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1307_0288_gb300 as kg  # noqa: E402

# FP32 storage rounds each vector element to 2^-24 relative at every recursion step;
# the error of the Chebyshev recursion grows at most linearly in the step count, so
# moments up to n ~ 10^3 carry ~1e-5 of C_0 at worst.
TOL_C64_MOMENTS = 2e-5
TOL_C64_SIGMA = 1e-5


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def test_c64_dos_moments_vs_oracle():
    for w in [ki.sheet_cells(32, 32, vacancy_conc=0.01), ki.zgnr(12, 64, anderson_w_ev=1.0, lattice_seed=3)]:
        h = kg.from_workload(w)
        ho = oracle.from_workload(w)
        phi = w.vectors(4)
        got = kg.dos_moments(h, phi, 1000, precision=kg.KG_C64)
        want = np.stack([oracle.kpm_moments(ho, phi[:, r], phi[:, r], 1000) for r in range(4)])
        errs = [_rel(got[r], want[r]) for r in range(4)]
        en = np.linspace(-3 * 2.7, 3 * 2.7, 201)
        rho_err = _rel(kg.kpm_sum(got.mean(axis=0).real, en, h.emax_ev, h.area_nm2),
                       kg.kpm_sum(want.mean(axis=0).real, en, h.emax_ev, h.area_nm2))
        print(f"c64 DOS vs oracle ({w.n_sites} sites): moments {max(errs):.2e}, rho(E) {rho_err:.2e}")
        assert max(errs) < TOL_C64_MOMENTS
        assert rho_err < TOL_C64_MOMENTS


def test_c64_vac_and_msd_vs_oracle():
    w = ki.sheet_cells(32, 32, vacancy_conc=0.01)
    h = kg.from_workload(w)
    ho = oracle.from_workload(w)
    phi = w.vectors(1)
    v = kg.vac(h, phi, 512, 10, 1.0, precision=kg.KG_C64)
    vo = oracle.vac_moments(ho, phi[:, 0], 512, 10, 1.0)
    m = kg.msd(h, phi, 512, 6, 2.0, precision=kg.KG_C64)
    mo = oracle.msd_moments(ho, phi[:, 0], 512, 6, 2.0)
    errs = {"VAC moments": _rel(v[0], vo), "MSD moments": _rel(m[0], mo),
            "sigma GK": _rel(_sigma(h, v, 1.0, kg.KG_SIGMA_GK), _sigma(h, vo[None], 1.0, kg.KG_SIGMA_GK)),
            "sigma E1": _rel(_sigma(h, m, 2.0, kg.KG_SIGMA_E1), _sigma(h, mo[None], 2.0, kg.KG_SIGMA_E1))}
    print("c64 vs oracle (4096 sites):", {k: f"{e:.2e}" for k, e in errs.items()})
    assert max(errs.values()) < TOL_C64_MOMENTS, errs


def _sigma(h, mu, dt, formula):
    """sigma(E, t) in e^2/h on the 201-point energy grid from vector-averaged moments."""
    en = np.linspace(-3 * 2.7, 3 * 2.7, 201)
    dens = kg.kpm_sum(mu.mean(axis=0).real, en, h.emax_ev, h.area_nm2)
    return kg.conductivity(formula, dens, dt * kg.HBAR_EV_FS / 2.7)


def test_c64_sigma_within_1e5_of_fp64_gpu():
    """sigma^GK (VAC) and sigma^E1 (MSD) from complex64 vectors vs the FP64 GPU path,
    on a 256 x 128-cell sheet (131,072 sites) with 1 % vacancies."""
    w = ki.sheet_cells(256, 128, vacancy_conc=0.01)
    h = kg.from_workload(w)
    phi = w.vectors(4)
    errs = {}
    for name, fn, dt, formula in [("GK", kg.vac, 1.0, kg.KG_SIGMA_GK),
                                  ("E1", kg.msd, 2.0, kg.KG_SIGMA_E1)]:
        ref = _sigma(h, fn(h, phi, 1000, 12, dt), dt, formula)
        got = _sigma(h, fn(h, phi, 1000, 12, dt, precision=kg.KG_C64), dt, formula)
        errs[name] = _rel(got, ref)
    print("c64 sigma relative error", errs)
    assert max(errs.values()) < TOL_C64_SIGMA, errs


def test_c64_full_size_sheet_sampled():
    """4096 x 2048 sites (8,388,608), 1 % vacancies, 8 vectors, M = 6000, one MSD step:
    complex64 moments vs the FP64 GPU path on the same inputs; the first 24 moments
    of two vectors also vs the oracle."""
    w = ki.sheet_cells(2048, 1024, vacancy_conc=0.01, n_vec=8)
    h = kg.from_workload(w)
    phi = w.vectors(8)
    c64 = kg.msd(h, phi, 6000, 2, 2.0, precision=kg.KG_C64)[:, 1]
    f64 = kg.msd(h, phi, 6000, 2, 2.0)[:, 1]
    errs = [_rel(c64[r], f64[r]) for r in range(8)]
    print(f"c64 vs FP64 GPU, 8.4M sites, M = 6000: MSD moments {max(errs):.2e}")
    assert max(errs) < TOL_C64_MOMENTS
    ho = oracle.from_workload(w)
    for r in range(2):
        want = oracle.msd_moments(ho, phi[:, r], 24, 2, 2.0)[1]
        assert _rel(c64[r, :24], want) < TOL_C64_MOMENTS
