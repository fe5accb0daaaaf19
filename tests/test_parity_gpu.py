"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same
seeded Hamiltonians and random-phase vectors.

Tolerance: relative error 1e-10 in FP64 with the norm
    max_{n,t} |C_gpu - C_oracle| / max_{n,t} |C_oracle|   per random vector
(the odd DOS moments are O(sqrt N) while C_0 = N, so element-wise relative error is
not meaningful).  Vectors from single products / time steps are compared the same
way at 1e-12.
"""
import numpy as np
import pytest

import kg_inputs as ki
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1307_0288_gb300 as kg  # noqa: E402

TOL_MOMENTS = 1e-10
TOL_VECTOR = 1e-12


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _rel_per_vector(gpu, ora):
    return max(_rel(gpu[r], ora[r]) for r in range(len(ora)))


def _systems():
    return [
        ki.sheet_cells(8, 6, vacancy_conc=0.04, anderson_w_ev=1.0, lattice_seed=17),
        ki.zgnr(9, 14, anderson_w_ev=1.5, vacancy_conc=0.01, lattice_seed=18),
        ki.Workload(ki.AGNR, 9, 24, vacancy_conc=0.03, lattice_seed=19),
        ki.sheet_cells(25, 13, vacancy_conc=0.01, lattice_seed=20),   # 1300 sites: ragged tail
        ki.Workload(ki.SHEET_OPEN_X, 14, 12, vacancy_conc=0.02, anderson_w_ev=0.7, lattice_seed=22),
    ]


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


# ------------------------------------------------------------------ single operators

@pytest.mark.parametrize("r", [1, 4])
def test_apply_matches_oracle(r):
    for w in _systems():
        h = kg.from_workload(w)
        ho = oracle.from_workload(w)
        phi = w.vectors(r)
        x = _dev(phi)
        out = torch.empty_like(x)
        for op, ref in [(kg.KG_OP_H, oracle.apply_h), (kg.KG_OP_XH, oracle.apply_xh),
                        (kg.KG_OP_V, oracle.apply_v)]:
            kg.apply(h, op, x, out)
            got = out.cpu().numpy()
            want = np.stack([ref(ho, phi[:, k]) for k in range(r)], axis=1)
            assert _rel(got, want) < TOL_VECTOR, (w.kind, op)


@pytest.mark.parametrize("dt", [0.41, 2.0])
def test_evolve_matches_oracle(dt):
    for w in _systems():
        h = kg.from_workload(w)
        ho = oracle.from_workload(w)
        tau = oracle.tau_of(ho, dt)
        phi = w.vectors(2)
        x = _dev(phi)
        out = torch.empty_like(x)
        for which, ref in [(kg.KG_U_FORWARD, lambda v: oracle.evolve(ho, v, tau, +1)),
                           (kg.KG_U_BACKWARD, lambda v: oracle.evolve(ho, v, tau, -1)),
                           (kg.KG_U_COMMUTATOR, lambda v: oracle.evolvex(ho, v, tau))]:
            kg.evolve(h, dt, which, x, out)
            got = out.cpu().numpy()
            want = np.stack([ref(phi[:, k]) for k in range(2)], axis=1)
            assert _rel(got, want) < TOL_VECTOR, (w.kind, which)


# ------------------------------------------------------------------ DOS moments

@pytest.mark.parametrize("m", [1, 2, 3, 4, 7, 64, 513])
def test_dos_moments_match_oracle(m):
    for w in _systems():
        h = kg.from_workload(w)
        ho = oracle.from_workload(w)
        phi = w.vectors(4)
        got = kg.dos_moments(h, phi, m)
        want = np.stack([oracle.kpm_moments(ho, phi[:, r], phi[:, r], m) for r in range(4)])
        assert _rel_per_vector(got, want) < TOL_MOMENTS, (w.kind, m)


@pytest.mark.parametrize("r", [1, 2, 8, 16, 32, 64])
def test_dos_moments_every_block_width(r):
    w = ki.zgnr(8, 40, anderson_w_ev=0.8, lattice_seed=21)
    h = kg.from_workload(w)
    ho = oracle.from_workload(w)
    phi = w.vectors(r)
    got = kg.dos_moments(h, phi, 100)
    want = np.stack([oracle.kpm_moments(ho, phi[:, k], phi[:, k], 100) for k in range(r)])
    assert _rel_per_vector(got, want) < TOL_MOMENTS


# ------------------------------------------------------------------ VAC / MSD

def test_vac_matches_oracle_small_sheet_4096_sites():
    """32 x 32 cells (4096 sites), 1 % vacancies, M = 512, one vector, 10 steps of
    dt = 1 hbar/gamma0: the full small VAC workload."""
    w = ki.sheet_cells(32, 32, vacancy_conc=0.01)
    h = kg.from_workload(w)
    ho = oracle.from_workload(w)
    phi = w.vectors(1)
    got = kg.vac(h, phi, 512, 10, 1.0)
    want = oracle.vac_moments(ho, phi[:, 0], 512, 10, 1.0)
    assert _rel(got[0], want) < TOL_MOMENTS


@pytest.mark.parametrize("w", [ki.zgnr(10, 30, anderson_w_ev=2.0, vacancy_conc=0.01, lattice_seed=4),
                               ki.Workload(ki.AGNR, 11, 40, vacancy_conc=0.02, lattice_seed=5)])
def test_vac_matches_oracle_ribbons(w):
    h = kg.from_workload(w)
    ho = oracle.from_workload(w)
    phi = w.vectors(2)
    got = kg.vac(h, phi, 96, 4, 2.0)
    for r in range(2):
        want = oracle.vac_moments(ho, phi[:, r], 96, 4, 2.0)
        assert _rel(got[r], want) < TOL_MOMENTS


def test_msd_matches_oracle_medium_sheet():
    """128 x 64 cells (32768 sites), 0.5 % vacancies, M = 400, 2 vectors, 4 steps of
    dt = 2 hbar/gamma0 (tau = 6.3, N_p = 28)."""
    w = ki.sheet_cells(128, 64, vacancy_conc=0.005)
    h = kg.from_workload(w)
    ho = oracle.from_workload(w)
    phi = w.vectors(2)
    got = kg.msd(h, phi, 400, 4, 2.0)
    assert np.all(got[:, 0] == 0)
    for r in range(2):
        want = oracle.msd_moments(ho, phi[:, r], 400, 4, 2.0)
        assert _rel(got[r], want) < TOL_MOMENTS


@pytest.mark.parametrize("w", [ki.zgnr(10, 30, anderson_w_ev=2.0, vacancy_conc=0.01, lattice_seed=6),
                               ki.Workload(ki.AGNR, 11, 40, vacancy_conc=0.02, lattice_seed=7)])
def test_msd_matches_oracle_ribbons(w):
    h = kg.from_workload(w)
    ho = oracle.from_workload(w)
    phi = w.vectors(4)
    got = kg.msd(h, phi, 65, 3, 1.5)
    for r in range(4):
        want = oracle.msd_moments(ho, phi[:, r], 65, 3, 1.5)
        assert _rel(got[r], want) < TOL_MOMENTS


def test_full_size_msd_sheet_sampled():
    """2048 x 1024 sites (2,097,152), 0.5 % vacancies, 4 vectors, M = 3000, dt = 2, in the
    launch configuration of the benchmark.  The oracle evaluates one time step and the
    first 24 moments of each vector; all 3000 moments obey |C_n| <= C_0 (Chebyshev bound
    |T_n| <= 1 on the spectrum of H~)."""
    w = ki.sheet_cells(1024, 512, vacancy_conc=0.005, n_vec=4)
    h = kg.from_workload(w)
    phi = w.vectors(4)
    got = kg.msd(h, phi, 3000, 2, 2.0)
    c = got[:, 1]
    assert np.all(np.abs(c.imag) == 0)
    assert np.all(np.abs(c.real) <= c[:, :1].real * (1 + 1e-12))
    ho = oracle.from_workload(w)
    for r in range(4):
        want = oracle.msd_moments(ho, phi[:, r], 24, 2, 2.0)[1]
        assert _rel(c[r, :24], want) < TOL_MOMENTS


# ------------------------------------------------------------------ edge cases

def test_all_sites_removed():
    """Every atom removed: trace vectors are zero there, so all moments vanish.  A
    caller's nonzero amplitude on removed atoms behaves as isolated E = 0 sites
    (empty rows of H~), identically in the oracle."""
    w = ki.Workload(ki.SHEET, 8, 4, vacancy_conc=1.0)
    h = kg.from_workload(w)
    assert np.all(kg.dos_moments(h, w.vectors(2), 9) == 0)
    assert np.all(kg.vac(h, w.vectors(2), 9, 3, 1.0) == 0)
    ones = np.ones((w.n_sites, 2), dtype=np.complex128)
    ho = oracle.from_workload(w)
    got = kg.dos_moments(h, ones, 9)
    want = oracle.kpm_moments(ho, ones[:, 0], ones[:, 0], 9)
    assert _rel(got[0], want) < TOL_MOMENTS


def test_single_time_has_no_evolution():
    w = _systems()[0]
    h = kg.from_workload(w)
    ho = oracle.from_workload(w)
    phi = w.vectors(1)
    got = kg.vac(h, phi, 33, 1, 1.0)
    want = oracle.vac_moments(ho, phi[:, 0], 33, 1, 1.0)
    assert _rel(got[0], want) < TOL_MOMENTS
    assert np.all(kg.msd(h, phi, 33, 1, 1.0) == 0)


def test_device_and_host_buffers_give_identical_results():
    w = _systems()[1]
    h = kg.from_workload(w)
    phi = w.vectors(4)
    host = kg.msd(h, phi, 50, 3, 1.0)
    out = torch.zeros((4, 3, 50), dtype=torch.complex128, device="cuda")
    kg.msd(h, _dev(phi), 50, 3, 1.0, out=out)
    assert np.array_equal(out.cpu().numpy(), host)
    again = kg.msd(h, phi, 50, 3, 1.0)
    assert np.array_equal(again, host)           # deterministic reductions


def test_invalid_runs_are_rejected():
    w = _systems()[0]
    h = kg.from_workload(w)
    phi = w.vectors(3)
    with pytest.raises(ValueError):
        kg.dos_moments(h, np.zeros((5, 1)), 10)
    with pytest.raises(kg.KgError):
        kg.dos_moments(h, phi, 10)              # R = 3 is not a power of two
    with pytest.raises(kg.KgError):
        kg.vac(h, w.vectors(1), 10, 3, -1.0)
    with pytest.raises(kg.KgError):
        kg.dos_moments(h, w.vectors(1), 0)


@pytest.mark.parametrize("precision,tol", [(kg.KG_FP64, TOL_MOMENTS), (kg.KG_C64, 2e-5)])
def test_vac_and_msd_at_the_maximum_block_of_64_vectors(precision, tol):
    """R = 64, the largest vector block: the first and last vectors of the block against
    the oracle (the complex64 path runs its float4 pair kernels at their widest)."""
    w = ki.sheet_cells(12, 10, vacancy_conc=0.02, lattice_seed=21, n_vec=64)
    h = kg.from_workload(w)
    ho = oracle.from_workload(w)
    phi = w.vectors(64)
    v = kg.vac(h, phi, 96, 3, 1.0, precision=precision)
    m = kg.msd(h, phi, 96, 3, 2.0, precision=precision)
    for r in (0, 63):
        assert _rel(v[r], oracle.vac_moments(ho, phi[:, r], 96, 3, 1.0)) < tol, r
        assert _rel(m[r], oracle.msd_moments(ho, phi[:, r], 96, 3, 2.0)) < tol, r


def test_fp64_moment_range_and_non_finite_results():
    """The FP64 path forms its inner products in double-float arithmetic: vector entries
    scaled by 2^40 or 2^-40 still give the oracle's moments at 1e-10 (the moments scale
    exactly by 2^80 / 2^-80); NaN entries or entries of 2^70 fail with KG_ENUMERIC."""
    w = _systems()[1]
    h = kg.from_workload(w)
    ho = oracle.from_workload(w)
    phi = w.vectors(2)
    want = np.stack([oracle.kpm_moments(ho, phi[:, r], phi[:, r], 300) for r in range(2)])
    for e in (40, -40):
        got = kg.dos_moments(h, phi * 2.0 ** e, 300) * 2.0 ** (-2 * e)
        assert _rel_per_vector(got, want) < TOL_MOMENTS, e
        got = kg.vac(h, phi * 2.0 ** e, 64, 3, 1.0) * 2.0 ** (-2 * e)
        ref = oracle.vac_moments(ho, phi[:, 0], 64, 3, 1.0)
        assert _rel(got[0], ref) < TOL_MOMENTS, e
    bad = phi.copy()
    bad[5, 1] = np.nan
    for x in (bad, phi * 2.0 ** 70):
        with pytest.raises(kg.KgError) as err:
            kg.dos_moments(h, x, 50)
        assert err.value.status == -5
        with pytest.raises(kg.KgError) as err:
            kg.msd(h, x, 50, 2, 1.0)
        assert err.value.status == -5
    # the handle stays usable
    assert _rel_per_vector(kg.dos_moments(h, phi, 300), want) < TOL_MOMENTS


def test_sigma_pipeline_matches_oracle():
    """sigma^GK (Eq. 6) from VAC moments and sigma^E1 / sigma^E2 (Eqs. 9, 11) from MSD
    moments on the 201-point energy grid: GPU moments + library sums against oracle
    moments + oracle sums (Eqs. 29-31, 35)."""
    from oracle import post
    w = ki.sheet_cells(32, 32, vacancy_conc=0.01)
    h = kg.from_workload(w)
    ho = oracle.from_workload(w)
    phi = w.vectors(2)
    en = post.energy_grid()
    for fn, ofn, dt, formulas in [(kg.vac, oracle.vac_moments, 1.0, [(kg.KG_SIGMA_GK, post.sigma_gk)]),
                                  (kg.msd, oracle.msd_moments, 2.0,
                                   [(kg.KG_SIGMA_E1, post.sigma_e1), (kg.KG_SIGMA_E2, post.sigma_e2)])]:
        mu = fn(h, phi, 512, 8, dt).mean(axis=0)
        mu_o = np.mean([ofn(ho, phi[:, r], 512, 8, dt) for r in range(2)], axis=0)
        dens = kg.kpm_sum(mu.real, en, h.emax_ev, h.area_nm2)
        dens_o = post.kpm_density(mu_o, en, ho.emax_ev, ho.area_nm2)
        t = post.time_grid(8, dt)
        for f, of in formulas:
            s = kg.conductivity(f, dens, t[1])
            so = of(dens_o, t)
            assert _rel(s, so) < TOL_MOMENTS, f


# ------------------------------------------------------------------ Fourier moments (FTM)

def test_ftm_moments_match_oracle():
    for w in _systems()[:3]:
        h = kg.from_workload(w)
        ho = oracle.from_workload(w)
        phi = w.vectors(2)
        got = kg.ftm_dos_moments(h, phi, 15)
        for r in range(2):
            want = oracle.ftm_moments(ho, phi[:, r], phi[:, r], 15)
            assert _rel(got[r], want) < TOL_MOMENTS


def test_kpm_is_cheaper_than_ftm_at_equal_resolution():
    """Sec. 4.2 / Fig. 2 workload: 2048 x 1024 sheet, 1 % vacancies.  KPM with N_m = 1000
    and FTM with 2 N_m + 1 = 1001 give consistent DOS (integrated windows within 5 %);
    at equal energy resolution (FTM N_m' = N_m / (2 pi)) KPM is cheaper by about
    N_p / pi (paper: 20/pi = 6.4; here the doubled moment recursion gives another 2x)."""
    import time
    from oracle import post
    w = ki.sheet_cells(1024, 512, vacancy_conc=0.01)
    h = kg.from_workload(w)
    phi = w.vectors(1)
    kg.dos_moments(h, phi, 64)
    t0 = time.perf_counter(); mu = kg.dos_moments(h, phi, 1000); t_kpm = time.perf_counter() - t0
    t0 = time.perf_counter(); f = kg.ftm_dos_moments(h, phi, 500); t_ftm = time.perf_counter() - t0
    t0 = time.perf_counter(); kg.ftm_dos_moments(h, phi, 80); t_ftm_eq = time.perf_counter() - t0
    en = np.linspace(-8.0, 8.0, 1601)
    rk = kg.kpm_sum(mu[0].real, en, h.emax_ev, h.area_nm2)
    rf = kg.ftm_sum(f[0], en, h.emax_ev, h.area_nm2)
    total = np.trapezoid(rk, en)
    for lo, hi in [(-8, -4), (-4, -1), (-1, 1), (1, 4), (4, 8)]:
        s = (en >= lo) & (en <= hi)
        assert abs(np.trapezoid(rk[s], en[s]) - np.trapezoid(rf[s], en[s])) < 0.05 * total
    print(f"KPM M=1000: {t_kpm:.3f} s, FTM N_m=500: {t_ftm:.3f} s, FTM N_m=80 (equal resolution): {t_ftm_eq:.3f} s")
    assert t_ftm_eq > 3 * t_kpm


def test_clean_zgnr_einstein_conductance_is_quantised():
    """Sec. 5.1 / Fig. 4: a clean zigzag ribbon (8 chains, 8192 cells, 131,072 sites) in the
    ballistic regime.  Where the Bloch bands give one mode (|E| < 1.32 eV), G = (W/L)
    sigma^E1 = 2 e^2/h (spin included); with three modes of different velocities the
    Einstein estimate exceeds 6 e^2/h (sqrt<v^2> > <|v|>, the overshoot the paper discusses)."""
    w = ki.zgnr(8, 8192, n_vec=16)
    h = kg.from_workload(w)
    phi = w.vectors(16)
    m, nc, dt = 1200, 4, 4.0
    dos = kg.dos_moments(h, phi, m).mean(axis=0)
    msd = kg.msd(h, phi, m, nc, dt).mean(axis=0)
    en = np.array([0.6, 0.8, 1.0, 1.7, 1.9])
    rho = kg.kpm_sum(dos.real, en, h.emax_ev, h.area_nm2)
    rdx = kg.kpm_sum(msd.real, en, h.emax_ev, h.area_nm2)
    dt_fs = dt * kg.HBAR_EV_FS / 2.7
    width = 1.5 * w.ny * w.bond_nm
    _, g = kg.ballistic(rho, rdx, dt_fs, width)
    assert np.allclose(g[2, :3], 2.0, rtol=0.05), g[2]
    assert np.all(g[2, 3:] > 6.0 * 0.97) and np.all(g[2, 3:] < 6.0 * 1.6), g[2]


def test_fp64_fma_rate_probe_is_plausible():
    """The in-library FP64 FMA probe (the benchmark's roofline denominator) reports a rate
    within a factor of two of the GB300's nominal 0.625e12 FMA/s (1.25 TFLOP/s), and
    the best of several launches is stable to a few per cent."""
    a = kg.fp64_fma_rate(5)
    b = kg.fp64_fma_rate(5)
    assert 0.3e12 < a < 1.3e12, a
    assert abs(a - b) / max(a, b) < 0.05, (a, b)
