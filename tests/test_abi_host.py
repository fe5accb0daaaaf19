"""CPU tests of the C-ABI library: it loads, exports every entry point that
include/kg.h declares, and its host-side logic (neighbour table, Bessel
coefficients, Jackson damping, Chebyshev sums, running conductivities) agrees
with the oracle.  No GPU compute is called here."""
import os
import re

import numpy as np
import pytest

import kg_inputs as ki
import oracle
import paper_1307_0288_gb300 as kg
from oracle import post

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(kg_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    lib = kg.lib()
    declared = _declared_functions()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), name
    assert {n for n, _, _ in kg.ABI} == declared
    assert kg.abi_version() == 1


def test_neighbor_table_matches_oracle_lattice():
    """The library's slot table (i-1, i+1, adjacent chain) and the oracle's
    distance-based bond search give the same bonds (Sec. 2 lattice)."""
    cases = [ki.sheet_cells(5, 4, vacancy_conc=0.05, lattice_seed=1),
             ki.zgnr(7, 9, vacancy_conc=0.03, lattice_seed=2),
             ki.Workload(ki.AGNR, 9, 12, vacancy_conc=0.04, lattice_seed=3),
             ki.Workload(ki.SHEET, 4, 2),
             ki.Workload(ki.AGNR, 2, 4),
             ki.Workload(ki.SHEET_OPEN_X, 7, 6, vacancy_conc=0.05, lattice_seed=4),
             ki.Workload(ki.SHEET_OPEN_X, 2, 2)]
    for w in cases:
        idx = kg.lattice_neighbors(w.kind, w.nx, w.ny, w.vacancies)
        h = oracle.from_workload(w)
        for n in range(w.n_sites):
            lib_set = sorted(int(m) for m in idx[:, n] if m >= 0)
            ora_set = sorted(int(m) for m in h.col[h.row_ptr[n]:h.row_ptr[n + 1]])
            assert lib_set == ora_set, (w.kind, n, lib_set, ora_set)


def test_invalid_lattices_are_rejected():
    for kind, nx, ny in [(ki.SHEET, 3, 4), (ki.SHEET, 2, 4), (ki.SHEET, 4, 3), (ki.ZGNR, 5, 3),
                         (ki.AGNR, 1, 4), (ki.SHEET, 0, 4), (ki.SHEET_OPEN_X, 1, 4), (ki.SHEET_OPEN_X, 6, 3),
                         (4, 8, 8)]:
        with pytest.raises(kg.KgError) as e:
            kg.lattice_neighbors(kind, nx, ny)
        assert e.value.status == -1
    with pytest.raises(kg.KgError):
        kg.lattice_neighbors(ki.SHEET, 8, 4, vacancies=[3, 3])
    with pytest.raises(kg.KgError):
        kg.lattice_neighbors(ki.SHEET, 8, 4, vacancies=[32])


def test_bessel_series_matches_oracle():
    """Eqs. 36-37: the library's J_m (trapezoid / power series) and N_p agree with the
    oracle's Miller recurrence."""
    for tau in [0.05, 0.41 * 3.15, np.pi, 3.15, 6.3, 9.45, 25.0]:
        j = kg.bessel_series(tau, 1e-15)
        jo, npo = oracle.bessel_series(tau, 1e-15)
        assert len(j) == npo
        assert np.max(np.abs(j - jo)) < 2e-16 * 8


def test_jackson_and_kpm_sum_match_oracle():
    m = 300
    assert np.max(np.abs(kg.jackson(m) - oracle.jackson(m))) < 1e-15
    rng = np.random.default_rng(0)
    mu = rng.normal(size=(3, m)) * np.exp(-np.arange(m) / 60.0)
    en = post.energy_grid()
    ref = post.kpm_density(mu, en, 8.505, 123.4)
    got = kg.kpm_sum(mu, en, 8.505, 123.4)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_conductivity_formulas_match_oracle():
    rng = np.random.default_rng(1)
    d = rng.normal(size=(12, 7))
    t = post.time_grid(12, 2.0)
    dt_fs = t[1]
    assert np.allclose(kg.conductivity(kg.KG_SIGMA_GK, d, dt_fs), post.sigma_gk(d, t), rtol=1e-13, atol=1e-13)
    assert np.allclose(kg.conductivity(kg.KG_SIGMA_E1, d, dt_fs), post.sigma_e1(d, t), rtol=1e-13, atol=1e-13)
    assert np.allclose(kg.conductivity(kg.KG_SIGMA_E2, d, dt_fs), post.sigma_e2(d, t), rtol=1e-13, atol=1e-13)


def test_gpu_entry_points_fail_loudly_without_a_device():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(kg.KgError) as e:
        kg.build_hamiltonian(ki.SHEET, 8, 8, emax_ev=8.505)
    assert e.value.status == -6


def test_ftm_sum_matches_oracle():
    rng = np.random.default_rng(5)
    nm = 40
    f = rng.normal(size=(2, 2 * nm + 1)) + 1j * rng.normal(size=(2, 2 * nm + 1))
    en = post.energy_grid()
    ref = post.ftm_density(f, en, 8.505, 77.7)
    got = kg.ftm_sum(f, en, 8.505, 77.7)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_ballistic_sigma_sc_and_pade_match_oracle():
    rng = np.random.default_rng(9)
    t = post.time_grid(16, 2.0)
    rho = rng.uniform(0.01, 0.1, size=7)
    rdx = np.cumsum(rng.uniform(0, 1, size=(16, 7)), axis=0) * rho
    rdx[0] = 0
    l1, g1 = kg.ballistic(rho, rdx, t[1], 9.0)
    l2, g2 = post.ballistic(rho, rdx, t, 9.0)
    assert np.allclose(l1, l2, rtol=1e-13) and np.allclose(g1, g2, rtol=1e-12, atol=1e-14)
    sig = rng.normal(size=(16, 7))
    mx, av = kg.sigma_sc(sig, t[1], t[3], t[12])
    assert np.allclose(mx, post.sigma_sc_max(sig))
    assert np.allclose(av, post.sigma_sc_average(sig, t, t[3], t[12]), rtol=1e-12)
    tt = np.linspace(1.0, 300.0, 80)
    y = 40 * tt / (1 + 0.05 * tt) + rng.normal(scale=0.05, size=80)
    c1 = kg.pade_fit(tt, y)
    c2 = post.pade_fit(tt, y)
    v1, d1 = kg.pade_eval(c1, tt)
    assert np.allclose(v1, post.pade_value(c2, tt), rtol=1e-6)
    fd = (post.pade_value(c1, tt + 1e-4) - post.pade_value(c1, tt - 1e-4)) / 2e-4
    assert np.allclose(d1, fd, rtol=1e-5)
    t2 = np.arange(100) * 20.0 + 200.0
    y2 = 400.0 * (1.0 - np.exp(-t2 / 600.0)) + rng.normal(scale=4.0, size=100)
    p1 = kg.pade_fit(t2, y2, positive=True)
    p2 = post.pade_fit_positive(t2, y2)
    assert np.all(p1[3:] >= 0)
    r1 = np.sum((post.pade_value(p1, t2) - y2) ** 2)
    r2 = np.sum((post.pade_value(p2, t2) - y2) ** 2)
    assert r1 <= r2 * (1 + 1e-6)
    assert np.allclose(post.pade_value(p1, t2), post.pade_value(p2, t2), rtol=1e-4)


def test_noalloc_binding_rejects_mismatched_buffers_before_the_library():
    """dos_moments_noalloc hands raw device pointers to a C entry point that cannot see
    buffer sizes, so the binding checks every tensor first: a short mu, an int64 or
    transposed neighbour table, a wrong dtype, or a host tensor raises ValueError
    (on a CPU-only machine, before any library call)."""
    torch = pytest.importorskip("torch")
    n, r, m = 64, 2, 16
    idx = torch.zeros((3, n), dtype=torch.int32)
    onsite = torch.zeros(n, dtype=torch.float64)
    phi = torch.zeros((n, r), dtype=torch.complex128)
    mu = torch.zeros((r, m), dtype=torch.complex128)
    bad = [
        dict(mu_dev=torch.zeros((r - 1, m), dtype=torch.complex128)),   # fewer rows than vectors
        dict(mu_dev=torch.zeros((r, m), dtype=torch.complex64)),
        dict(idx_dev=torch.zeros((3, n), dtype=torch.int64)),
        dict(idx_dev=torch.zeros((n, 3), dtype=torch.int32)),
        dict(idx_dev=torch.zeros((3, n - 1), dtype=torch.int32)),
        dict(onsite_dev=torch.zeros(n - 1, dtype=torch.float64)),
        dict(onsite_dev=torch.zeros(n, dtype=torch.float32)),
        dict(phi_dev=torch.zeros((n + 1, r), dtype=torch.complex128)),
        dict(phi_dev=torch.zeros((n, r), dtype=torch.float64)),
    ]
    for change in bad:
        args = dict(idx_dev=idx, onsite_dev=onsite, phi_dev=phi, mu_dev=mu)
        args.update(change)
        with pytest.raises(ValueError):
            kg.dos_moments_noalloc(args["idx_dev"], args["onsite_dev"], n, -0.3, args["phi_dev"],
                                   args["mu_dev"])
    # right shapes, but host tensors (or a non-contiguous view): still refused
    with pytest.raises(ValueError, match="CUDA|contiguous"):
        kg.dos_moments_noalloc(idx, onsite, n, -0.3, phi, mu)
    with pytest.raises(ValueError):
        kg.dos_moments_noalloc(idx, onsite, n, -0.3, phi, torch.zeros((m, r), dtype=torch.complex128).t())


def test_seeded_inputs_from_the_c_abi_match_the_input_module():
    """The library's SplitMix64 input generators (kg_splitmix64, kg_n_vacancies,
    kg_vacancy_sites, kg_anderson_onsite, kg_random_phase_vectors) reproduce the Python
    input module: words, vacancy sites, Anderson energies and the phases bit for bit,
    the cos/sin of the phases within one unit in the last place (both call the C
    library here; exact when the platform's numpy and libm agree)."""
    for seed, stream in [(20130701, 0), (1000, 16), (2**64 - 1, 5)]:
        assert np.array_equal(kg.splitmix64(seed, stream, 1000, start=7),
                              ki.splitmix64(seed, stream, 1000, start=7))
    for n, conc in [(4096, 0.01), (2097152, 0.005), (1000, 0.0025), (10, 0.05)]:
        assert kg.n_vacancies(n, conc) == ki.n_vacancies(n, conc)
    for w in [ki.sheet_cells(32, 32, vacancy_conc=0.01), ki.zgnr(20, 100, vacancy_conc=0.02, lattice_seed=9),
              ki.sheet_cells(64, 32, vacancy_conc=0.005, anderson_w_ev=1.5, lattice_seed=3, vector_seed=77)]:
        nv = kg.n_vacancies(w.n_sites, w.vacancy_conc)
        vac = kg.vacancy_sites(w.n_sites, nv, w.lattice_seed)
        assert np.array_equal(vac, w.vacancies)
        if w.anderson_w_ev > 0:
            assert np.array_equal(kg.anderson_onsite(w.n_sites, w.anderson_w_ev, w.lattice_seed), w.onsite)
        got = kg.random_phase_vectors(w.n_sites, 3, w.vector_seed, vac)
        want = w.vectors(3)
        ulp = np.spacing(np.maximum(np.abs(want.real), np.abs(want.imag)).max(initial=1.0))
        assert np.max(np.abs(got - want)) <= ulp
        assert np.all(got[vac] == 0)
        print(f"{w.n_sites} sites: phase vectors bit-identical: {np.array_equal(got, want)}")


def test_jackknife_error_of_sigma_sc_plateau():
    """The jackknife over random vectors (regimes.jackknife_sigma_sc): identical vectors
    give a zero error; for sigma_sc by block average, a linear function of the averaged
    moments (Chebyshev sum, Eq. 31; central differences, Eq. 9; block average, Eq. 54),
    the jackknife standard error equals the textbook standard error of the mean of the
    single-vector estimates."""
    from paper_1307_0288_gb300 import regimes
    rng = np.random.default_rng(5)
    n, nt, m = 7, 12, 64
    en = np.linspace(-1.0, 1.0, 21)
    base_d = np.zeros(m)
    base_d[0] = 1000.0
    base_m = np.outer(np.arange(nt) ** 2, np.exp(-np.arange(m) / 8.0)) * 50.0
    c = {"t_fs": np.arange(nt) * 0.5, "energies": en, "emax_ev": 8.5, "area_nm2": 400.0,
         "mu_dos_r": np.tile(base_d, (n, 1)), "mu_msd_r": np.tile(base_m, (n, 1, 1))}
    plateau = np.abs(en) <= 0.3
    jm, se_max, ja, se_avg, nj = regimes.jackknife_sigma_sc(c, (1.0, 4.0), plateau)
    assert nj == n and se_max <= 1e-12 * abs(jm) and se_avg <= 1e-12 * abs(ja)   # rounding only
    c["mu_msd_r"] = base_m[None] * (1.0 + 0.2 * rng.standard_normal((n, 1, 1))) + \
        rng.standard_normal((n, nt, m)) * 5.0
    jm, se_max, ja, se_avg, _ = regimes.jackknife_sigma_sc(c, (1.0, 4.0), plateau)
    single = []
    for i in range(n):
        rdx = kg.kpm_sum(c["mu_msd_r"][i], en, 8.5, 400.0)
        s = kg.conductivity(kg.KG_SIGMA_E1, rdx, 0.5)
        single.append(kg.sigma_sc(s, 0.5, 1.0, 4.0)[1][plateau].mean())
    single = np.array(single)
    assert se_avg > 0
    assert abs(se_avg - single.std(ddof=1) / np.sqrt(n)) < 1e-9 * max(1.0, se_avg)
    assert abs(ja - single.mean()) < 1e-9 * max(1.0, abs(ja))


def test_fp64_fma_rate_rejects_bad_arguments():
    """kg_fp64_fma_rate validates its arguments before touching a GPU."""
    for bad in (0, 101, -3):
        with pytest.raises(kg.KgError) as e:
            kg.fp64_fma_rate(bad)
        assert e.value.status == -1


def test_mlp_forward_checks_shapes_and_output_dtype():
    """The inference kernel reads device inputs and writes device outputs in place, so the
    binding rejects a wrong input shape or an output of the wrong dtype or size before the
    library is called (checked without a GPU on an unconstructed handle)."""
    net = object.__new__(kg.Mlp)
    net._m = None
    x = np.zeros((10, 3), dtype=np.float32)
    with pytest.raises(ValueError):
        net.forward(np.zeros((10, 4), dtype=np.float32))
    with pytest.raises(ValueError):
        net.forward(x, out=np.zeros(10, dtype=np.float64))
    with pytest.raises(ValueError):
        net.forward(x, out=np.zeros(9, dtype=np.float32))
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        net.forward(torch.zeros((10, 3), dtype=torch.float32), out=torch.zeros(10, dtype=torch.float16))
