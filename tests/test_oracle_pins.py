"""Pins for the CPU oracle: each test checks the oracle against something other
than itself -- exact diagonalisation, closed forms, a library routine, a sum
rule, or a number printed in the paper -- so that a plausible mistake (a
dropped term, a wrong sign or index, a transposed operand) fails at least one.
``test_planted_mistakes_are_caught`` plants such mistakes in the oracle and
checks that they are caught.
"""
import os

import numpy as np
import pytest
from scipy import special
from scipy.special import jv

import kg_inputs as ki
import oracle
from oracle import post

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
A_NM = 0.142
G0 = 2.7


def _golden(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def _rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300)


def _systems():
    """Small disordered systems (<= 512 sites) used for exact diagonalisation."""
    return [
        ki.sheet_cells(4, 4, vacancy_conc=0.05, anderson_w_ev=1.0, lattice_seed=7),
        ki.sheet_cells(8, 4, vacancy_conc=0.02, lattice_seed=11),
        ki.zgnr(6, 12, anderson_w_ev=2.0, vacancy_conc=0.01, lattice_seed=3),
        ki.Workload(ki.AGNR, 9, 20, vacancy_conc=0.03, anderson_w_ev=0.5, lattice_seed=5),
        ki.Workload(ki.SHEET_OPEN_X, 10, 16, vacancy_conc=0.02, anderson_w_ev=0.8, lattice_seed=9),
    ]


class _ED:
    """Exact diagonalisation of the oracle's dense H~ (numpy eigh)."""

    def __init__(self, h):
        self.h = h
        self.e, self.v = np.linalg.eigh(h.dense())
        self.d = self.v.T @ h.dense_xh() @ self.v     # [X, H~] in the eigenbasis

    def moments(self, l, r, m):
        a = self.v.T @ l
        b = self.v.T @ r
        t = np.cos(np.outer(np.arange(m), np.arccos(np.clip(self.e, -1, 1))))
        return t @ (np.conj(a) * b)

    def u(self, x, tau):
        """exp(-i H~ tau) x."""
        return self.v @ (np.exp(-1j * tau * self.e) * (self.v.T @ x))

    def xu(self, x, tau):
        """[X, exp(-i H~ tau)] x by divided differences in the eigenbasis."""
        ej, ek = np.meshgrid(self.e, self.e, indexing="ij")
        de = ek - ej
        small = np.abs(de) < 1e-12
        with np.errstate(divide="ignore", invalid="ignore"):
            dd = -2j * np.exp(-0.5j * tau * (ej + ek)) * np.sin(0.5 * tau * de) / de
        dd[small] = (-1j * tau * np.exp(-1j * tau * ek))[small]
        return self.v @ ((self.d * dd) @ (self.v.T @ x))


def _vec(n, seed, vac=None):
    return ki.random_phase_vectors(n, 1, seed, vac)[:, 0]


# ------------------------------------------------------------------ geometry / lattice

def test_sample_lengths_match_printed_values():
    """L_x = sqrt(3) N_x a / 2 reproduces the sample sizes printed in Sec. 5."""
    for nx, length, tol, _ in _golden("geometry.txt"):
        h = oracle.build_hamiltonian(ki.AGNR if int(nx) % 2 else ki.SHEET, int(nx), 4,
                                     emax_ev=8.505)
        lx = h.area_nm2 / (1.5 * 4 * A_NM)
        assert abs(lx - float(length)) < float(tol), (nx, lx)


def test_lattice_is_bipartite_honeycomb():
    """Every bulk site has 3 neighbours, bonds are symmetric, the graph is bipartite
    (two-colourable), and the x-displacements are 0 or +-sqrt(3)a/2 (Sec. 2)."""
    h = oracle.build_hamiltonian(ki.SHEET, 16, 12, emax_ev=8.505)
    deg = np.diff(h.row_ptr)
    assert np.all(deg == 3)
    hd = h.dense()
    assert np.array_equal(hd, hd.T)
    colour = -np.ones(h.n, dtype=int)
    colour[0] = 0
    stack = [0]
    while stack:
        u = stack.pop()
        for k in range(h.row_ptr[u], h.row_ptr[u + 1]):
            w = h.col[k]
            if colour[w] < 0:
                colour[w] = 1 - colour[u]
                stack.append(w)
            assert colour[w] != colour[u]
    assert np.allclose(np.sort(np.unique(np.round(np.abs(h.disp), 12))),
                       [0.0, np.sqrt(3) * A_NM / 2])
    assert len(h.col) == 3 * h.n          # 3N/2 bonds, both directions stored


def test_pristine_spectrum_matches_bloch_bands():
    """Eigenvalues of a pristine periodic sheet equal +-gamma0 |sum_delta exp(i k.delta)|
    on the sample's k-grid (textbook graphene bands; Sec. 2 Hamiltonian)."""
    nx, ny = 12, 8
    emax = 8.505
    h = oracle.build_hamiltonian(ki.SHEET, nx, ny, emax_ev=emax)
    ev = np.sort(np.linalg.eigvalsh(h.dense()) * emax)
    lx, ly = np.sqrt(3) * nx * A_NM / 2, 1.5 * ny * A_NM
    deltas = np.array([[np.sqrt(3) * A_NM / 2, -A_NM / 2], [-np.sqrt(3) * A_NM / 2, -A_NM / 2],
                       [0.0, A_NM]])
    bands = []
    for p in range(nx):
        for q in range(ny):
            k = np.array([2 * np.pi * p / lx, 2 * np.pi * q / ly])
            f = np.abs(np.exp(1j * deltas @ k).sum())
            bands += [G0 * f, -G0 * f]
    bands = np.sort(bands)[::2]           # every k of the grid appears twice
    assert np.max(np.abs(ev - bands)) < 1e-10


# ------------------------------------------------------------------ Chebyshev moments

def test_kpm_moments_match_exact_diagonalisation():
    """C_n = <L|T_n(H~)|R> (Algorithm 5) equals sum_k conj(L_k) R_k cos(n arccos e_k)."""
    for w in _systems():
        h = oracle.from_workload(w)
        ed = _ED(h)
        l = _vec(h.n, 1, w.vacancies)
        r = _vec(h.n, 2, w.vacancies) * (1 + 0.3j)
        for (a, b) in [(l, l), (l, r)]:
            c = oracle.kpm_moments(h, a, b, 200)
            assert _rel(c, ed.moments(a, b, 200)) < 1e-12


def test_exact_trace_moments_match_bloch_sum():
    """Tr T_n(H~) summed over basis vectors equals sum over the Bloch bands of
    T_n(E_k / E_max); odd moments vanish (bipartite lattice)."""
    nx, ny, emax, m = 8, 6, 8.505, 40
    h = oracle.build_hamiltonian(ki.SHEET, nx, ny, emax_ev=emax)
    tr = np.zeros(m, dtype=complex)
    for j in range(h.n):
        e = np.zeros(h.n, dtype=complex)
        e[j] = 1.0
        tr += oracle.kpm_moments(h, e, e, m)
    lx, ly = np.sqrt(3) * nx * A_NM / 2, 1.5 * ny * A_NM
    deltas = np.array([[np.sqrt(3) * A_NM / 2, -A_NM / 2], [-np.sqrt(3) * A_NM / 2, -A_NM / 2],
                       [0.0, A_NM]])
    eps = []
    for p in range(nx):
        for q in range(ny):
            k = np.array([2 * np.pi * p / lx, 2 * np.pi * q / ly])
            f = G0 * np.abs(np.exp(1j * deltas @ k).sum()) / emax
            eps += [f, -f]
    eps = np.array(eps)
    bloch = 0.5 * np.cos(np.outer(np.arange(m), np.arccos(eps))).sum(axis=1)
    assert _rel(tr, bloch) < 1e-12
    assert np.max(np.abs(tr[1::2])) < 1e-12 * h.n


# ------------------------------------------------------------------ Bessel coefficients

def test_bessel_matches_library_and_sum_rule():
    """Miller recurrence J_m(x) vs scipy.special.jv; J_0 + 2 sum J_2k = 1 (A&S 9.1.46)."""
    for x in [1e-3, 0.41, np.pi, 3.15, 6.3, 12.6, 30.0]:
        j = oracle.bessel_j(x, 80)
        ref = jv(np.arange(81), x)
        big = np.abs(ref) > 1e-290
        assert np.max(np.abs(j[big] - ref[big]) / np.maximum(np.abs(ref[big]), 1e-300)
                      * (np.abs(ref[big]) > 1e-200)) < 1e-12
        assert abs(j[0] + 2 * j[2::2].sum() - 1) < 1e-14


def test_bessel_term_count_matches_printed_value():
    """Sec. 4.2: argument pi, accuracy 1e-15 -> about N_p = 20 terms."""
    for x, tol, printed, dev, _ in _golden("bessel_terms.txt"):
        n = oracle.bessel_terms(float(x), float(tol))
        assert abs(n - int(printed)) <= int(dev)
        j = jv(np.arange(n + 5), float(x))
        assert abs(j[n]) < float(tol) and abs(j[n - 1]) >= float(tol)


# ------------------------------------------------------------------ time evolution

def test_evolve_matches_exact_propagator_and_is_unitary():
    """Eq. (36): U(+dt) = exp(-i H~ tau), U(-dt) = U(dt)^dagger; norm conserved,
    U(-dt)U(dt) = 1, U(dt)U(dt) = U(2dt)."""
    for w in _systems():
        h = oracle.from_workload(w)
        ed = _ED(h)
        x = _vec(h.n, 4, w.vacancies)
        for tau in [0.41 * 3.15, 3.15, 6.3]:
            up = oracle.evolve(h, x, tau, +1)
            um = oracle.evolve(h, x, tau, -1)
            assert _rel(up, ed.u(x, tau)) < 1e-13
            assert _rel(um, ed.u(x, -tau)) < 1e-13
            assert abs(np.linalg.norm(up) / np.linalg.norm(x) - 1) < 1e-13
            assert _rel(oracle.evolve(h, up, tau, -1), x) < 1e-13
            assert _rel(oracle.evolve(h, up, tau, +1), oracle.evolve(h, x, 2 * tau, +1)) < 1e-12


def test_evolvex_matches_divided_differences():
    """Eq. (37): [X, U(dt)] x equals the divided-difference form in the eigenbasis,
    which is what the commutator recursion Eq. (39) sums to."""
    for w in _systems():
        h = oracle.from_workload(w)
        ed = _ED(h)
        x = _vec(h.n, 5, w.vacancies)
        for tau in [1.3, 6.3]:
            assert _rel(oracle.evolvex(h, x, tau), ed.xu(x, tau)) < 1e-12


def test_commutator_iteration_equals_direct_double_step():
    """Eq. (44): [X,U(2dt)]x = U(dt)[X,U(dt)]x + [X,U(dt)]U(dt)x."""
    w = _systems()[0]
    h = oracle.from_workload(w)
    x = _vec(h.n, 6, w.vacancies)
    tau = 3.15
    lhs = oracle.evolvex(h, x, 2 * tau)
    rhs = oracle.evolve(h, oracle.evolvex(h, x, tau), tau, +1) + \
        oracle.evolvex(h, oracle.evolve(h, x, tau, +1), tau)
    assert _rel(rhs, lhs) < 1e-12


# ------------------------------------------------------------------ VAC / MSD loops

def test_vac_moments_match_exact_diagonalisation():
    """Algorithm 2: C^VAC_n(t_m) = <V U^+(t)phi| T_n |U^+(t) V phi> (Eq. 33)."""
    for w in _systems()[:3]:
        h = oracle.from_workload(w)
        ed = _ED(h)
        phi = _vec(h.n, 7, w.vacancies)
        dt, nc, m = 1.0, 4, 64
        tau = oracle.tau_of(h, dt)
        c = oracle.vac_moments(h, phi, m, nc, dt)
        vphi = oracle.apply_v(h, phi)
        for t in range(nc):
            a = ed.u(phi, -t * tau)
            b = ed.u(vphi, -t * tau)
            ref = ed.moments(oracle.apply_v(h, a), b, m)
            assert _rel(c[t], ref) < 1e-11


def test_msd_moments_match_exact_diagonalisation():
    """Algorithm 3: C^MSD_n(t_m) = <[X,U(t)]phi| T_n |[X,U(t)]phi> (Eq. 34)."""
    for w in _systems():
        h = oracle.from_workload(w)
        ed = _ED(h)
        phi = _vec(h.n, 8, w.vacancies)
        dt, nc, m = 2.0, 4, 64
        tau = oracle.tau_of(h, dt)
        c = oracle.msd_moments(h, phi, m, nc, dt)
        assert np.all(c[0] == 0)
        for t in range(1, nc):
            xi = ed.xu(phi, t * tau)
            assert _rel(c[t], ed.moments(xi, xi, m)) < 1e-11


def test_velocity_sum_rule_pristine():
    """Exact trace of V^2 for pristine graphene: each site has two in-chain bonds with
    (X_n - X_m)^2 = 3a^2/4, so Tr V^2 = N (3/2) a^2 gamma0^2 / hbar^2 (Eq. 15)."""
    h = oracle.build_hamiltonian(ki.SHEET, 8, 6, emax_ev=8.505)
    tr = 0.0
    for j in range(h.n):
        e = np.zeros(h.n, dtype=complex)
        e[j] = 1.0
        tr += oracle.vac_moments(h, e, 1, 1, 1.0)[0, 0].real
    exact = h.n * 1.5 * A_NM ** 2 * G0 ** 2 / oracle.HBAR_EV_FS ** 2
    assert abs(tr / exact - 1) < 1e-12


def test_msd_short_time_limit_is_velocity_correlation():
    """[X,U(t)]phi -> t V phi as t -> 0, so C^MSD(t)/t^2 -> C^VAC(0) with O(t)
    error (Eqs. 15, 33-34): ties the MSD path to the VAC path."""
    w = _systems()[1]
    h = oracle.from_workload(w)
    phi = _vec(h.n, 9, w.vacancies)
    m = 32
    c0 = oracle.vac_moments(h, phi, m, 1, 1.0)[0]
    errs = []
    for dt in [1e-3, 1e-4]:
        t_fs = dt * oracle.HBAR_EV_FS / G0
        cm = oracle.msd_moments(h, phi, m, 2, dt)[1] / t_fs ** 2
        errs.append(_rel(cm, c0))
    assert errs[1] < 2e-4 and errs[1] < errs[0] / 5


def test_green_kubo_equals_einstein_with_exact_trace():
    """Sec. 5.2: sigma^GK(E,t) = sigma^E1(E,t).  With the exact trace (all basis
    vectors) the identity d^2 DX^2/dt^2 = 2 C_vv holds up to time discretisation,
    so the trapezoid GK and the central-difference E1 agree to O(dt^2)."""
    w = ki.sheet_cells(3, 3, vacancy_conc=0.06, anderson_w_ev=1.5, lattice_seed=2)
    h = oracle.from_workload(w)
    m, nc, dt = 48, 24, 0.25
    cv = np.zeros((nc, m), dtype=complex)
    cx = np.zeros((nc, m), dtype=complex)
    for j in range(h.n):
        if w.vacancy_mask()[j]:
            continue
        e = np.zeros(h.n, dtype=complex)
        e[j] = 1.0
        cv += oracle.vac_moments(h, e, m, nc, dt)
        cx += oracle.msd_moments(h, e, m, nc, dt)
    en = np.linspace(-6, 6, 9)
    t = post.time_grid(nc, dt)
    gk = post.sigma_gk(post.kpm_density(cv, en, h.emax_ev, h.area_nm2), t)
    e1 = post.sigma_e1(post.kpm_density(cx, en, h.emax_ev, h.area_nm2), t)
    scale = np.max(np.abs(gk))
    assert np.max(np.abs(gk[2:-2] - e1[2:-2])) / scale < 0.02


def test_einstein_e2_is_half_of_e1_when_ballistic():
    """Sec. 5.1: in the ballistic regime DX^2 = v^2 t^2, so sigma^E2 = sigma^E1 / 2."""
    h = oracle.build_hamiltonian(ki.SHEET, 48, 24, emax_ev=8.505)
    phi = _vec(h.n, 10)
    m, nc, dt = 64, 6, 0.05
    c = oracle.msd_moments(h, phi, m, nc, dt)
    en = np.array([-1.0, 0.5, 2.0])
    t = post.time_grid(nc, dt)
    rho = post.kpm_density(c, en, h.emax_ev, h.area_nm2)
    e1 = post.sigma_e1(rho, t)
    e2 = post.sigma_e2(rho, t)
    assert np.allclose(e2[2:4] / e1[2:4], 0.5, rtol=0.03)


# ------------------------------------------------------------------ sums and damping

def test_jackson_closed_forms():
    """Eq. (35): g_0 = 1, g_1 = cos(pi/(M+1)), and g_M would vanish (1 - M a = a)."""
    for m in [2, 10, 512, 3000]:
        g = oracle.jackson(m)
        assert abs(g[0] - 1) < 1e-15
        assert abs(g[1] - np.cos(np.pi / (m + 1))) < 1e-14
        assert np.all(np.diff(g) < 0) and g[-1] > 0


def test_dos_integrates_to_state_count_and_is_positive():
    """Eq. (29): int rho dE = (2/Omega) mu_0 = 2 N_active / Omega for the exact trace;
    with Jackson damping the exact-trace DOS is non-negative."""
    w = ki.sheet_cells(4, 4, vacancy_conc=0.05, anderson_w_ev=1.0, lattice_seed=7)
    h = oracle.from_workload(w)
    m = 128
    mu = np.zeros(m, dtype=complex)
    for j in range(h.n):
        if w.vacancy_mask()[j]:
            continue                      # removed atoms are not part of the system
        e = np.zeros(h.n, dtype=complex)
        e[j] = 1.0
        mu += oracle.kpm_moments(h, e, e, m)
    th = (np.arange(4000) + 0.5) * np.pi / 4000
    en = np.cos(th) * h.emax_ev
    rho = post.kpm_density(mu, en, h.emax_ev, h.area_nm2)
    integral = np.sum(rho * np.sin(th)) * (np.pi / 4000) * h.emax_ev
    assert abs(integral / (2 * h.n_active / h.area_nm2) - 1) < 1e-12
    assert np.min(rho) > -1e-12 * np.max(rho)


def _bloch_levels(nx, ny, emax):
    """All N eigenvalues of a pristine periodic sheet from the Bloch bands, / E_max."""
    lx, ly = np.sqrt(3) * nx * A_NM / 2, 1.5 * ny * A_NM
    kx = 2 * np.pi * np.arange(nx)[:, None] / lx
    ky = 2 * np.pi * np.arange(ny)[None, :] / ly
    deltas = [(np.sqrt(3) * A_NM / 2, -A_NM / 2), (-np.sqrt(3) * A_NM / 2, -A_NM / 2),
              (0.0, A_NM)]
    f = sum(np.exp(1j * (kx * dx + ky * dy)) for dx, dy in deltas)
    e = G0 * np.abs(f).ravel() / emax
    return np.concatenate([e, -e])        # each level twice (see the spectrum test)


def _chebyshev_trace(eps, m):
    """sum_k T_n(eps_k) by the three-term recurrence, halved for the double count."""
    mu = np.zeros(m)
    t0, t1 = np.ones_like(eps), eps.copy()
    mu[0], mu[1] = t0.sum(), t1.sum()
    for n in range(2, m):
        t0, t1 = t1, 2 * eps * t1 - t0
        mu[n] = t1.sum()
    return 0.5 * mu


def test_dos_sum_reproduces_dirac_slope():
    """Eq. (29) applied to exact Bloch-band moments of a large pristine sheet gives the
    linear Dirac-cone DOS rho(E) = 2|E| / (pi (hbar v_F)^2), hbar v_F = 3 gamma0 a / 2
    (spin included; Castro Neto et al., the paper's graphene reference)."""
    nx = ny = 512
    emax = 8.505
    mu = _chebyshev_trace(_bloch_levels(nx, ny, emax), 300)
    area = (np.sqrt(3) * nx * A_NM / 2) * (1.5 * ny * A_NM)
    en = np.array([0.3, 0.4, 0.5])
    rho = post.kpm_density(mu, en, emax, area)
    exact = 2 * en / (np.pi * (1.5 * G0 * A_NM) ** 2)
    assert np.allclose(rho, exact, rtol=0.02)


def _graphene_dos_per_cell(x):
    """Closed-form DOS of the nearest-neighbour honeycomb per unit cell, spin included, in
    units of 1/gamma0 at x = E/gamma0 (Hobson and Nierenberg 1953; Castro Neto et al. 2009,
    the paper's graphene reference): a complete elliptic integral of the first kind."""
    x = np.abs(x)
    a = (1 + x) ** 2 - (x * x - 1) ** 2 / 4
    z0 = np.where(x <= 1, a, 4 * x)
    z1 = np.where(x <= 1, 4 * x, a)
    return 4 / np.pi ** 2 * x / np.sqrt(z0) * special.ellipk(np.minimum(z1 / z0, 1 - 1e-16))


def test_dos_matches_closed_form_over_the_band():
    """Eq. (29) with Jackson damping, applied to the exact Bloch-band moments of a
    512 x 512-site pristine sheet, reproduces the closed-form graphene DOS over the whole
    band (away from the Dirac point, the van Hove singularity at gamma0 and the band edge
    at 3 gamma0, where the M = 500 kernel broadening matters) and puts the van Hove peak at
    E = gamma0.  The closed form itself is checked first: 4 states per cell (2 atoms x 2
    spins) and the Dirac slope 4 |x| / (sqrt(3) pi)."""
    n = 2_000_000
    x = (np.arange(n) + 0.5) * 3.0 / n
    assert abs(2 * np.sum(_graphene_dos_per_cell(x)) * 3.0 / n - 4.0) < 1e-4
    assert abs(_graphene_dos_per_cell(np.array([1e-6]))[0] / 1e-6 - 4 / (np.sqrt(3) * np.pi)) < 1e-5
    nx = ny = 512
    emax = 1.05 * 3 * G0
    mu = _chebyshev_trace(_bloch_levels(nx, ny, emax), 500)
    area = (np.sqrt(3) * nx * A_NM / 2) * (1.5 * ny * A_NM)
    cell = 3 * np.sqrt(3) / 2 * A_NM ** 2
    en = np.concatenate([np.linspace(0.2, 2.2, 21), np.linspace(3.3, 7.5, 22), -np.linspace(0.4, 7.4, 8)])
    rho = post.kpm_density(mu, en, emax, area)
    exact = _graphene_dos_per_cell(en / G0) / G0 / cell
    assert np.max(np.abs(rho / exact - 1)) < 0.01, np.abs(rho / exact - 1)
    e_vh = np.linspace(2.0, 3.4, 1401)
    peak = e_vh[np.argmax(post.kpm_density(mu, e_vh, emax, area))]
    assert abs(peak - G0) < 0.02, peak


def test_random_vector_trace_is_unbiased():
    """Sec. 3.1.1: <phi|T_n(H~)|phi> estimates Tr T_n(H~) with an error of order
    sqrt(N) per vector (relative O(1/sqrt(N_r N))).  Checked against the exact
    Bloch-band trace of a 128 x 96 pristine sheet."""
    nx, ny, emax, m = 128, 96, 8.505, 120
    h = oracle.build_hamiltonian(ki.SHEET, nx, ny, emax_ev=emax)
    exact = _chebyshev_trace(_bloch_levels(nx, ny, emax), m)
    est = np.zeros(m)
    nr = 4
    for r in range(nr):
        phi = _vec(h.n, 30 + r)
        est += oracle.kpm_moments(h, phi, phi, m).real / nr
    assert abs(est[0] - h.n) < 1e-9 * h.n
    assert np.max(np.abs(est - exact)) < 6 * np.sqrt(h.n / nr)


# ------------------------------------------------------------------ planted mistakes

def _pin_errors():
    """A compact set of pins whose errors are returned (not asserted)."""
    w = _systems()[0]
    h = oracle.from_workload(w)
    ed = _ED(h)
    l = _vec(h.n, 1, w.vacancies)
    r = _vec(h.n, 2, w.vacancies) * (1 + 0.3j)
    errs = {}
    errs["kpm"] = _rel(oracle.kpm_moments(h, l, r, 64), ed.moments(l, r, 64))
    errs["evolve"] = _rel(oracle.evolve(h, l, 3.15, +1), ed.u(l, 3.15))
    errs["evolvex"] = _rel(oracle.evolvex(h, l, 3.15), ed.xu(l, 3.15))
    g = oracle.jackson(64)
    errs["jackson"] = abs(g[1] - np.cos(np.pi / 65))
    return errs


@pytest.mark.parametrize("mutation", [1, 2, 3, 4, 5])
def test_planted_mistakes_are_caught(mutation):
    clean = _pin_errors()
    assert max(clean.values()) < 1e-11
    with oracle.mutation(mutation):
        bad = _pin_errors()
    assert max(bad.values()) > 1e-6, bad


# ------------------------------------------------------------------ surrogate MLP oracle

def test_mlp_oracle_gradients_match_finite_differences():
    """Reverse-mode gradients of the FP64 MLP equal central finite differences of the
    loss (relative 1e-6) for sampled parameters of every layer."""
    from oracle import mlp
    hidden = 16                      # same code path, small enough for differences
    flat = mlp.init_params(3, hidden) + 0.01
    rng = np.random.default_rng(4)
    x = rng.normal(size=(37, 3))
    t = rng.normal(size=37)
    l0, g = mlp.gradients(flat, x, t, hidden)
    assert abs(l0 - mlp.loss(flat, x, t, hidden)) < 1e-14
    idx = np.concatenate([rng.choice(len(flat), 60, replace=False), [len(flat) - 1, 0]])
    h = 1e-6
    for k in idx:
        e = np.zeros_like(flat)
        e[k] = h
        fd = (mlp.loss(flat + e, x, t, hidden) - mlp.loss(flat - e, x, t, hidden)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(abs(fd), 1e-3), (k, fd, g[k])


def test_mlp_oracle_adam_closed_forms():
    """Adam with bias correction (Kingma and Ba, 2015): under a constant gradient g the
    corrected moments are exactly g and g^2 at every step, so each step moves a
    parameter by lr g / (|g| + eps); a gradient that flips sign after one step
    moves it back by less than lr in the second step."""
    from oracle import mlp
    rng = np.random.default_rng(2)
    flat = rng.normal(size=50)
    g = rng.normal(size=50)
    m = np.zeros(50)
    v = np.zeros(50)
    lr, eps = 1e-2, 1e-8
    x = flat.copy()
    for step in range(1, 6):
        x_new, m, v = mlp.adam_step(x, g, m, v, step, lr, eps=eps)
        assert np.allclose(x - x_new, lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)
        x = x_new
    x1, m1, v1 = mlp.adam_step(flat, g, np.zeros(50), np.zeros(50), 1, lr)
    x2, _, _ = mlp.adam_step(x1, -g, m1, v1, 2, lr)
    step2 = x2 - x1
    assert np.all(np.sign(step2) == np.sign(g)) and np.all(np.abs(step2) < lr)


def test_mlp_oracle_gelu_and_layout():
    """GELU closed forms (GELU(0) = 0, GELU(z) -> z for large z, GELU' = derivative, the tanh
    form within 5e-4 of z Phi(z))
    and the parameter count 3*256 + 256 + 3*(256^2 + 256) + 256 + 1."""
    from oracle import mlp
    from scipy.special import erf
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu(np.array([10.0]))[0] - 10.0) < 1e-12
    zz = np.linspace(-6, 6, 2001)
    exact = 0.5 * zz * (1.0 + erf(zz / np.sqrt(2.0)))        # z Phi(z), which the tanh form approximates
    assert np.max(np.abs(mlp.gelu(zz) - exact)) < 5e-4
    z = np.linspace(-4, 4, 41)
    fd = (mlp.gelu(z + 1e-6) - mlp.gelu(z - 1e-6)) / 2e-6
    assert np.max(np.abs(fd - mlp.gelu_grad(z))) < 1e-8
    assert mlp.n_params() == 3 * 256 + 256 + 3 * (256 * 256 + 256) + 256 + 1 == 198657



# ------------------------------------------------------------------ Fourier moments (FTM)

def test_ftm_moments_match_exact_diagonalisation():
    """Algorithm 4: F_n = <L|U(n dtau)|R> = sum_k conj(L_k) R_k exp(-i pi n e_k) for the
    scaled step dtau -> pi (Sec. 4.2), n = -N_m..N_m."""
    for w in _systems()[:3]:
        h = oracle.from_workload(w)
        ed = _ED(h)
        l = _vec(h.n, 1, w.vacancies)
        r = _vec(h.n, 2, w.vacancies) * (1 + 0.3j)
        f = oracle.ftm_moments(h, l, r, 12)
        a, b = ed.v.T @ l, ed.v.T @ r
        n = np.arange(-12, 13)
        ref = np.exp(-1j * np.pi * np.outer(n, ed.e)) @ (np.conj(a) * b)
        assert _rel(f, ref) < 1e-12


def test_ftm_dos_integrates_to_state_count():
    """Eq. (22) with the Hanning window (Eq. 28, w_0 = 1): int rho dE over
    [-E_max, E_max] = 2 F_0 / Omega, and FTM agrees with KPM on integrated windows
    (both are approximations of the same delta function, Sec. 4.2)."""
    w = ki.sheet_cells(12, 12, vacancy_conc=0.02, lattice_seed=3)
    h = oracle.from_workload(w)
    phi = _vec(h.n, 5, w.vacancies)
    f = oracle.ftm_moments(h, phi, phi, 60)
    en = np.linspace(-h.emax_ev, h.emax_ev, 4001)
    rho = post.ftm_density(f, en, h.emax_ev, h.area_nm2)
    integral = np.trapezoid(rho, en)
    assert abs(integral / (2 * f[60].real / h.area_nm2) - 1) < 1e-3
    mu = oracle.kpm_moments(h, phi, phi, 200)
    en2 = np.linspace(-8.0, 8.0, 1601)
    rk = post.kpm_density(mu, en2, h.emax_ev, h.area_nm2)
    rf = post.ftm_density(f, en2, h.emax_ev, h.area_nm2)
    for lo, hi in [(-8, -4), (-4, -1), (-1, 1), (1, 4), (4, 8)]:
        sel = (en2 >= lo) & (en2 <= hi)
        ik, iff = np.trapezoid(rk[sel], en2[sel]), np.trapezoid(rf[sel], en2[sel])
        assert abs(ik - iff) < 0.05 * max(abs(ik), 1e-3 * integral), (lo, hi, ik, iff)


# ------------------------------------------------------------------ ballistic, sigma_sc, Pade

def test_ballistic_conductance_forms_agree_when_msd_is_quadratic():
    """Sec. 5.1: with DX^2 = v^2 t^2, L = 2 v t (Eq. 50) and G = (W/L) sigma^E1 (Eq. 51)
    equals (W/2) e^2 rho sqrt(v^2) (Eq. 52), i.e. (W/2) h rho v in units of e^2/h."""
    t = post.time_grid(9, 1.0)
    rho = np.array([0.02, 0.05, 0.11])
    v = np.array([0.3, 0.6, 0.9])
    rdx = rho[None, :] * (v[None, :] * t[:, None]) ** 2
    length, g = post.ballistic(rho, rdx, t, 12.0)
    assert np.allclose(length[1:], 2 * v[None, :] * t[1:, None], rtol=1e-12)
    ref = 0.5 * 12.0 * post.H_EV_FS * rho * v
    assert np.allclose(g[1:-1], ref[None, :], rtol=1e-12)


def test_pade_fit_positive_kkt():
    """The bounded fit (b_k >= 0, true residual) returns an exact approximant with positive
    b unchanged; on noisy saturating data it follows the data to the noise level, and it
    satisfies the first-order (KKT) conditions of bounded least squares on the true
    residual: zero gradient J^T r in the free coefficients and a non-negative gradient for
    every b_k held at 0."""
    t = np.linspace(1.0, 200.0, 60)
    coef = np.array([0.5, 3.0, 0.02, 0.01, 2e-4])
    assert np.allclose(post.pade_value(post.pade_fit_positive(t, post.pade_value(coef, t)), t),
                       post.pade_value(coef, t), rtol=1e-9)
    rng = np.random.default_rng(7)
    tt = np.arange(190) * 20.0 + 200.0
    y = 400.0 * (1.0 - np.exp(-tt / 300.0)) + rng.normal(scale=5.0, size=190)
    c = post.pade_fit_positive(tt, y)
    assert np.all(c[3:] >= 0)
    r = post.pade_value(c, tt) - y
    assert np.sqrt(np.mean(r ** 2)) < 1.2 * 5.0
    den = 1.0 + c[3] * tt + c[4] * tt ** 2
    val = post.pade_value(c, tt)
    jac = np.stack([tt ** 0 / den, tt / den, tt ** 2 / den, -val * tt / den, -val * tt ** 2 / den], axis=1)
    grad = jac.T @ r
    scale = np.linalg.norm(jac, axis=0) * np.linalg.norm(r)
    for k in range(5):
        if k >= 3 and c[k] == 0.0:
            assert grad[k] >= -1e-6 * scale[k]
        else:
            assert abs(grad[k]) <= 1e-5 * scale[k], (k, grad[k], scale[k])


def test_sigma_sc_definitions():
    """Eq. (53) maximum and Eq. (54) block average: a plateau gives its value for both;
    a ramp sigma = c t averages to c (t1 + t2) / 2."""
    t = post.time_grid(21, 1.0)
    plateau = np.full((21, 3), 2.5)
    plateau[0] = 0.0
    assert np.allclose(post.sigma_sc_max(plateau), 2.5)
    assert np.allclose(post.sigma_sc_average(plateau, t, t[4], t[15]), 2.5)
    ramp = np.outer(t, [1.0, 2.0])
    assert np.allclose(post.sigma_sc_average(ramp, t, t[2], t[10]), np.array([1.0, 2.0]) * (t[2] + t[10]) / 2)


def test_pade_fit_recovers_a_rational_function():
    """Eq. (58) [2/2]: data drawn from a known approximant are fitted back exactly."""
    t = np.linspace(1.0, 200.0, 60)
    coef = np.array([0.5, 3.0, 0.02, 0.01, 2e-4])
    y = post.pade_value(coef, t)
    got = post.pade_fit(t, y)
    assert np.allclose(got, coef, rtol=1e-8)
