"""CPU oracle for the linear-scaling Kubo-Greenwood method (arXiv 1307.0288).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path never
imports this package.

The heavy loops (lattice, recursion, Bessel series, correlation-time loops) are
plain FP64 C in ``kg_oracle.c``, loaded with ctypes; the energy sums and the
conductivity formulas are plain numpy in ``post.py``.  Each function cites the
passage of the paper it follows.

Parity pins: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_pins.py`` (exact diagonalisation, closed forms, sum rules,
library routines, printed numbers of the paper).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HBAR_EV_FS = 0.6582119569  # reduced Planck constant, eV fs (CODATA 2018)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kg_oracle.c")
_LIB = os.path.join(_HERE, "libkgoracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``kg_oracle.c`` with gcc (no FMA contraction, so results are the
    same on x86-64 and aarch64 hosts)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", _LIB, _SRC, "-lm"])
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        D = ctypes.c_double
        I = ctypes.c_int
        L.ora_build_hamiltonian.restype = I64
        L.ora_build_hamiltonian.argtypes = [I, I64, I64, D, D, D, P, P, P, P, P, P, P]
        hargs = [I64, P, P, P, P, P]
        L.ora_apply_h.argtypes = hargs + [P, P]
        L.ora_apply_xh.argtypes = hargs + [P, P]
        L.ora_apply_v.argtypes = hargs + [D, D, P, P]
        L.ora_dot.argtypes = [I64, P, P, P]
        L.ora_kpm_moments.argtypes = hargs + [P, P, I, P]
        L.ora_bessel_j.argtypes = [D, I, P]
        L.ora_bessel_terms.restype = I
        L.ora_bessel_terms.argtypes = [D, D]
        L.ora_evolve.argtypes = hargs + [P, I, I, P, P]
        L.ora_evolvex.argtypes = hargs + [P, I, P, P]
        L.ora_vac.argtypes = hargs + [D, D, P, I, I, P, I, P]
        L.ora_msd.argtypes = hargs + [P, I, I, P, I, P]
        L.ora_jackson.argtypes = [I, P]
        L.ora_kpm_sum.argtypes = [I, P, P, I, P, P]
        L.ora_ftm_moments.argtypes = hargs + [P, P, I, P, I, P]
        L.ora_set_mutation.argtypes = [I]
        L.ora_get_mutation.restype = I
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _cvec(v) -> np.ndarray:
    return np.ascontiguousarray(v, dtype=np.complex128)


@dataclass
class Hamiltonian:
    """Scaled Hamiltonian H~ = H / E_max in CSR form (Sec. 2, Eq. 13)."""
    kind: int
    nx: int
    ny: int
    bond_nm: float
    gamma0_ev: float
    emax_ev: float
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    disp: np.ndarray
    diag: np.ndarray
    vacancy_mask: np.ndarray

    @property
    def n(self) -> int:
        return self.nx * self.ny

    @property
    def n_active(self) -> int:
        return int(self.n - self.vacancy_mask.sum())

    @property
    def area_nm2(self) -> float:
        """Omega = L_x L_y = (sqrt(3) N_x a / 2)(3 N_y a / 2) (Sec. 2)."""
        return (np.sqrt(3.0) * self.nx * self.bond_nm / 2.0) * (1.5 * self.ny * self.bond_nm)

    def _hargs(self):
        return (self.n, _p(self.row_ptr), _p(self.col), _p(self.val), _p(self.disp),
                _p(self.diag))

    def dense(self) -> np.ndarray:
        """Dense H~ (for exact diagonalisation in tests)."""
        h = np.zeros((self.n, self.n))
        for r in range(self.n):
            for k in range(self.row_ptr[r], self.row_ptr[r + 1]):
                h[r, self.col[k]] += self.val[k]
        h[np.arange(self.n), np.arange(self.n)] += self.diag
        return h

    def dense_xh(self) -> np.ndarray:
        """Dense [X, H~] with elements (X_n - X_m) H~_nm (Eq. 15)."""
        d = np.zeros((self.n, self.n))
        for r in range(self.n):
            for k in range(self.row_ptr[r], self.row_ptr[r + 1]):
                d[r, self.col[k]] += self.disp[k] * self.val[k]
        return d


def build_hamiltonian(kind: int, nx: int, ny: int, *, emax_ev: float,
                      vacancies=None, onsite_ev=None, bond_nm: float = 0.142,
                      gamma0_ev: float = 2.7) -> Hamiltonian:
    n = nx * ny
    vac = np.zeros(n, dtype=np.uint8)
    if vacancies is not None and len(vacancies):
        vac[np.asarray(vacancies, dtype=np.int64)] = 1
    on = None if onsite_ev is None else np.ascontiguousarray(onsite_ev, dtype=np.float64)
    rp = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(3 * n, dtype=np.int64)
    val = np.zeros(3 * n)
    disp = np.zeros(3 * n)
    diag = np.zeros(n)
    nnz = lib().ora_build_hamiltonian(kind, nx, ny, bond_nm, gamma0_ev, emax_ev, _p(vac),
                                      None if on is None else _p(on), _p(rp), _p(col),
                                      _p(val), _p(disp), _p(diag))
    return Hamiltonian(kind, nx, ny, bond_nm, gamma0_ev, emax_ev, rp, col[:nnz].copy(),
                       val[:nnz].copy(), disp[:nnz].copy(), diag, vac)


def from_workload(w) -> Hamiltonian:
    """Hamiltonian of a ``kg_inputs.Workload``."""
    return build_hamiltonian(w.kind, w.nx, w.ny, emax_ev=w.emax_ev, vacancies=w.vacancies,
                             onsite_ev=w.onsite, bond_nm=w.bond_nm, gamma0_ev=w.gamma0_ev)


def apply_h(h: Hamiltonian, x) -> np.ndarray:
    x = _cvec(x); y = np.empty_like(x)
    lib().ora_apply_h(*h._hargs(), _p(x), _p(y)); return y


def apply_xh(h: Hamiltonian, x) -> np.ndarray:
    x = _cvec(x); y = np.empty_like(x)
    lib().ora_apply_xh(*h._hargs(), _p(x), _p(y)); return y


def apply_v(h: Hamiltonian, x, hbar: float = HBAR_EV_FS) -> np.ndarray:
    """V x with V = (i/hbar)[H, X] (Eq. 15), in nm/fs."""
    x = _cvec(x); y = np.empty_like(x)
    lib().ora_apply_v(*h._hargs(), h.emax_ev, hbar, _p(x), _p(y)); return y


def dot(l, v) -> complex:
    l = _cvec(l); v = _cvec(v); out = np.zeros(2)
    lib().ora_dot(len(l), _p(l), _p(v), _p(out)); return complex(out[0], out[1])


def kpm_moments(h: Hamiltonian, phi_l, phi_r, n_moments: int) -> np.ndarray:
    """C_n = <phi_L|T_n(H~)|phi_R>, n < M (Algorithm 5).  Complex [M]."""
    l = _cvec(phi_l); r = _cvec(phi_r); c = np.zeros(2 * n_moments)
    lib().ora_kpm_moments(*h._hargs(), _p(l), _p(r), n_moments, _p(c))
    return c[0::2] + 1j * c[1::2]


def bessel_j(x: float, nmax: int) -> np.ndarray:
    """J_m(x), m = 0..nmax (Miller backward recurrence)."""
    out = np.zeros(nmax + 1)
    lib().ora_bessel_j(float(x), nmax, _p(out)); return out


def bessel_terms(x: float, tol: float = 1e-15) -> int:
    """N_p: number of terms kept in Eqs. (36)-(37)."""
    return int(lib().ora_bessel_terms(float(x), float(tol)))


def tau_of(h: Hamiltonian, dt_hbar_over_gamma0: float) -> float:
    """Scaled Bessel argument tau = E_max dt / hbar for dt in units of hbar/gamma0
    (Sec. 3.1.3: scaling H by 1/E_max scales time by E_max)."""
    return h.emax_ev * dt_hbar_over_gamma0 / h.gamma0_ev


def bessel_series(tau: float, tol: float = 1e-15):
    np_ = bessel_terms(tau, tol)
    return bessel_j(tau, np_ - 1 if np_ > 0 else 0), np_


def evolve(h: Hamiltonian, x, tau: float, direction: int = +1, tol: float = 1e-15) -> np.ndarray:
    """U(+-dt) x (Eq. 36, Algorithm 6)."""
    jm, np_ = bessel_series(tau, tol)
    x = _cvec(x); y = np.empty_like(x)
    lib().ora_evolve(*h._hargs(), _p(jm), np_, direction, _p(x), _p(y)); return y


def evolvex(h: Hamiltonian, x, tau: float, tol: float = 1e-15) -> np.ndarray:
    """[X, U(dt)] x (Eq. 37, Algorithm 7)."""
    jm, np_ = bessel_series(tau, tol)
    x = _cvec(x); y = np.empty_like(x)
    lib().ora_evolvex(*h._hargs(), _p(jm), np_, _p(x), _p(y)); return y


def vac_moments(h: Hamiltonian, phi, n_moments: int, n_times: int,
                dt_hbar_over_gamma0: float, tol: float = 1e-15,
                hbar: float = HBAR_EV_FS) -> np.ndarray:
    """C_n^VAC(t_m), complex [N_c][M] (Algorithm 2, Eq. 33)."""
    jm, np_ = bessel_series(tau_of(h, dt_hbar_over_gamma0), tol)
    phi = _cvec(phi); c = np.zeros(2 * n_moments * n_times)
    lib().ora_vac(*h._hargs(), h.emax_ev, hbar, _p(phi), n_moments, n_times, _p(jm), np_,
                  _p(c))
    c = c.reshape(n_times, n_moments, 2)
    return c[..., 0] + 1j * c[..., 1]


def msd_moments(h: Hamiltonian, phi, n_moments: int, n_times: int,
                dt_hbar_over_gamma0: float, tol: float = 1e-15) -> np.ndarray:
    """C_n^MSD(t_m), complex [N_c][M] (Algorithm 3, Eq. 34)."""
    jm, np_ = bessel_series(tau_of(h, dt_hbar_over_gamma0), tol)
    phi = _cvec(phi); c = np.zeros(2 * n_moments * n_times)
    lib().ora_msd(*h._hargs(), _p(phi), n_moments, n_times, _p(jm), np_, _p(c))
    c = c.reshape(n_times, n_moments, 2)
    return c[..., 0] + 1j * c[..., 1]


def ftm_moments(h: Hamiltonian, phi_l, phi_r, n_m: int, tol: float = 1e-15) -> np.ndarray:
    """Fourier moments F_n = <phi_L|U(n dtau)|phi_R>, n = -N_m..N_m, dtau = pi hbar for H~
    (Algorithm 4, Sec. 4.2).  Complex [2 N_m + 1], index n + N_m."""
    jm, np_ = bessel_series(np.pi, tol)
    l = _cvec(phi_l); r = _cvec(phi_r); f = np.zeros(2 * (2 * n_m + 1))
    lib().ora_ftm_moments(*h._hargs(), _p(l), _p(r), n_m, _p(jm), np_, _p(f))
    return f[0::2] + 1j * f[1::2]


def jackson(n_moments: int) -> np.ndarray:
    """Jackson damping factors g_n (Eq. 35)."""
    g = np.zeros(n_moments)
    lib().ora_jackson(n_moments, _p(g)); return g


def kpm_sum(mu, e_scaled, g=None) -> np.ndarray:
    """2/(pi sqrt(1-e^2)) sum_n g_n (2 - delta_n0) T_n(e) Re mu_n (Eqs. 29-31, no 1/Omega)."""
    mu = np.ascontiguousarray(np.real(mu), dtype=np.float64)
    e = np.ascontiguousarray(e_scaled, dtype=np.float64)
    if g is None:
        g = jackson(len(mu))
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros(len(e))
    lib().ora_kpm_sum(len(mu), _p(mu), _p(g), len(e), _p(e), _p(out)); return out


class mutation:
    """Context manager that plants one deliberate mistake in the oracle (tests only).

    1: the T_{n-2} term is dropped from the moment recursion (Algorithm 5).
    2: the (2 - delta_m0) factor of the m = 1 Bessel term is lost (Eq. 36).
    3: the commutator [X, H] is transposed (sign of X_n - X_m flipped, Eq. 15).
    4: the Jackson parameter is a = 1/M instead of 1/(M + 1) (Eq. 35).
    5: the inner product conjugates the right operand instead of the left (Eq. 46).
    """

    def __init__(self, m: int):
        self.m = m

    def __enter__(self):
        lib().ora_set_mutation(self.m)

    def __exit__(self, *a):
        lib().ora_set_mutation(0)
