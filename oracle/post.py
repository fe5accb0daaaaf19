"""Oracle post-processing: energy sums and running conductivities (plain numpy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Units: energies in eV, lengths in nm, times in fs, hbar in eV fs, densities of
states per eV per nm^2 (spin included), conductivities in units of e^2/h.
"""
from __future__ import annotations

import numpy as np

from . import HBAR_EV_FS, jackson, kpm_sum

H_EV_FS = 2.0 * np.pi * HBAR_EV_FS  # Planck constant h, eV fs


def energy_grid(gamma0_ev: float = 2.7, n_e: int = 201) -> np.ndarray:
    """Reading: n_e energies uniform in [-3 gamma0, 3 gamma0] eV, ends included."""
    return np.linspace(-3.0 * gamma0_ev, 3.0 * gamma0_ev, n_e)


def kpm_density(mu, energies_ev, emax_ev: float, area_nm2: float) -> np.ndarray:
    """Eqs. (29)-(31): 2/(pi Omega sqrt(1-E~^2)) sum_n g_n (2-delta_n0) T_n(E~) Re mu_n,
    with E~ = E / E_max, converted to per-eV by the Jacobian 1/E_max.

    ``mu`` is [..., M] (moments averaged over random vectors); returns [..., n_E].
    """
    mu = np.asarray(mu)
    lead = mu.shape[:-1]
    m = mu.shape[-1]
    g = jackson(m)
    e = np.asarray(energies_ev) / emax_ev
    flat = np.real(mu).reshape(-1, m)
    out = np.stack([kpm_sum(row, e, g) for row in flat])
    return (out / (area_nm2 * emax_ev)).reshape(*lead, len(e))


def time_grid(n_times: int, dt_hbar_over_gamma0: float, gamma0_ev: float = 2.7) -> np.ndarray:
    """t_m = m dt in fs, dt given in units of hbar / gamma0."""
    return np.arange(n_times) * dt_hbar_over_gamma0 * HBAR_EV_FS / gamma0_ev


def sigma_gk(rho_cvv: np.ndarray, t_fs: np.ndarray) -> np.ndarray:
    """Green-Kubo running conductivity, Eq. (6): sigma = e^2 int_0^t rho C_vv dt'.

    ``rho_cvv`` is [N_c, n_E] in nm^2 fs^-2 / (eV nm^2).  Reading: trapezoid rule on
    the t_m grid.  Returns [N_c, n_E] in e^2/h.
    """
    out = np.zeros_like(rho_cvv)
    for m in range(1, len(t_fs)):
        out[m] = out[m - 1] + 0.5 * (t_fs[m] - t_fs[m - 1]) * (rho_cvv[m] + rho_cvv[m - 1])
    return H_EV_FS * out


def sigma_e1(rho_dx2: np.ndarray, t_fs: np.ndarray) -> np.ndarray:
    """Einstein running conductivity, Eq. (9): sigma = e^2 d(rho DX^2)/(2 dt).

    Reading: central differences inside, one-sided differences at both ends."""
    d = np.gradient(rho_dx2, t_fs, axis=0, edge_order=1)
    return H_EV_FS * 0.5 * d


def sigma_e2(rho_dx2: np.ndarray, t_fs: np.ndarray) -> np.ndarray:
    """Division-based Einstein conductivity, Eq. (11): e^2 rho DX^2 / (2 t); 0 at t = 0."""
    out = np.zeros_like(rho_dx2)
    t = np.asarray(t_fs)
    nz = t > 0
    out[nz] = rho_dx2[nz] / (2.0 * t[nz, None])
    return H_EV_FS * out


def hanning(n_m: int) -> np.ndarray:
    """Hanning window w_n = (1 + cos(pi n / (N_m + 1))) / 2, n = -N_m..N_m (Eq. 28)."""
    n = np.arange(-n_m, n_m + 1)
    return 0.5 * (1.0 + np.cos(np.pi * n / (n_m + 1)))


def ftm_density(f, energies_ev, emax_ev: float, area_nm2: float) -> np.ndarray:
    """Eq. (22): rho(E) = dtau / (pi hbar Omega) sum_n w_n exp(i E n dtau / hbar) F_n.
    With H~ = H / E_max the step is dtau = pi hbar / E_max (scaled step pi), so
    rho(E) = 1 / (E_max Omega) sum_n w_n exp(i pi n E / E_max) F_n; real part returned."""
    f = np.asarray(f)
    n_m = (f.shape[-1] - 1) // 2
    n = np.arange(-n_m, n_m + 1)
    w = hanning(n_m)
    e = np.asarray(energies_ev) / emax_ev
    phase = np.exp(1j * np.pi * np.outer(e, n))
    return np.real(phase @ (w * f).T).T / (emax_ev * area_nm2)


def ballistic(rho, rho_dx2, t_fs, width_nm: float):
    """Eqs. (50)-(51): DX^2 = rho DX^2 / rho, L = 2 sqrt(DX^2), G = (W / L) sigma^E1."""
    dx2 = np.where(np.asarray(rho)[None, :] > 0, rho_dx2 / np.asarray(rho)[None, :], 0.0)
    length = 2.0 * np.sqrt(np.maximum(dx2, 0.0))
    s1 = sigma_e1(rho_dx2, t_fs)
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.where(length > 0, width_nm / length * s1, 0.0)
    return length, g


def sigma_sc_max(sigma):
    """Eq. (53): maximum over the correlation times t > 0."""
    return np.max(np.asarray(sigma)[1:], axis=0)


def sigma_sc_average(sigma, t_fs, t1: float, t2: float):
    """Eq. (54): (1/(t2 - t1)) int_{t1}^{t2} sigma dt, trapezoid on the grid points in [t1, t2]."""
    t = np.asarray(t_fs)
    sel = (t >= t1 - 1e-9) & (t <= t2 + 1e-9)
    return np.trapezoid(np.asarray(sigma)[sel], t[sel], axis=0) / (t[sel][-1] - t[sel][0])


def pade_fit(t, y, m: int = 2, n: int = 2):
    """Eq. (58) with the denominator sum from k = 1: least squares (numpy.linalg.lstsq) on
    sum_j a_j t^j - y sum_k b_k t^k = y."""
    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    cols = [t ** j for j in range(m + 1)] + [-y * t ** k for k in range(1, n + 1)]
    a = np.stack(cols, axis=1)
    s = np.linalg.norm(a, axis=0)
    x = np.linalg.lstsq(a / s, y, rcond=None)[0]
    return x / s


def pade_fit_positive(t, y, m: int = 2, n: int = 2, passes: int = 100):
    """The fit of pade_fit with every b_k >= 0 (no pole for t >= 0) on the true residual
    sum (R(t_i) - y_i)^2.  Starting points: Sanathanan-Koerner reweighting of the bounded
    linearised problem (scipy.optimize.lsq_linear; rows divided by the previous pass's
    denominator until the weights settle) from the weight profiles (1 + |t| / s)^-n,
    s = inf, t_max, t_max/10, t_max/100; each refined by bounded nonlinear least squares
    (scipy.optimize.least_squares); the smallest residual is returned."""
    from scipy.optimize import least_squares, lsq_linear
    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    cols = [t ** j for j in range(m + 1)] + [-y * t ** k for k in range(1, n + 1)]
    a = np.stack(cols, axis=1)
    lb = np.concatenate([np.full(m + 1, -np.inf), np.zeros(n)])
    ub = np.full(m + 1 + n, np.inf)
    t_max = np.max(np.abs(t))
    best, best_r = None, np.inf
    for s_start in [np.inf, t_max, t_max / 10, t_max / 100]:
        w = (1.0 + np.abs(t) / s_start) ** (-n)
        x = None
        for _ in range(passes):
            aw = a * w[:, None]
            s = np.linalg.norm(aw, axis=0)
            x = lsq_linear(aw / s, y * w, bounds=(lb * s, ub), method="bvls", tol=1e-15).x / s
            den = 1.0 + sum(x[m + k] * t ** k for k in range(1, n + 1))
            w_new = 1.0 / den
            done = np.max(np.abs(w_new - w) / w) < 1e-12
            w = w_new
            if done:
                break
        x = np.maximum(x, lb)
        fit = least_squares(lambda c: pade_value(c, t, m, n) - y, x, bounds=(lb, ub), x_scale="jac",
                            method="trf", ftol=1e-15, xtol=1e-15, gtol=1e-15, max_nfev=5000)
        r = np.sum(fit.fun ** 2)
        if r < best_r:
            best, best_r = fit.x, r
    return best


def pade_value(coef, t, m: int = 2, n: int = 2):
    t = np.asarray(t, dtype=np.float64)
    num = sum(coef[j] * t ** j for j in range(m + 1))
    den = 1.0 + sum(coef[m + k] * t ** k for k in range(1, n + 1))
    return num / den
