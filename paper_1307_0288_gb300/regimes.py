"""The three transport regimes of Sec. 5, computed with the library.

* Ballistic (Sec. 5.1, Eq. 50): the length L(E, t) = 2 sqrt(DX^2(E, t)) of pristine
  graphene with periodic boundaries grows as sqrt(2) v_F t near the Dirac point (the
  in-plane average of v_x^2 is v_F^2 / 2), whatever the sample length.
* Diffusive (Sec. 5.2, Eqs. 53-54): the semi-classical conductivity of a sheet with
  vacancies, by the maximum over correlation times and by a block average, against the
  minimum conductivity 4 e^2 / (pi h) the paper finds for |E| < 0.25 eV at n = 1 %.
* Localized (Sec. 5.3, Eqs. 58-59): long-time MSD of an armchair ribbon, a Pade [2/2] fit
  of its late part, sigma^E1 from the fit and sigma^E2 from the raw MSD, and the
  length-dependent conductance G = (W / L) sigma with its exponential decay length.

Every number comes from the C ABI (moments on the GPU, sums on the host); this module
only chooses workloads and combines the library's outputs.
"""
from __future__ import annotations

import json
import time

import numpy as np

import kg_inputs as ki

from . import (HBAR_EV_FS, KG_FP64, KG_SIGMA_E1, KG_SIGMA_E2, KG_SIGMA_GK, conductivity,
               dos_moments, from_workload, kpm_sum, msd, pade_eval, pade_fit, sigma_sc, vac)

H_EV_FS = 2.0 * np.pi * HBAR_EV_FS   # Planck constant in eV fs: conductivities in e^2/h


def fermi_velocity(gamma0_ev: float = 2.7, bond_nm: float = 0.142) -> float:
    """v_F = 3 gamma0 a / (2 hbar) in nm/fs."""
    return 3.0 * gamma0_ev * bond_nm / (2.0 * HBAR_EV_FS)


def _blocks(n_vec: int, block: int):
    if block & (block - 1) or n_vec % block:
        raise ValueError("block must be a power of two dividing n_vec")
    return [(b, b + block) for b in range(0, n_vec, block)]


def einstein_curves(w, n_vec: int, n_moments: int, n_times: int, dt: float, energies_ev, *,
                    block: int = 16, precision: int = KG_FP64, per_vector: bool = False):
    """rho(E), rho DX^2(E, t_m) and the Einstein conductivities (Eqs. 9, 11) averaged over
    n_vec random vectors, run in blocks of ``block`` vectors.  dt in hbar/gamma0.  With
    per_vector, also each vector's DOS and MSD moments (keys mu_dos_r, mu_msd_r)."""
    h = from_workload(w)
    phi = w.vectors(n_vec)
    mu_dos = np.zeros(n_moments)
    mu_msd = np.zeros((n_times, n_moments))
    keep_dos, keep_msd = [], []
    t0 = time.perf_counter()
    for b0, b1 in _blocks(n_vec, block):
        ph = np.ascontiguousarray(phi[:, b0:b1])
        d = dos_moments(h, ph, n_moments, precision=precision).real
        m = msd(h, ph, n_moments, n_times, dt, precision=precision).real
        mu_dos += d.sum(axis=0)
        mu_msd += m.sum(axis=0)
        if per_vector:
            keep_dos.append(d)
            keep_msd.append(m)
    seconds = time.perf_counter() - t0
    rho = kpm_sum(mu_dos / n_vec, energies_ev, h.emax_ev, h.area_nm2)
    rdx = kpm_sum(mu_msd / n_vec, energies_ev, h.emax_ev, h.area_nm2)
    t_fs = np.arange(n_times) * dt * HBAR_EV_FS / w.gamma0_ev
    out = {"t_fs": t_fs, "energies": np.asarray(energies_ev), "rho": rho, "rho_dx2": rdx,
           "sigma_e1": conductivity(KG_SIGMA_E1, rdx, t_fs[1]),
           "sigma_e2": conductivity(KG_SIGMA_E2, rdx, t_fs[1]),
           "emax_ev": h.emax_ev, "area_nm2": h.area_nm2, "gpu_seconds": seconds}
    if per_vector:
        out["mu_dos_r"] = np.concatenate(keep_dos, axis=0)
        out["mu_msd_r"] = np.concatenate(keep_msd, axis=0)
    return out


def jackknife_sigma_sc(c, t_block, plateau):
    """Leave-one-vector-out (jackknife) estimates of the plateau means of sigma_sc by
    maximum and by block average, from the per-vector moments of einstein_curves:
    the stochastic trace (Sec. 3.1.1) averages independent random vectors, so the
    spread of the leave-one-out estimates measures the statistical error of the
    n-vector result.  Returns (mean_max, se_max, mean_avg, se_avg, n)."""
    d, m = c["mu_dos_r"], c["mu_msd_r"]
    n = d.shape[0]
    sd, sm = d.sum(axis=0), m.sum(axis=0)
    t = c["t_fs"]
    est_max, est_avg = [], []
    for i in range(n):
        rdx = kpm_sum((sm - m[i]) / (n - 1), c["energies"], c["emax_ev"], c["area_nm2"])
        s_max, s_avg = sigma_sc(conductivity(KG_SIGMA_E1, rdx, t[1]), t[1], *t_block)
        est_max.append(s_max[plateau].mean())
        est_avg.append(s_avg[plateau].mean())
    est_max, est_avg = np.array(est_max), np.array(est_avg)

    def se(v):
        return float(np.sqrt((n - 1) / n * np.sum((v - v.mean()) ** 2)))

    return float(est_max.mean()), se(est_max), float(est_avg.mean()), se(est_avg), n


def green_kubo_curves(w, n_vec: int, n_moments: int, n_times: int, dt: float, energies_ev, *,
                      block: int = 16, precision: int = KG_FP64):
    """rho C_vv(E, t_m) and sigma^GK (Eq. 6) averaged over n_vec random vectors."""
    h = from_workload(w)
    phi = w.vectors(n_vec)
    mu = np.zeros((n_times, n_moments))
    t0 = time.perf_counter()
    for b0, b1 in _blocks(n_vec, block):
        ph = np.ascontiguousarray(phi[:, b0:b1])
        mu += vac(h, ph, n_moments, n_times, dt, precision=precision).real.sum(axis=0)
    seconds = time.perf_counter() - t0
    rcvv = kpm_sum(mu / n_vec, energies_ev, h.emax_ev, h.area_nm2)
    t_fs = np.arange(n_times) * dt * HBAR_EV_FS / w.gamma0_ev
    return {"t_fs": t_fs, "rho_cvv": rcvv, "sigma_gk": conductivity(KG_SIGMA_GK, rcvv, t_fs[1]),
            "gpu_seconds": seconds}


def window_length(curves, e_lo: float, e_hi: float):
    """L(t) = 2 sqrt(DX^2) over the energies with e_lo <= |E| <= e_hi: the ratio of the
    summed rho DX^2 to the summed rho (a DOS-weighted average of DX^2)."""
    e = np.abs(curves["energies"])
    sel = (e >= e_lo) & (e <= e_hi)
    dx2 = curves["rho_dx2"][:, sel].sum(axis=1) / curves["rho"][sel].sum()
    return 2.0 * np.sqrt(np.maximum(dx2, 0.0))


# ------------------------------------------------------------------ ballistic

def run_ballistic(cells=((512, 512), (1024, 512)), n_vec: int = 4, n_moments: int = 2000,
                  n_times: int = 21, dt: float = 10.0, window=(0.2, 0.5), open_cells=None,
                  open_times: int = 61, open_dt: float = 41.0):
    """Pristine sheets along the zigzag transport direction.  Periodic samples (default
    1024 x 1024 and 2048 x 1024 sites: 126 nm and 252 nm): L(t) over the energy window,
    its ratio to sqrt(2) v_F t, and the difference between the two lengths.  Samples open
    along x (open_cells, e.g. (512, 512): 126 nm), the non-periodic boundary of Sec. 5.1, run
    for open_times steps of open_dt: L(t) grows ballistically and then stays below the sample
    length (classical free flight between the two ends, with uniformly spread starting points
    and an isotropic velocity, peaks near 0.93 L_x at t = L_x / v_F and settles at
    2 L_x / sqrt(6) = 0.82 L_x).  dt in hbar/gamma0 (41 = 10 fs at gamma0 = 2.7 eV)."""
    en = np.linspace(-1.0, 1.0, 201)
    v_f = fermi_velocity()
    out = {"v_f_nm_per_fs": v_f, "window_ev": list(window), "samples": []}
    lengths = []
    runs = [(ki.SHEET, cx, cy, n_times, dt) for cx, cy in cells]
    if open_cells is not None:
        runs.append((ki.SHEET_OPEN_X, open_cells[0], open_cells[1], open_times, open_dt))
    for kind, cx, cy, nt, step in runs:
        w = ki.Workload(kind, 2 * cx, 2 * cy, n_vec=n_vec)
        c = einstein_curves(w, n_vec, n_moments, nt, step, en, block=n_vec)
        length = window_length(c, *window)
        t = c["t_fs"]
        ratio = length[1:] / (np.sqrt(2.0) * v_f * t[1:])
        lx = w.nx * np.sqrt(3) / 2 * w.bond_nm
        entry = {"boundary_x": "periodic" if kind == ki.SHEET else "open", "sites": w.n_sites,
                 "sample_length_nm": lx, "t_fs": t.tolist(), "L_nm": length.tolist(),
                 "ratio_to_sqrt2_vF_t": ratio.tolist(), "gpu_seconds": c["gpu_seconds"]}
        if kind == ki.SHEET:
            lengths.append(length)
        else:
            entry["L_over_sample_length"] = (length / lx).tolist()
        out["samples"].append(entry)
    if len(lengths) == 2:
        out["max_rel_diff_between_lengths"] = float(np.max(np.abs(lengths[0][1:] - lengths[1][1:])
                                                           / lengths[1][1:]))
    return out


# ------------------------------------------------------------------ diffusive

def run_diffusive(cells=(1024, 512), conc: float = 0.01, n_vec: int = 32, n_moments: int = 3000,
                  n_times: int = 101, dt: float = 0.82, t_block=(10.0, 20.0), gk_vectors: int = 8,
                  gk_times: int = 51, block: int = 16):
    """Sheet of 2048 x 1024 sites with n = 1 % vacancies: sigma^E1(E, t) over 32 random
    vectors up to t = (n_times - 1) dt, the semi-classical conductivity by maximum (Eq. 53)
    and by block average over t_block (Eq. 54), their means over 0.1 <= |E| <= 0.25 eV
    against 4 / pi, and sigma^GK from the VAC on the first gk_vectors vectors against
    sigma^E1 on the same vectors (Green-Kubo = Einstein, Sec. 5.2)."""
    en = np.round(np.linspace(-1.0, 1.0, 81), 10)
    w = ki.sheet_cells(*cells, vacancy_conc=conc, n_vec=n_vec)
    c = einstein_curves(w, n_vec, n_moments, n_times, dt, en, block=block, per_vector=True)
    t = c["t_fs"]
    s_max, s_avg = sigma_sc(c["sigma_e1"], t[1], *t_block)
    plateau = (np.abs(en) >= 0.1 - 1e-9) & (np.abs(en) <= 0.25 + 1e-9)
    jm, jse_max, ja, jse_avg, nj = jackknife_sigma_sc(c, t_block, plateau)
    pm, pa = float(s_max[plateau].mean()), float(s_avg[plateau].mean())
    out = {"sites": w.n_sites, "vacancies": len(w.vacancies), "vectors": n_vec, "moments": n_moments,
           "dt_fs": float(t[1]), "t_max_fs": float(t[-1]), "t_block_fs": list(t_block),
           "energies_ev": en.tolist(), "sigma_sc_max": s_max.tolist(), "sigma_sc_average": s_avg.tolist(),
           "plateau_mean_max": pm, "plateau_mean_average": pa,
           # jackknife over the n vectors: standard error of the n-vector plateau means, and the
           # bias estimate (n - 1)(mean of leave-one-out - full) of each estimator
           "plateau_se_max": jse_max, "plateau_se_average": jse_avg,
           "plateau_jackknife_bias_max": (nj - 1) * (jm - pm),
           "plateau_jackknife_bias_average": (nj - 1) * (ja - pa),
           "plateau_max_minus_4_over_pi_in_se": (pm - 4.0 / np.pi) / jse_max if jse_max > 0 else None,
           "plateau_average_minus_4_over_pi_in_se": (pa - 4.0 / np.pi) / jse_avg if jse_avg > 0 else None,
           "sigma_min_4_over_pi": 4.0 / np.pi, "gpu_seconds_einstein": c["gpu_seconds"]}
    if gk_vectors:
        wg = ki.sheet_cells(*cells, vacancy_conc=conc, n_vec=gk_vectors)
        g = green_kubo_curves(wg, gk_vectors, n_moments, gk_times, dt, en, block=min(block, gk_vectors))
        e1 = einstein_curves(wg, gk_vectors, n_moments, gk_times, dt, en, block=min(block, gk_vectors))
        sel = np.abs(en) >= 0.3
        diff = np.abs(g["sigma_gk"][1:, sel] - e1["sigma_e1"][1:, sel])
        out["gk_vs_e1"] = {"vectors": gk_vectors, "times": gk_times,
                           "max_abs_diff_e2h_abs_E_ge_0.3": float(diff.max()),
                           "max_sigma": float(np.abs(e1["sigma_e1"][1:, sel]).max()),
                           "gk_mean_abs_E_ge_0.3": g["sigma_gk"][:, sel].mean(axis=1).tolist(),
                           "e1_mean_abs_E_ge_0.3": e1["sigma_e1"][:, sel].mean(axis=1).tolist(),
                           "gpu_seconds_vac": g["gpu_seconds"]}
    return out


# ------------------------------------------------------------------ localized

def fit_msd(t, dx2, t_from: float, m: int = 2, n: int = 2):
    """Pade [m/n] fit (Eq. 58) of DX^2(t) over t >= t_from with every denominator
    coefficient b_k >= 0 (kg_pade_fit_positive): the free linearised fit can put a pole
    among flat, noisy late-time data, the bounded one has none for t >= 0."""
    sel = t >= t_from
    return pade_fit(t[sel], dx2[sel], m, n, positive=True)


def run_localized(nx: int = 95, ny: int = 32768, conc: float = 0.01, n_vec: int = 4,
                  n_moments: int = 3000, n_times: int = 201, dt: float = 82.05, energy: float = 0.3,
                  fit_from_fs: float = 200.0, block: int = 4):
    """Armchair ribbon of 95 dimer lines (W = 11.7 nm) and 32768 chains along the periodic
    transport direction, n = 1 % vacancies, MSD up to (n_times - 1) dt (dt = 82.05 hbar/gamma0
    = 20 fs, 4 ps in all).  At ``energy``: the raw MSD, its Pade fit over t >= fit_from_fs
    (Eq. 58), sigma^E1 from the fitted derivative, sigma^E2 from the raw MSD, L = 2 sqrt(DX^2),
    and G = (W / L) sigma^E1 (Eq. 59) with a fit ln G = ln G_0 - L / xi over 0.1 <= G <= G_0 / 2
    (e^2/h)."""
    en = np.array([energy])
    w = ki.Workload(ki.AGNR, nx, ny, vacancy_conc=conc, n_vec=n_vec)
    c = einstein_curves(w, n_vec, n_moments, n_times, dt, en, block=block)
    t = c["t_fs"]
    rho = float(c["rho"][0])
    dx2 = c["rho_dx2"][:, 0] / rho
    width = nx * np.sqrt(3.0) / 2.0 * w.bond_nm
    sel = t >= fit_from_fs
    m, n = 2, 2
    coef = fit_msd(t, dx2, fit_from_fs, m, n)
    fit, dfit = pade_eval(coef, t, m, n)
    sigma_e1_fit = H_EV_FS * 0.5 * rho * dfit
    sigma_e1_raw = c["sigma_e1"][:, 0]
    sigma_e2_raw = c["sigma_e2"][:, 0]
    # raw MSD before the fitted range, the fit inside it
    msd_used = np.where(sel, fit, dx2)
    sigma_used = np.where(sel, sigma_e1_fit, sigma_e1_raw)
    length = 2.0 * np.sqrt(np.maximum(msd_used, 0.0))
    g = np.where(length > 0, width / np.maximum(length, 1e-300) * sigma_used, 0.0)
    out = {"sites": w.n_sites, "width_nm": width, "vacancies": len(w.vacancies), "vectors": n_vec,
           "energy_ev": energy, "t_fs": t.tolist(), "msd_raw_nm2": dx2.tolist(), "msd_fit_nm2": fit.tolist(),
           "pade_order": [m, n], "pade_coef": coef.tolist(), "fit_from_fs": fit_from_fs,
           "fit_rel_rms": float(np.sqrt(np.mean((fit[sel] - dx2[sel]) ** 2)) / np.mean(dx2[sel])),
           "sigma_e1_fit": sigma_e1_fit.tolist(), "sigma_e1_raw": sigma_e1_raw.tolist(),
           "sigma_e2_raw": sigma_e2_raw.tolist(), "length_nm": length.tolist(),
           "conductance_e2h": g.tolist(), "gpu_seconds": c["gpu_seconds"]}
    gmax = g[1:].max()
    ok = (g > 0.1) & (g <= 0.5 * gmax) & (t > 0)
    ok &= np.arange(len(t)) > int(np.argmax(g))
    if ok.sum() >= 3:
        slope, icept = np.polyfit(length[ok], np.log(g[ok]), 1)
        out["xi_nm"] = float(-1.0 / slope) if slope < 0 else None
        out["g0_e2h"] = float(np.exp(icept))
    return out


def main(argv=None):
    import argparse

    ap = argparse.ArgumentParser(description="Transport regimes of Sec. 5 on one GPU")
    ap.add_argument("--which", choices=["ballistic", "diffusive", "localized", "all"], default="all")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    res = {}
    t0 = time.perf_counter()
    if a.which in ("ballistic", "all"):
        res["ballistic"] = run_ballistic(open_cells=(512, 512))
    if a.which in ("diffusive", "all"):
        res["diffusive"] = run_diffusive()
    if a.which in ("localized", "all"):
        res["localized"] = run_localized()
    res["wall_seconds"] = time.perf_counter() - t0
    text = json.dumps(res)
    print(text)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text + "\n")


if __name__ == "__main__":
    main()
