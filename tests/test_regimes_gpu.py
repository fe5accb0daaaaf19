"""Transport regimes of Sec. 5 through the library, at reduced sizes: ballistic length
of pristine graphene (Eq. 50), Green-Kubo = Einstein in the diffusive regime with the
semi-classical conductivity definitions (Eqs. 53-54), and the localized-regime Pade fit
of the MSD (Eq. 58) with the conductance of Eq. 59."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1307_0288_gb300 import regimes  # noqa: E402


def test_pristine_ballistic_length_grows_as_sqrt2_vf_t():
    """Periodic pristine sheet: DX^2 = <v_x^2> t^2 with <v_x^2> = v_F^2 / 2 near the Dirac
    point, so L = 2 sqrt(DX^2) -> sqrt(2) v_F t.  Interband (Zitterbewegung) terms add a
    bounded O((hbar v_F / 2E)^2) to DX^2, so L / (sqrt(2) v_F t) falls towards 1; from
    t = 10 fs on it is within 3 %.  Two sample lengths give the same L."""
    res = regimes.run_ballistic(cells=((256, 256), (512, 256)), n_vec=4, n_moments=1500, n_times=9, dt=10.0)
    for s in res["samples"]:
        t = np.array(s["t_fs"][1:])
        r = np.array(s["ratio_to_sqrt2_vF_t"])
        assert np.all(np.diff(r) < 0), r
        assert np.all(np.abs(r[t >= 10.0] - 1.0) < 0.03), r
    assert res["max_rel_diff_between_lengths"] < 0.03


def test_open_boundary_length_saturates_below_the_sample_length():
    """Sec. 5.1, non-periodic boundary along the transport direction (126 nm sample): L(t)
    first follows the periodic sample, then stays below the sample length L_x (classical
    free flight between the two ends peaks near 0.93 L_x at t = L_x / v_F and settles at
    0.82 L_x), while L(t) of the periodic sample of the same size keeps growing."""
    res = regimes.run_ballistic(cells=((512, 128),), n_vec=4, n_moments=1500, n_times=21, dt=41.0,
                                open_cells=(512, 128), open_times=61, open_dt=41.0)
    per, opn = res["samples"]
    assert opn["boundary_x"] == "open" and per["boundary_x"] == "periodic"
    lx = opn["sample_length_nm"]
    t = np.array(opn["t_fs"])
    l_open = np.array(opn["L_nm"])
    l_per = np.array(per["L_nm"])
    assert abs(l_open[1] / l_per[1] - 1.0) < 0.08, (l_open[1], l_per[1])     # t = 10 fs
    late = t >= 1.5 * lx / res["v_f_nm_per_fs"]
    assert np.all(l_open < lx), l_open / lx
    assert np.all(l_open[late] > 0.6 * lx), l_open[late] / lx
    assert l_per[-1] > 1.2 * lx


def test_green_kubo_and_einstein_agree_in_the_diffusive_regime():
    """Sheet with 2 % vacancies: sigma^GK (VAC) and sigma^E1 (MSD) from the same vectors
    agree (Sec. 5.2), and sigma_sc by block average is below sigma_sc by maximum."""
    res = regimes.run_diffusive(cells=(128, 128), conc=0.02, n_vec=8, n_moments=1000, n_times=41, dt=0.82,
                                t_block=(3.0, 8.0), gk_vectors=8, gk_times=41, block=8)
    g = res["gk_vs_e1"]
    gk = np.array(g["gk_mean_abs_E_ge_0.3"][1:])
    e1 = np.array(g["e1_mean_abs_E_ge_0.3"][1:])
    assert np.max(np.abs(gk - e1)) < 0.05 * np.max(np.abs(e1)), (gk, e1)
    s_max, s_avg = np.array(res["sigma_sc_max"]), np.array(res["sigma_sc_average"])
    assert np.all(s_avg <= s_max + 1e-12)
    assert np.all(np.isfinite(s_max)) and np.all(s_max > 0)


def test_localized_msd_pade_fit_and_conductance():
    """Armchair ribbon with 2 % vacancies over long times: the Pade [2/2] fit follows the
    raw MSD over the fitted range, sigma^E2 stays positive, and G = (W/L) sigma^E1
    decreases with the length."""
    res = regimes.run_localized(nx=23, ny=8192, conc=0.02, n_vec=16, n_moments=1000, n_times=81, dt=20.0,
                                energy=0.3, fit_from_fs=100.0, block=16)
    assert res["fit_rel_rms"] < 0.05, res["fit_rel_rms"]
    assert min(res["pade_coef"][3:]) >= 0.0          # no pole for t >= 0
    e2 = np.array(res["sigma_e2_raw"][1:])
    assert np.all(e2 > 0)
    t = np.array(res["t_fs"])
    g = np.array(res["conductance_e2h"])
    late = t >= 100.0
    assert g[late][-1] < g[late][0]
