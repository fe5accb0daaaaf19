"""Batched uneven instances in one persistent launch (kg_batched_dos_moments):
parity with the oracle and with the single-instance path, the autotuner, and the
failure detection of the bounded inter-CTA waits."""
import numpy as np
import pytest

import kg_inputs as ki
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1307_0288_gb300 as kg  # noqa: E402

TOL_MOMENTS = 1e-10


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def _ribbons(n_vec):
    """Five uneven zigzag ribbons: widths 8..40 chains, lengths 40..700 cells, Anderson
    W = 0.5..2 eV, some with vacancies; the last is tiny (a ragged, single-CTA member)."""
    spec = [(8, 700, 0.5, 0.0), (23, 90, 1.0, 0.01), (40, 40, 2.0, 0.0), (15, 300, 1.5, 0.02),
            (9, 4, 0.8, 0.0)]
    return [ki.zgnr(w, l, anderson_w_ev=W, vacancy_conc=v, lattice_seed=100 + i, n_vec=n_vec)
            for i, (w, l, W, v) in enumerate(spec)]


@pytest.fixture(autouse=True)
def _fresh_batch():
    yield
    kg.batched_release()


def test_batched_matches_oracle_and_single_path():
    ws = _ribbons(8)
    hs = [kg.from_workload(w) for w in ws]
    phis = [w.vectors(8) for w in ws]
    got = kg.batched_dos_moments(hs, phis, 101)
    for i, (w, h, phi) in enumerate(zip(ws, hs, phis)):
        single = kg.dos_moments(h, phi, 101)
        assert _rel(got[i], single) < 1e-12, i
        ho = oracle.from_workload(w)
        for r in (0, 7):
            want = oracle.kpm_moments(ho, phi[:, r], phi[:, r], 101)
            assert _rel(got[i, r], want) < TOL_MOMENTS, (i, r)
    t = kg.batched_tuning()
    assert t["block_width"] == 8 and t["n_ctas"] >= len(ws)


def test_batched_64_vectors_autotuned():
    ws = _ribbons(64)[:3]
    hs = [kg.from_workload(w) for w in ws]
    phis = [w.vectors(64) for w in ws]
    got = kg.batched_dos_moments(hs, phis, 64)
    t = kg.batched_tuning()
    assert t["block_width"] in (8, 16, 32, 64)
    # every block width with both tile schedules (one occupancy wave of CTAs, or half)
    assert sorted(bw for bw, _, _ in t["log"]) == [8, 8, 16, 16, 32, 32, 64, 64]
    for bw in (8, 16, 32, 64):
        ctas = sorted(c for w_, c, _ in t["log"] if w_ == bw)
        assert ctas[0] < ctas[1] and ctas[0] >= len(ws)
    for i, (h, phi) in enumerate(zip(hs, phis)):
        assert _rel(got[i], kg.dos_moments(h, phi, 64)) < 1e-12
    # repeated calls replay the captured graph and give identical results
    again = kg.batched_dos_moments(hs, phis, 64)
    assert np.array_equal(again, got)


def test_batched_wait_timeout_is_reported_and_recoverable():
    """A CTA that stops publishing its step flag makes its neighbours' bounded waits
    run out: the call returns KG_ETIMEOUT, and the next normal call succeeds."""
    ws = _ribbons(8)[:2]
    hs = [kg.from_workload(w) for w in ws]
    phis = [w.vectors(8) for w in ws]
    ref = kg.batched_dos_moments(hs, phis, 41)
    kg.batched_test_stall(1)
    with pytest.raises(kg.KgError) as e:
        kg.batched_dos_moments(hs, phis, 41)
    assert e.value.status == -4
    kg.batched_test_stall(-1)
    assert np.array_equal(kg.batched_dos_moments(hs, phis, 41), ref)


def test_batched_sixteen_uneven_ribbons_sampled():
    """The 16-ribbon set (widths 8..64 chains, lengths 1k..16k cells, W = 0.5..2 eV) with
    8 vectors, M = 400: every moment bounded by C_0, the first 12 moments of vector 0
    of every ribbon against the oracle."""
    ws = ki.ribbon_set_16(n_vec=8)
    hs = [kg.from_workload(w) for w in ws]
    phis = [w.vectors(8) for w in ws]
    got = kg.batched_dos_moments(hs, phis, 400)
    assert np.all(np.abs(got.real) <= got[..., :1].real * (1 + 1e-12))
    for i, (w, phi) in enumerate(zip(ws, phis)):
        ho = oracle.from_workload(w)
        want = oracle.kpm_moments(ho, phi[:, 0], phi[:, 0], 12)
        assert _rel(got[i, 0, :12], want) < TOL_MOMENTS, i
