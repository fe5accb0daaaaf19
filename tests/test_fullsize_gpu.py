"""GPU parity at sizes where every kernel runs its full-size code path.

The per-step recursion kernels use one resident wave of CTAs (SMs x CTAs per SM x
threads) and a grid-stride loop over the N R site-vectors; the fused surrogate kernel
runs one CTA per SM over pairs of 128-row tiles, with a weight ring, mbarrier phases
and double-buffered TMEM accumulators reused from one pair to the next.  Small cases
run each of these loops once per thread or CTA; the cases here run them many times,
with ragged tails, and compare with the oracle:

* VAC (Algorithm 2) and MSD (Algorithm 3) on a 1,048,576-site sheet, FP64 at 1e-10,
  with and without Anderson disorder (the on-site variants of the kernels), and in
  complex64 at 2e-5 (the paired float4 kernels);
* all 3000 DOS moments (Algorithm 5, Chebyshev doubling) of a 524,288-site sheet with
  4 vectors, the high-order moments where rounding accumulates;
* the surrogate network (3 -> 256^4 -> 1, GELU) on 131,072 + 77 rows, every output
  against the FP64 oracle network, and on the 1,048,576-row batch of the benchmark on
  sampled rows, plus the invariance of each row's output under a permutation of the
  batch (a row's result must not depend on the tile, CTA or ring slot that computed it).

Tolerances and norms are those of the other parity tests: per vector
max |C_gpu - C_oracle| / max |C_oracle|.
"""
import numpy as np
import pytest

import kg_inputs as ki
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1307_0288_gb300 as kg  # noqa: E402
from oracle import mlp as omlp  # noqa: E402

TOL_MOMENTS = 1e-10
TOL_C64_MOMENTS = 2e-5
TOL_BF16 = 3e-2   # surrogate outputs: BF16 weights and activations, FP32 accumulation


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _one_wave_threads():
    return torch.cuda.get_device_properties(0).multi_processor_count * 2 * 512


# ------------------------------------------------------------------ VAC / MSD at 1M sites

SHEET_1M = dict(cx=512, cy=512, vacancy_conc=0.01)


@pytest.mark.parametrize("anderson", [0.0, 1.0])
def test_vac_1m_sites_grid_stride_matches_oracle(anderson):
    """512 x 512 cells (1,048,576 sites), 1 % vacancies, 2 vectors (2.1M site-vectors,
    about 13 items per thread of the one-wave grid), 2 correlation times of
    dt = hbar/gamma0, M = 32."""
    w = ki.sheet_cells(SHEET_1M["cx"], SHEET_1M["cy"], vacancy_conc=SHEET_1M["vacancy_conc"],
                       anderson_w_ev=anderson, lattice_seed=41, n_vec=2)
    assert w.n_sites * 2 > 8 * _one_wave_threads()
    h = kg.from_workload(w)
    ho = oracle.from_workload(w)
    phi = w.vectors(2)
    got = kg.vac(h, phi, 32, 2, 1.0)
    for r in range(2):
        want = oracle.vac_moments(ho, phi[:, r], 32, 2, 1.0)
        assert _rel(got[r], want) < TOL_MOMENTS, (anderson, r)


def test_msd_1m_sites_anderson_grid_stride_matches_oracle():
    """The MSD loop (U(dt), [X,U(dt)] and the doubling KPM step, on-site variants) on the
    1,048,576-site sheet with Anderson disorder W = 1 eV, 2 vectors, dt = 2 hbar/gamma0."""
    w = ki.sheet_cells(SHEET_1M["cx"], SHEET_1M["cy"], vacancy_conc=SHEET_1M["vacancy_conc"],
                       anderson_w_ev=1.0, lattice_seed=42, n_vec=2)
    h = kg.from_workload(w)
    ho = oracle.from_workload(w)
    phi = w.vectors(2)
    got = kg.msd(h, phi, 32, 2, 2.0)
    for r in range(2):
        want = oracle.msd_moments(ho, phi[:, r], 32, 2, 2.0)
        assert _rel(got[r], want) < TOL_MOMENTS, r


@pytest.mark.parametrize("fn", ["vac", "msd"])
def test_c64_1m_sites_grid_stride_matches_oracle(fn):
    """complex64 vectors (paired float4 kernels, 4 vectors) on the 1,048,576-site sheet
    with Anderson disorder, against the FP64 oracle at the complex64 tolerance."""
    w = ki.sheet_cells(SHEET_1M["cx"], SHEET_1M["cy"], vacancy_conc=SHEET_1M["vacancy_conc"],
                       anderson_w_ev=0.8, lattice_seed=43, n_vec=4)
    h = kg.from_workload(w)
    ho = oracle.from_workload(w)
    phi = w.vectors(4)
    run = kg.vac if fn == "vac" else kg.msd
    ref = oracle.vac_moments if fn == "vac" else oracle.msd_moments
    got = run(h, phi, 32, 2, 1.5, precision=kg.KG_C64)
    for r in (0, 3):
        want = ref(ho, phi[:, r], 32, 2, 1.5)
        assert _rel(got[r], want) < TOL_C64_MOMENTS, r


def test_dos_3000_moments_half_million_sites_all_moments():
    """All M = 3000 DOS moments (1499 doubling steps) of a 1024 x 512-site sheet
    (524,288 sites, 0.5 % vacancies) with 4 vectors, the block width of the
    benchmark: moments up to n = 2999 against the oracle's plain recursion for vector
    0 (the oracle does not use the doubling identity, so this also pins the doubling
    at high order)."""
    w = ki.sheet_cells(512, 256, vacancy_conc=0.005, lattice_seed=44, n_vec=4)
    h = kg.from_workload(w)
    phi = w.vectors(4)
    got = kg.dos_moments(h, phi, 3000)
    ho = oracle.from_workload(w)
    want = oracle.kpm_moments(ho, phi[:, 0], phi[:, 0], 3000)
    assert _rel(got[0], want) < TOL_MOMENTS
    # the last ten moments against their own magnitude (O(sqrt N) against C_0 = N)
    tail = slice(2990, 3000)
    assert _rel(got[0, tail], want[tail]) < 1e-8


# ------------------------------------------------------------------ surrogate at full size

def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, size=(n, 3)).astype(np.float32)


@pytest.mark.parametrize("rows", [131072, 131072 + 77])
def test_mlp_forward_persistent_loop_matches_oracle(rows):
    """131,072 (+77) rows = 1024 (+1) tiles of 128 rows: each of the SM-count CTAs of the
    fused kernel runs three or four tile pairs, so the 3-slot weight ring wraps across
    pairs and every mbarrier phase and TMEM buffer is reused.  Every output against the
    FP64 oracle network."""
    assert rows >= 2 * torch.cuda.get_device_properties(0).multi_processor_count * 128 * 3
    p = omlp.init_params(7)
    net = kg.Mlp(p.astype(np.float32))
    x = _inputs(rows, 11)
    y = np.asarray(net.forward(x), dtype=np.float64)
    ref = omlp.forward(p, x)
    assert np.all(np.isfinite(y))
    assert _rel(y, ref) < TOL_BF16


def test_mlp_forward_batch_1m_sampled_and_permutation_invariant():
    """The benchmark's batch of 1,048,576 rows on device tensors (27 tile pairs per CTA):
    9,000 sampled rows (spread over the batch, and the last tile) against the oracle,
    and every row's output bit-identical after a random permutation of the batch."""
    n = 1 << 20
    p = omlp.init_params(3)
    net = kg.Mlp(p.astype(np.float32))
    x = _inputs(n, 12)
    xd = torch.from_numpy(x).to("cuda")
    y = torch.zeros(n, dtype=torch.float32, device="cuda")
    net.forward(xd, out=y)
    rows = np.unique(np.concatenate([np.linspace(0, n - 1, 8872).astype(np.int64), np.arange(n - 128, n)]))
    got = y.cpu().numpy()
    assert np.all(np.isfinite(got))
    ref = omlp.forward(p, x[rows])
    assert _rel(got[rows], ref) < TOL_BF16
    perm = torch.from_numpy(np.random.default_rng(13).permutation(n)).to("cuda")
    y2 = torch.zeros(n, dtype=torch.float32, device="cuda")
    net.forward(xd[perm].contiguous(), out=y2)
    assert torch.equal(y2, y[perm])


def test_dos_3000_moments_bench_sheet_all_moments():
    """The benchmark's sheet and launch configuration (2048 x 1024 sites, 0.5 % vacancies,
    4 vectors, M = 3000): every one of the 3000 DOS moments of vector 0 against the oracle's
    plain recursion, so the high-order moments of the doubling identity are pinned at full
    size (about 45 s of single-thread oracle time)."""
    w = ki.sheet_cells(1024, 512, vacancy_conc=0.005, n_vec=4)
    h = kg.from_workload(w)
    phi = w.vectors(4)
    got = kg.dos_moments(h, phi, 3000)
    ho = oracle.from_workload(w)
    want = oracle.kpm_moments(ho, phi[:, 0], phi[:, 0], 3000)
    assert _rel(got[0], want) < TOL_MOMENTS
    tail = slice(2990, 3000)
    assert _rel(got[0, tail], want[tail]) < 1e-8
