"""Seeded synthetic inputs for the Kubo-Greenwood transport path.

This module is the only code shared by the CUDA path's tests/benchmark and the
CPU oracle.  It holds none of the method's arithmetic: it only draws the random
numbers that the method consumes as inputs (which atoms are removed, the Anderson
on-site energies, the random phases of the trace-estimator vectors) and lays
them out.  Everything downstream (lattice, Hamiltonian, recursion, sums) is
computed independently by each side.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used in counter mode:
``x_k = mix64(key + (k + 1) * GAMMA)`` with ``key = mix64(seed + stream * GAMMA)``,
where ``mix64`` is the SplitMix64 output finaliser.  Streams separate the
independent draws of one workload.

Lattice sizes follow the paper's convention (Sec. 2): ``N = N_x * N_y`` carbon
atoms, ``N_x`` dimer lines along the zigzag direction and ``N_y`` zigzag chains.
A rectangular 4-atom cell is 2 dimer lines x 2 chains, so ``c_x x c_y`` cells
give ``N_x = 2 c_x`` and ``N_y = 2 c_y``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_VACANCY = 0
STREAM_ANDERSON = 1
STREAM_VECTOR0 = 16  # random vector r uses stream STREAM_VECTOR0 + r

SHEET, ZGNR, AGNR, SHEET_OPEN_X = 0, 1, 2, 3


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def splitmix64(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Counter-mode SplitMix64 words ``x_start .. x_{start+count-1}`` of one stream."""
    with np.errstate(over="ignore"):
        key = _mix64(np.array([(seed + stream * 0x9E3779B97F4A7C15) & (2**64 - 1)],
                              dtype=np.uint64))[0]
        k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix64(key + k * GAMMA)


def uniform53(seed: int, stream: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1): the top 53 bits of each word times 2^-53."""
    return (splitmix64(seed, stream, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def vacancy_sites(n_sites: int, n_vac: int, seed: int) -> np.ndarray:
    """Exactly ``n_vac`` distinct sites, by a seeded partial Fisher-Yates shuffle.

    Step k swaps position k with position ``k + floor(w_k * (N - k) / 2^32)``,
    ``w_k`` the top 32 bits of word k (integer arithmetic, never out of range).
    Returned sorted, as int64.
    """
    if n_vac < 0 or n_vac > n_sites:
        raise ValueError("n_vac out of range")
    if n_vac == 0:
        return np.zeros(0, dtype=np.int64)
    w = splitmix64(seed, STREAM_VACANCY, n_vac) >> np.uint64(32)
    perm = np.arange(n_sites, dtype=np.int64)
    for k in range(n_vac):
        m = n_sites - k
        j = k + int((int(w[k]) * m) >> 32)
        perm[k], perm[j] = perm[j], perm[k]
    return np.sort(perm[:n_vac])


def anderson_onsite(n_sites: int, w_ev: float, seed: int) -> np.ndarray:
    """On-site energies uniform in [-W/2, W/2] eV (Anderson disorder)."""
    u = uniform53(seed, STREAM_ANDERSON, n_sites)
    return w_ev * (u - 0.5)


def random_phase_vectors(n_sites: int, n_vec: int, seed: int,
                         vacancies: np.ndarray | None = None) -> np.ndarray:
    """Random-phase vectors ``phi_n = exp(i theta_n)``, ``theta_n = 2 pi u_n``.

    Layout ``[N][R]`` complex128 (site-major, vector-minor).  Components on removed
    atoms are zero, so ``<phi|phi> = N - N_v`` for every vector.
    """
    out = np.empty((n_sites, n_vec), dtype=np.complex128)
    for r in range(n_vec):
        theta = 2.0 * math.pi * uniform53(seed, STREAM_VECTOR0 + r, n_sites)
        out[:, r] = np.cos(theta) + 1j * np.sin(theta)
    if vacancies is not None and len(vacancies):
        out[vacancies, :] = 0.0
    return out


def n_vacancies(n_sites: int, concentration: float) -> int:
    """``N_v = round(n * N)`` for defect concentration ``n = N_v / N``."""
    return int(round(concentration * n_sites))


@dataclass
class Workload:
    """One synthetic system: lattice, defects and trace vectors."""
    kind: int
    nx: int
    ny: int
    gamma0_ev: float = 2.7
    bond_nm: float = 0.142
    vacancy_conc: float = 0.0
    anderson_w_ev: float = 0.0
    emax_margin: float = 1.05
    lattice_seed: int = 20130701
    vector_seed: int = 1000
    n_vec: int = 1
    vacancies: np.ndarray = field(default=None, repr=False)
    onsite: np.ndarray | None = field(default=None, repr=False)

    def __post_init__(self):
        n = self.nx * self.ny
        if self.vacancies is None:
            self.vacancies = vacancy_sites(n, n_vacancies(n, self.vacancy_conc),
                                           self.lattice_seed)
        if self.onsite is None and self.anderson_w_ev > 0:
            self.onsite = anderson_onsite(n, self.anderson_w_ev, self.lattice_seed)

    @property
    def n_sites(self) -> int:
        return self.nx * self.ny

    @property
    def emax_ev(self) -> float:
        """Spectral scale: margin * (3 gamma0 + W/2), an upper bound on |E|."""
        return self.emax_margin * (3.0 * self.gamma0_ev + 0.5 * self.anderson_w_ev)

    def vectors(self, n_vec: int | None = None) -> np.ndarray:
        return random_phase_vectors(self.n_sites, n_vec or self.n_vec,
                                    self.vector_seed, self.vacancies)

    def vacancy_mask(self) -> np.ndarray:
        m = np.zeros(self.n_sites, dtype=np.uint8)
        m[self.vacancies] = 1
        return m


def sheet_cells(cx: int, cy: int, **kw) -> Workload:
    """2D periodic sheet of ``cx x cy`` rectangular 4-atom cells."""
    return Workload(SHEET, 2 * cx, 2 * cy, **kw)


def zgnr(width_chains: int, length_cells: int, **kw) -> Workload:
    """Zigzag ribbon, ``w`` chains wide and ``l`` cells long (periodic along x)."""
    return Workload(ZGNR, 2 * length_cells, width_chains, **kw)


def ribbon_set_16(seed0: int = 20130701, n_vec: int = 64):
    """Sixteen uneven zigzag ribbons with Anderson disorder.

    Ribbon i (0..15): ``w_i = round(8 + 56 i / 15)`` chains,
    ``l_i = round(1024 * 16^(((7 i) mod 16) / 15))`` cells, ``W_i = 0.5 + 1.5 i / 15`` eV.
    """
    out = []
    for i in range(16):
        w = int(round(8 + 56 * i / 15))
        ell = int(round(1024 * 16 ** (((7 * i) % 16) / 15)))
        out.append(zgnr(w, ell, anderson_w_ev=0.5 + 1.5 * i / 15,
                        lattice_seed=seed0 + i, n_vec=n_vec))
    return out
