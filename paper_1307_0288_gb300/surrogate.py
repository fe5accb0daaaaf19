"""Learned surrogate of sigma(E, t) across vacancy concentration.

The method generates the data: for each (concentration n, disorder seed) a periodic
sheet with n N random vacancies is built, kg_vac gives the VAC moments, and the host
sums give the Green-Kubo running conductivity sigma^GK(E, t) (Eqs. 6, 30, 35) on an
energy grid and the correlation times t_m.  A small MLP (kg_mlp, BF16 tensor-core
kernels) learns (log n, E / E_max, log t) -> sigma.  Concentrations held out of the
training set are predicted and compared with the ensemble average of plain-method runs
at those concentrations; the method stays the fallback and the reference for the error.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

import kg_inputs as ki

from . import (KG_C64, KG_FP64, KG_SIGMA_GK, HBAR_EV_FS, Mlp, conductivity, from_workload,
               kpm_sum, vac)


@dataclass
class Grid:
    """Sampling of one sigma(E, t) surface."""
    cells: tuple = (512, 512)
    n_moments: int = 2000
    n_times: int = 64
    dt: float = 1.0                 # hbar / gamma0
    n_energies: int = 201
    gamma0_ev: float = 2.7
    n_min: float = 0.0005           # vacancy concentration range (0.05 % .. 2 %)
    n_max: float = 0.02

    @property
    def energies(self) -> np.ndarray:
        return np.linspace(-3 * self.gamma0_ev, 3 * self.gamma0_ev, self.n_energies)

    @property
    def times_fs(self) -> np.ndarray:
        return np.arange(self.n_times) * self.dt * HBAR_EV_FS / self.gamma0_ev


def init_params(seed: int, hidden: int = 256) -> np.ndarray:
    """Initial FP32 parameters in the library's flat layout: weights uniform in
    +-1/sqrt(fan_in), biases zero."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in [(hidden, 3), (hidden, hidden), (hidden, hidden), (hidden, hidden), (1, hidden)]:
        b = 1.0 / np.sqrt(fan_in)
        parts += [rng.uniform(-b, b, size=fan_out * fan_in), np.zeros(fan_out)]
    return np.concatenate(parts).astype(np.float32)


def sigma_surface(conc: float, seed: int, grid: Grid, precision: int = KG_C64):
    """sigma^GK(E, t_m) [N_c][n_E] in e^2/h for one disorder realisation (one vector),
    and the seconds the method took."""
    w = ki.sheet_cells(*grid.cells, vacancy_conc=conc, lattice_seed=seed, vector_seed=seed + 1)
    t0 = time.perf_counter()
    h = from_workload(w)
    mu = vac(h, w.vectors(1), grid.n_moments, grid.n_times, grid.dt, precision=precision)[0]
    dens = kpm_sum(mu.real, grid.energies, h.emax_ev, h.area_nm2)
    sig = conductivity(KG_SIGMA_GK, dens, grid.times_fs[1])
    return sig, time.perf_counter() - t0, h.emax_ev


def features(conc, energies_ev, times_fs, emax_ev: float, grid: Grid) -> np.ndarray:
    """[len(t) * len(E)][3] float32: scaled log concentration, E / E_max, scaled log t."""
    lo, hi = np.log(grid.n_min), np.log(grid.n_max)
    f0 = 2.0 * (np.log(conc) - lo) / (hi - lo) - 1.0
    t = np.asarray(times_fs)
    t1, tn = grid.times_fs[1], grid.times_fs[-1]
    f2 = 2.0 * np.log(t / t1) / np.log(tn / t1) - 1.0
    ee, tt = np.meshgrid(np.asarray(energies_ev) / emax_ev, f2, indexing="xy")
    return np.stack([np.full(ee.size, f0), ee.ravel(), tt.ravel()], axis=1).astype(np.float32)


@dataclass
class Dataset:
    grid: Grid
    concentrations: np.ndarray
    seeds: int
    held_out: list
    surfaces: dict = field(default_factory=dict)     # (i, s) -> sigma [N_c][n_E]
    method_seconds: list = field(default_factory=list)
    emax_ev: float = 0.0

    def samples(self, idx, scale: float):
        """Training pairs (t >= t_1) of concentrations idx, all seeds."""
        xs, ys = [], []
        for i in idx:
            for s in range(self.seeds):
                sig = self.surfaces[(i, s)][1:]
                xs.append(features(self.concentrations[i], self.grid.energies, self.grid.times_fs[1:],
                                   self.emax_ev, self.grid))
                ys.append((sig / scale).astype(np.float32).ravel())
        return np.concatenate(xs), np.concatenate(ys)


def generate(grid: Grid, n_conc: int = 40, seeds: int = 5, held_out=None, precision=KG_C64,
             train_precision=None, log=None) -> Dataset:
    conc = np.geomspace(grid.n_min, grid.n_max, n_conc)
    if held_out is None:
        held_out = list(range(2, n_conc, 5))
    ds = Dataset(grid, conc, seeds, list(held_out))
    for i, c in enumerate(conc):
        # held-out concentrations are the reference: plain FP64 runs
        prec = KG_FP64 if i in held_out else (train_precision if train_precision is not None else precision)
        for s in range(seeds):
            sig, sec, emax = sigma_surface(float(c), 7000 + 10 * i + s, grid, prec)
            ds.surfaces[(i, s)] = sig
            ds.method_seconds.append(sec)
            ds.emax_ev = emax
            if log:
                log(f"conc {c:.5f} seed {s}: {sec:.2f} s")
    return ds


def train(ds: Dataset, init_params, *, scale: float = 10.0, epochs: int = 20, batch: int = 8192,
          lr: float = 2e-3, seed: int = 0, log=None):
    train_idx = [i for i in range(len(ds.concentrations)) if i not in ds.held_out]
    x, y = ds.samples(train_idx, scale)
    net = Mlp(np.asarray(init_params, dtype=np.float32))
    rng = np.random.default_rng(seed)
    losses = []
    t0 = time.perf_counter()
    steps = 0
    for ep in range(epochs):
        order = rng.permutation(len(x))
        cur_lr = lr * 0.5 * (1 + np.cos(np.pi * ep / epochs))
        ep_loss = []
        for k in range(0, len(x) - batch + 1, batch):
            sel = order[k:k + batch]
            ep_loss.append(net.train_step(x[sel], y[sel], cur_lr))
            steps += 1
        losses.append(float(np.mean(ep_loss)))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.3e}")
    return net, {"losses": losses, "train_seconds": time.perf_counter() - t0, "steps": steps,
                 "samples": int(len(x)), "scale": scale}


def evaluate(ds: Dataset, net: Mlp, scale: float):
    """For every held-out concentration: relative L2 error of the surrogate against the
    ensemble mean of the plain-method runs, and of a single method run against the
    mean of the remaining runs (what one run of the method gives without the network)."""
    out = []
    for i in ds.held_out:
        runs = np.stack([ds.surfaces[(i, s)][1:] for s in range(ds.seeds)])
        mean = runs.mean(axis=0)
        x = features(ds.concentrations[i], ds.grid.energies, ds.grid.times_fs[1:], ds.emax_ev, ds.grid)
        t0 = time.perf_counter()
        pred = net.forward(x).reshape(mean.shape) * scale
        infer_s = time.perf_counter() - t0
        single = []
        for s in range(ds.seeds):
            others = np.delete(runs, s, axis=0).mean(axis=0)
            single.append(np.linalg.norm(runs[s] - others) / np.linalg.norm(others))
        out.append({"concentration": float(ds.concentrations[i]),
                    "surrogate_rel_err": float(np.linalg.norm(pred - mean) / np.linalg.norm(mean)),
                    "single_run_rel_err": float(np.mean(single)),
                    "surrogate_seconds": infer_s})
    return out


def main(argv=None):
    """Full workflow: 40 concentrations (0.05 % .. 2 %, log-spaced) x 5 seeds of
    512 x 512-cell sheets (1,048,576 sites), M = 2000, 64 correlation times of
    dt = hbar/gamma0, 201 energies; 8 concentrations held out (plain FP64 runs), the
    rest generated in complex64; train, evaluate, print one JSON summary."""
    import argparse
    import json

    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--n-conc", type=int, default=40)
    ap.add_argument("--seeds", type=int, default=5)
    ap.add_argument("--epochs", type=int, default=20)
    a = ap.parse_args(argv)
    grid = Grid()
    t0 = time.perf_counter()
    ds = generate(grid, n_conc=a.n_conc, seeds=a.seeds)
    gen_s = time.perf_counter() - t0
    net, info = train(ds, init_params(1), epochs=a.epochs)
    res = evaluate(ds, net, info["scale"])
    summary = {
        "grid": {"sites": 4 * grid.cells[0] * grid.cells[1], "moments": grid.n_moments,
                 "times": grid.n_times, "energies": grid.n_energies},
        "runs": len(ds.surfaces), "generation_seconds": gen_s,
        "method_seconds_per_run": float(np.mean(ds.method_seconds)),
        "train": info, "held_out": res,
        "mean_surrogate_rel_err": float(np.mean([r["surrogate_rel_err"] for r in res])),
        "mean_single_run_rel_err": float(np.mean([r["single_run_rel_err"] for r in res])),
        "mean_surrogate_seconds": float(np.mean([r["surrogate_seconds"] for r in res])),
    }
    text = json.dumps(summary)
    print(text)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text + "\n")


if __name__ == "__main__":
    main()
