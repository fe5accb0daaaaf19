"""Python binding of the GB300 Kubo-Greenwood transport library (``libkg.so``).

Thin ctypes layer over the C ABI declared in ``include/kg.h``: every function here
has the name of the C entry point without the ``kg_`` prefix and only marshals
arguments (numpy arrays for host memory, torch CUDA tensors for device memory).
All computation runs in the library's CUDA kernels or its host C++ code; there is
no Python or CPU fallback.  If the library cannot be loaded, importing this
package raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

KG_SHEET, KG_ZGNR, KG_AGNR, KG_SHEET_OPEN_X = 0, 1, 2, 3
KG_FP64, KG_C64 = 0, 1
KG_OP_H, KG_OP_XH, KG_OP_V = 0, 1, 2
KG_U_FORWARD, KG_U_BACKWARD, KG_U_COMMUTATOR = 0, 1, 2
KG_SIGMA_GK, KG_SIGMA_E1, KG_SIGMA_E2 = 0, 1, 2
HBAR_EV_FS = 0.6582119569

_STATUS = {0: "KG_OK", -1: "KG_EINVAL", -2: "KG_ENOMEM", -3: "KG_ECUDA", -4: "KG_ETIMEOUT",
           -5: "KG_ENUMERIC", -6: "KG_ENODEV"}


class KgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Lattice(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("nx", ctypes.c_int64),
                ("ny", ctypes.c_int64), ("gamma0_ev", ctypes.c_double),
                ("bond_nm", ctypes.c_double), ("emax_ev", ctypes.c_double)]


class _Run(ctypes.Structure):
    _fields_ = [("n_moments", ctypes.c_int32), ("n_vectors", ctypes.c_int32),
                ("n_times", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("dt", ctypes.c_double), ("bessel_tol", ctypes.c_double)]


class _Timing(ctypes.Structure):
    _fields_ = [("kpm_ms", ctypes.c_double), ("evolve_ms", ctypes.c_double),
                ("kpm_launches", ctypes.c_int64), ("evolve_launches", ctypes.c_int64),
                ("other_launches", ctypes.c_int64), ("kpm_site_steps", ctypes.c_double),
                ("evolve_site_steps", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double

# (name, restype, argtypes) of every exported entry point of include/kg.h
ABI = [
    ("kg_last_error", ctypes.c_char_p, []),
    ("kg_abi_version", _I, []),
    ("kg_build_hamiltonian", _I, [ctypes.POINTER(_Lattice), _P, _I64, _P, _P, ctypes.POINTER(_P)]),
    ("kg_hamiltonian_info", _I, [_P, _P, _P, _P, _P]),
    ("kg_destroy_hamiltonian", None, [_P]),
    ("kg_lattice_neighbors", _I, [ctypes.POINTER(_Lattice), _P, _I64, _P]),
    ("kg_dos_moments", _I, [_P, ctypes.POINTER(_Run), _P, _P]),
    ("kg_vac", _I, [_P, ctypes.POINTER(_Run), _P, _P]),
    ("kg_msd", _I, [_P, ctypes.POINTER(_Run), _P, _P]),
    ("kg_apply", _I, [_P, _I, _P, _P, _I]),
    ("kg_evolve", _I, [_P, _D, _I, _D, _P, _P, _I]),
    ("kg_timing_enable", _I, [_P, _I]),
    ("kg_timing_read", _I, [_P, ctypes.POINTER(_Timing)]),
    ("kg_fp64_fma_rate", _I, [_I, ctypes.POINTER(_D)]),
    ("kg_splitmix64", _I, [ctypes.c_uint64, ctypes.c_uint64, _I64, _I64, _P]),
    ("kg_n_vacancies", _I, [_I64, _D, ctypes.POINTER(_I64)]),
    ("kg_vacancy_sites", _I, [_I64, _I64, ctypes.c_uint64, _P]),
    ("kg_anderson_onsite", _I, [_I64, _D, ctypes.c_uint64, _P]),
    ("kg_random_phase_vectors", _I, [_I64, _I, ctypes.c_uint64, _P, _I64, _P]),
    ("kg_bessel_series", _I, [_D, _D, _I, _P, ctypes.POINTER(_I)]),
    ("kg_jackson", _I, [_I, _P]),
    ("kg_kpm_sum", _I, [_P, _I, _I, _P, _I, _D, _D, _P]),
    ("kg_conductivity", _I, [_I, _P, _I, _I, _D, _P]),
    ("kg_dos_moments_noalloc", _I, [_P, _P, _I64, _D, _I, _I, _P, _P, _P]),
    ("kg_batched_dos_moments", _I, [_P, _I, ctypes.POINTER(_Run), _P, _P]),
    ("kg_batched_tuning", _I, [_P, _P, _P, _I, _P, _P, _P]),
    ("kg_batched_release", _I, []),
    ("kg_batched_test_stall", _I, [_I]),
    ("kg_msd_resume", _I, [_P, ctypes.POINTER(_Run), _P, _P, _P, _P, _P]),
    ("kg_vac_resume", _I, [_P, ctypes.POINTER(_Run), _P, _P, _P, _P, _P]),
    ("kg_test_alloc_cap", _I, [ctypes.c_uint64]),
    ("kg_set_small_persistent", _I, [_I]),
    ("kg_ftm_dos_moments", _I, [_P, ctypes.POINTER(_Run), _P, _P]),
    ("kg_ftm_sum", _I, [_P, _I, _I, _P, _I, _D, _D, _P]),
    ("kg_ballistic", _I, [_P, _P, _I, _I, _D, _D, _P, _P]),
    ("kg_sigma_sc", _I, [_P, _I, _I, _D, _D, _D, _P, _P]),
    ("kg_pade_fit", _I, [_P, _P, _I, _I, _I, _P]),
    ("kg_pade_fit_positive", _I, [_P, _P, _I, _I, _I, _P]),
    ("kg_pade_eval", _I, [_P, _I, _I, _P, _I, _P, _P]),
    ("kg_mlp_create", _I, [_P, _P, ctypes.POINTER(_P)]),
    ("kg_mlp_destroy", None, [_P]),
    ("kg_mlp_get_params", _I, [_P, _P]),
    ("kg_mlp_forward", _I, [_P, _P, _I64, _P]),
    ("kg_mlp_gradients", _I, [_P, _P, _P, _I64, _P, ctypes.POINTER(_D)]),
    ("kg_mlp_train_step", _I, [_P, _P, _P, _I64, ctypes.c_float, ctypes.POINTER(_D)]),
    ("kg_mlp_launches", _I, [_P, ctypes.POINTER(_I64)]),
    ("kg_mlp_timing_enable", _I, [_P, _I]),
    ("kg_mlp_timing_read", _I, [_P, ctypes.POINTER(_D), ctypes.POINTER(_I64), ctypes.POINTER(_D)]),
    ("kg_mlp_gemm_test", _I, [_P, _P, _I64, _I, _P]),
]

_lib = None


def lib() -> ctypes.CDLL:
    """Loads ``libkg.so`` (building it from source first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise ImportError(f"libkg.so not found at {path}")
        L = ctypes.CDLL(path)
        for name, res, args in ABI:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise KgError(status, lib().kg_last_error().decode())


def last_error() -> str:
    return lib().kg_last_error().decode()


def abi_version() -> int:
    return lib().kg_abi_version()


# ----------------------------------------------------------------- pointer marshalling

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype=None, shape=None, writable=False):
    """(address, keep-alive object) of a numpy array or torch tensor."""
    if x is None:
        return None, None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), x
    a = np.asarray(x)
    if dtype is not None and a.dtype != dtype:
        if writable:
            raise ValueError(f"output array must have dtype {dtype}")
        a = a.astype(dtype)
    if not a.flags["C_CONTIGUOUS"]:
        if writable:
            raise ValueError("output array must be C-contiguous")
        a = np.ascontiguousarray(a)
    if shape is not None and a.size != int(np.prod(shape)):
        raise ValueError(f"array has {a.size} elements, expected {int(np.prod(shape))}")
    return a.ctypes.data, a


def _lattice(kind, nx, ny, gamma0_ev, bond_nm, emax_ev) -> _Lattice:
    return _Lattice(int(kind), 0, int(nx), int(ny), float(gamma0_ev), float(bond_nm), float(emax_ev))


# ----------------------------------------------------------------- Hamiltonian

class Hamiltonian:
    """Owns a ``kg_hamiltonian*`` (device-resident H~)."""

    def __init__(self, handle: int, kind: int, nx: int, ny: int):
        self._h = ctypes.c_void_p(handle)
        self.kind, self.nx, self.ny = kind, nx, ny
        n, na, emax, area = (ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double(),
                             ctypes.c_double())
        _check(lib().kg_hamiltonian_info(self._h, ctypes.byref(n), ctypes.byref(na),
                                         ctypes.byref(emax), ctypes.byref(area)))
        self.n, self.n_active, self.emax_ev, self.area_nm2 = n.value, na.value, emax.value, area.value

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None and self._h.value:
            lib().kg_destroy_hamiltonian(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_hamiltonian(kind: int, nx: int, ny: int, *, emax_ev: float, vacancies=None,
                      onsite_ev=None, gamma0_ev: float = 2.7, bond_nm: float = 0.142,
                      stream=None) -> Hamiltonian:
    """kg_build_hamiltonian.  ``stream``: a torch.cuda.Stream, a raw cudaStream_t, or None."""
    lat = _lattice(kind, nx, ny, gamma0_ev, bond_nm, emax_ev)
    vac = np.zeros(0, np.int64) if vacancies is None else np.ascontiguousarray(vacancies, np.int64)
    on = None if onsite_ev is None else np.ascontiguousarray(onsite_ev, np.float64)
    s = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
    out = ctypes.c_void_p()
    _check(lib().kg_build_hamiltonian(ctypes.byref(lat), vac.ctypes.data if len(vac) else None,
                                      len(vac), None if on is None else on.ctypes.data,
                                      ctypes.c_void_p(s), ctypes.byref(out)))
    return Hamiltonian(out.value, kind, nx, ny)


def from_workload(w, stream=None) -> Hamiltonian:
    """Hamiltonian of a ``kg_inputs.Workload``."""
    return build_hamiltonian(w.kind, w.nx, w.ny, emax_ev=w.emax_ev, vacancies=w.vacancies,
                             onsite_ev=w.onsite, gamma0_ev=w.gamma0_ev, bond_nm=w.bond_nm,
                             stream=stream)


def lattice_neighbors(kind: int, nx: int, ny: int, vacancies=None, *, gamma0_ev=2.7,
                      bond_nm=0.142, emax_ev=8.505) -> np.ndarray:
    """kg_lattice_neighbors (host only): int32 [3][N], -1 where absent."""
    lat = _lattice(kind, nx, ny, gamma0_ev, bond_nm, emax_ev)
    vac = np.zeros(0, np.int64) if vacancies is None else np.ascontiguousarray(vacancies, np.int64)
    out = np.empty((3, nx * ny), dtype=np.int32)
    _check(lib().kg_lattice_neighbors(ctypes.byref(lat), vac.ctypes.data if len(vac) else None,
                                      len(vac), out.ctypes.data))
    return out


# ----------------------------------------------------------------- moments

def _run(n_moments, n_vectors, n_times=1, precision=KG_FP64, dt=1.0, bessel_tol=1e-15) -> _Run:
    return _Run(int(n_moments), int(n_vectors), int(n_times), int(precision), float(dt),
                float(bessel_tol))


def _nvec(phi, n):
    shape = tuple(phi.shape)
    if len(shape) == 1:
        return 1
    if len(shape) == 2 and shape[0] == n:
        return int(shape[1])
    raise ValueError(f"phi must be [N] or [N][R] complex with N = {n}")


def _complex_in(phi):
    if _is_torch(phi):
        import torch
        if phi.dtype != torch.complex128:
            raise ValueError("device phi must be complex128")
        return _ptr(phi)
    return _ptr(np.ascontiguousarray(phi, dtype=np.complex128))


def _moments_call(fn, h: Hamiltonian, phi, run: _Run, shape, out):
    pp, keep = _complex_in(phi)
    if out is None:
        res = np.zeros(shape, dtype=np.complex128)
        op, keep_o = res.ctypes.data, res
    else:
        op, keep_o = _ptr(out, writable=True)
        res = out
    _check(fn(h.handle, ctypes.byref(run), ctypes.c_void_p(pp), ctypes.c_void_p(op)))
    return res


def dos_moments(h: Hamiltonian, phi, n_moments: int, precision: int = KG_FP64, out=None):
    """kg_dos_moments -> complex [R][M] (numpy, or ``out`` if given)."""
    r = _nvec(phi, h.n)
    run = _run(n_moments, r, 1, precision)
    return _moments_call(lib().kg_dos_moments, h, phi, run, (r, n_moments), out)


def vac(h: Hamiltonian, phi, n_moments: int, n_times: int, dt: float, *, bessel_tol=1e-15,
        precision: int = KG_FP64, out=None):
    """kg_vac -> complex [R][N_c][M]."""
    r = _nvec(phi, h.n)
    run = _run(n_moments, r, n_times, precision, dt, bessel_tol)
    return _moments_call(lib().kg_vac, h, phi, run, (r, n_times, n_moments), out)


def msd(h: Hamiltonian, phi, n_moments: int, n_times: int, dt: float, *, bessel_tol=1e-15,
        precision: int = KG_FP64, out=None):
    """kg_msd -> complex [R][N_c][M]."""
    r = _nvec(phi, h.n)
    run = _run(n_moments, r, n_times, precision, dt, bessel_tol)
    return _moments_call(lib().kg_msd, h, phi, run, (r, n_times, n_moments), out)


def _resume_call(fn, h: Hamiltonian, s0, s1, n_moments, n_times, dt, bessel_tol, precision):
    r = _nvec(s0, h.n)
    run = _run(n_moments, r, n_times, precision, dt, bessel_tol)
    p0, k0 = _complex_in(s0)
    p1, k1 = (_complex_in(s1) if s1 is not None else (0, None))
    mu = np.zeros((r, n_times, n_moments), dtype=np.complex128)
    o0 = np.zeros((h.n, r), dtype=np.complex128)
    o1 = np.zeros((h.n, r), dtype=np.complex128)
    _check(fn(h.handle, ctypes.byref(run), ctypes.c_void_p(p0), ctypes.c_void_p(p1 or None),
              ctypes.c_void_p(mu.ctypes.data), ctypes.c_void_p(o0.ctypes.data), ctypes.c_void_p(o1.ctypes.data)))
    squeeze = len(s0.shape) == 1
    return mu, (o0[:, 0] if squeeze else o0), (o1[:, 0] if squeeze else o1)


def msd_resume(h: Hamiltonian, psi, xi, n_moments: int, n_times: int, dt: float, *, bessel_tol=1e-15,
               precision: int = KG_FP64):
    """kg_msd_resume: advance (psi, xi) by n_times steps (xi None = fresh start) ->
    (moments [R][n_times][M] at the new times, psi', xi')."""
    return _resume_call(lib().kg_msd_resume, h, psi, xi, n_moments, n_times, dt, bessel_tol, precision)


def vac_resume(h: Hamiltonian, a, b, n_moments: int, n_times: int, dt: float, *, bessel_tol=1e-15,
               precision: int = KG_FP64):
    """kg_vac_resume: advance (A, B) by n_times steps (b None = fresh start, B = V A) ->
    (moments [R][n_times][M] at the new times, A', B')."""
    return _resume_call(lib().kg_vac_resume, h, a, b, n_moments, n_times, dt, bessel_tol, precision)


def test_alloc_cap(n_bytes: int):
    """kg_test_alloc_cap: workspace allocations above n_bytes fail with KG_ENOMEM (0 = off)."""
    _check(lib().kg_test_alloc_cap(int(n_bytes)))


def set_small_persistent(enable: bool):
    """kg_set_small_persistent: small instances run each 256 recursion steps in one
    cluster launch (True, the default) or one launch per step (False)."""
    _check(lib().kg_set_small_persistent(1 if enable else 0))


def ftm_dos_moments(h: Hamiltonian, phi, n_m: int, *, bessel_tol=1e-15, out=None):
    """kg_ftm_dos_moments -> complex [R][2 N_m + 1] (index n + N_m)."""
    r = _nvec(phi, h.n)
    run = _run(n_m, r, 1, KG_FP64, 1.0, bessel_tol)
    return _moments_call(lib().kg_ftm_dos_moments, h, phi, run, (r, 2 * n_m + 1), out)


def ftm_sum(f, energies_ev, emax_ev: float, area_nm2: float) -> np.ndarray:
    """kg_ftm_sum: f complex [..., 2 N_m + 1] -> [..., n_E] (Eqs. 22, 28)."""
    f = np.ascontiguousarray(f, dtype=np.complex128)
    lead, width = f.shape[:-1], f.shape[-1]
    e = np.ascontiguousarray(energies_ev, dtype=np.float64)
    sets = int(np.prod(lead)) if lead else 1
    out = np.zeros((sets, len(e)))
    _check(lib().kg_ftm_sum(f.ctypes.data, sets, (width - 1) // 2, e.ctypes.data, len(e), float(emax_ev),
                            float(area_nm2), out.ctypes.data))
    return out.reshape(*lead, len(e))


def apply(h: Hamiltonian, op: int, x, out):
    """kg_apply on device tensors x, out (complex128 [N] or [N][R])."""
    r = _nvec(x, h.n)
    _check(lib().kg_apply(h.handle, int(op), ctypes.c_void_p(x.data_ptr()),
                          ctypes.c_void_p(out.data_ptr()), r))
    return out


def evolve(h: Hamiltonian, dt: float, which: int, x, out, bessel_tol: float = 1e-15):
    """kg_evolve on device tensors x, out (complex128 [N] or [N][R])."""
    r = _nvec(x, h.n)
    _check(lib().kg_evolve(h.handle, float(dt), int(which), float(bessel_tol),
                           ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), r))
    return out


def _noalloc_args(idx_dev, onsite_dev, n_sites: int, phi_dev, mu_dev):
    """Checks the tensors of dos_moments_noalloc before any pointer reaches the
    library, which cannot see buffer sizes: a short or mistyped buffer there would be
    read or written out of bounds on the GPU.  Shapes and dtypes are checked first,
    then that every tensor is a contiguous CUDA tensor on the current device.
    Returns (R, M).  Raises ValueError."""
    import torch
    n = int(n_sites)
    if n < 1:
        raise ValueError("n_sites must be >= 1")
    if idx_dev.dtype != torch.int32 or tuple(idx_dev.shape) not in ((3, n), (3 * n,)):
        raise ValueError(f"idx_dev must be int32 [3][N] with N = {n}, got {idx_dev.dtype} {tuple(idx_dev.shape)}")
    if onsite_dev is not None and (onsite_dev.dtype != torch.float64 or tuple(onsite_dev.shape) != (n,)):
        raise ValueError(f"onsite_dev must be float64 [N] with N = {n}, got {onsite_dev.dtype} "
                         f"{tuple(onsite_dev.shape)}")
    if phi_dev.dtype != torch.complex128 or phi_dev.dim() not in (1, 2) or phi_dev.shape[0] != n:
        raise ValueError(f"phi_dev must be complex128 [N] or [N][R] with N = {n}, got {phi_dev.dtype} "
                         f"{tuple(phi_dev.shape)}")
    r = 1 if phi_dev.dim() == 1 else int(phi_dev.shape[1])
    if mu_dev.dtype != torch.complex128 or mu_dev.dim() != 2 or mu_dev.shape[0] != r or mu_dev.shape[1] < 1:
        raise ValueError(f"mu_dev must be complex128 [R][M] with R = {r} (the vectors of phi_dev), got "
                         f"{mu_dev.dtype} {tuple(mu_dev.shape)}")
    tensors = [("idx_dev", idx_dev), ("phi_dev", phi_dev), ("mu_dev", mu_dev)]
    if onsite_dev is not None:
        tensors.append(("onsite_dev", onsite_dev))
    for name, t in tensors:
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    dev = torch.cuda.current_device()
    for name, t in tensors:
        if t.device.index != dev:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{dev}")
    return r, int(mu_dev.shape[1])


# ----------------------------------------------------------------- seeded inputs

def splitmix64(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """kg_splitmix64: counter-mode SplitMix64 words x_start .. x_{start+count-1}."""
    out = np.zeros(int(count), dtype=np.uint64)
    _check(lib().kg_splitmix64(int(seed) % 2**64, int(stream) % 2**64, int(start), int(count),
                               ctypes.c_void_p(out.ctypes.data)))
    return out


def n_vacancies(n_sites: int, concentration: float) -> int:
    """kg_n_vacancies: round(n N), half to even."""
    v = ctypes.c_int64()
    _check(lib().kg_n_vacancies(int(n_sites), float(concentration), ctypes.byref(v)))
    return v.value


def vacancy_sites(n_sites: int, n_vac: int, seed: int) -> np.ndarray:
    """kg_vacancy_sites: n_vac distinct removed sites, sorted (int64)."""
    out = np.zeros(int(n_vac), dtype=np.int64)
    _check(lib().kg_vacancy_sites(int(n_sites), int(n_vac), int(seed) % 2**64,
                                  ctypes.c_void_p(out.ctypes.data)))
    return out


def anderson_onsite(n_sites: int, w_ev: float, seed: int) -> np.ndarray:
    """kg_anderson_onsite: eps_n = W (u_n - 1/2) eV."""
    out = np.zeros(int(n_sites), dtype=np.float64)
    _check(lib().kg_anderson_onsite(int(n_sites), float(w_ev), int(seed) % 2**64,
                                    ctypes.c_void_p(out.ctypes.data)))
    return out


def random_phase_vectors(n_sites: int, n_vec: int, seed: int, vacancies=None) -> np.ndarray:
    """kg_random_phase_vectors -> complex128 [N][R], zero on the removed sites."""
    vac = np.ascontiguousarray(np.zeros(0, dtype=np.int64) if vacancies is None else vacancies, dtype=np.int64)
    out = np.zeros((int(n_sites), int(n_vec)), dtype=np.complex128)
    _check(lib().kg_random_phase_vectors(int(n_sites), int(n_vec), int(seed) % 2**64,
                                         ctypes.c_void_p(vac.ctypes.data) if vac.size else None, int(vac.size),
                                         ctypes.c_void_p(out.ctypes.data)))
    return out


def fp64_fma_rate(repeats: int = 5) -> float:
    """kg_fp64_fma_rate: measured FP64 FMA instructions per second of the current
    device (best of ``repeats`` timed probe launches)."""
    v = ctypes.c_double()
    _check(lib().kg_fp64_fma_rate(int(repeats), ctypes.byref(v)))
    return v.value


def dos_moments_noalloc(idx_dev, onsite_dev, n_sites: int, hopping: float, phi_dev, mu_dev,
                        stream=None):
    """kg_dos_moments_noalloc on caller-owned device tensors (no device allocation).

    idx_dev int32 [3][N] (-1 = absent), onsite_dev float64 [N] (eps/E_max, 0 on removed
    sites) or None, phi_dev complex128 [N] or [N][R], mu_dev complex128 [R][M] (written).
    Every tensor must be contiguous and on the current CUDA device (ValueError
    otherwise)."""
    r, m = _noalloc_args(idx_dev, onsite_dev, n_sites, phi_dev, mu_dev)
    s = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
    _check(lib().kg_dos_moments_noalloc(
        ctypes.c_void_p(idx_dev.data_ptr()),
        None if onsite_dev is None else ctypes.c_void_p(onsite_dev.data_ptr()),
        int(n_sites), float(hopping), r, m, ctypes.c_void_p(phi_dev.data_ptr()),
        ctypes.c_void_p(mu_dev.data_ptr()), ctypes.c_void_p(s)))
    return mu_dev


def batched_dos_moments(hs, phis, n_moments: int, out=None):
    """kg_batched_dos_moments -> complex [n_h][R][M].  hs: list of Hamiltonian;
    phis: list of [N_i][R] complex128 (numpy or torch CUDA), same R for all."""
    n_h = len(hs)
    r = _nvec(phis[0], hs[0].n)
    keep = []
    ptrs = (ctypes.c_void_p * n_h)()
    for i, (h, p) in enumerate(zip(hs, phis)):
        if _nvec(p, h.n) != r:
            raise ValueError("all members need the same number of vectors")
        addr, k = _complex_in(p)
        keep.append(k)
        ptrs[i] = addr
    handles = (ctypes.c_void_p * n_h)(*[h.handle.value for h in hs])
    if out is None:
        res = np.zeros((n_h, r, n_moments), dtype=np.complex128)
        op = res.ctypes.data
    else:
        res = out
        op = out.data_ptr()
    run = _run(n_moments, r, 1, KG_FP64)
    _check(lib().kg_batched_dos_moments(handles, n_h, ctypes.byref(run), ptrs, ctypes.c_void_p(op)))
    return res


def batched_tuning() -> dict:
    """kg_batched_tuning: the autotuner's choice and its measurements."""
    bw, nc = ctypes.c_int(), ctypes.c_int()
    ms = ctypes.c_double()
    lw = (ctypes.c_int * 16)()
    lc = (ctypes.c_int * 16)()
    lm = (ctypes.c_double * 16)()
    _check(lib().kg_batched_tuning(ctypes.byref(bw), ctypes.byref(ms), ctypes.byref(nc), 16, lw, lc, lm))
    log = [(lw[k], lc[k], lm[k]) for k in range(16) if lw[k]]
    return {"block_width": bw.value, "ms_per_step": ms.value, "n_ctas": nc.value, "log": log}


def batched_release():
    _check(lib().kg_batched_release())


def batched_test_stall(cta: int):
    _check(lib().kg_batched_test_stall(int(cta)))


KG_MLP_PARAMS = 198657


def _f32(x):
    if _is_torch(x):
        import torch
        if x.dtype != torch.float32:
            raise ValueError("expected float32")
        return _ptr(x)
    return _ptr(np.ascontiguousarray(x, dtype=np.float32))


class Mlp:
    """Owns a ``kg_mlp*`` (surrogate network on the device)."""

    def __init__(self, params, stream=None):
        pp, keep = _f32(params)
        if (keep.numel() if _is_torch(keep) else keep.size) != KG_MLP_PARAMS:
            raise ValueError(f"expected {KG_MLP_PARAMS} parameters")
        s = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
        out = ctypes.c_void_p()
        _check(lib().kg_mlp_create(ctypes.c_void_p(pp), ctypes.c_void_p(s), ctypes.byref(out)))
        self._m = out

    def close(self):
        if self._m is not None and self._m.value:
            lib().kg_mlp_destroy(self._m)
        self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.zeros(KG_MLP_PARAMS, dtype=np.float32)
        _check(lib().kg_mlp_get_params(self._m, ctypes.c_void_p(out.ctypes.data)))
        return out

    def forward(self, x, out=None):
        """kg_mlp_forward: x [n][3] float32 -> y [n].  Device inputs and outputs are read and
        written in place by the kernel, so their dtype and size are checked here."""
        xp, kx = _f32(x)
        n = int(x.shape[0])
        if tuple(x.shape) != (n, 3):
            raise ValueError("x must have shape [n][3]")
        if out is None:
            res = np.zeros(n, dtype=np.float32)
            op = res.ctypes.data
        else:
            if _is_torch(out):
                import torch
                if out.dtype != torch.float32 or out.numel() < n:
                    raise ValueError("out must be a float32 tensor with at least n elements")
            elif np.asarray(out).dtype != np.float32 or np.asarray(out).size < n:
                raise ValueError("out must be a float32 array with at least n elements")
            res, op = out, _ptr(out, writable=True)[0]
        _check(lib().kg_mlp_forward(self._m, ctypes.c_void_p(xp), n, ctypes.c_void_p(op)))
        return res

    def gradients(self, x, t):
        """kg_mlp_gradients -> (loss, grad [KG_MLP_PARAMS])."""
        xp, kx = _f32(x)
        tp, kt = _f32(t)
        g = np.zeros(KG_MLP_PARAMS, dtype=np.float32)
        loss = ctypes.c_double()
        _check(lib().kg_mlp_gradients(self._m, ctypes.c_void_p(xp), ctypes.c_void_p(tp), int(x.shape[0]),
                                      ctypes.c_void_p(g.ctypes.data), ctypes.byref(loss)))
        return loss.value, g

    def train_step(self, x, t, lr: float) -> float:
        """kg_mlp_train_step (one Adam step) -> loss before the step."""
        xp, kx = _f32(x)
        tp, kt = _f32(t)
        loss = ctypes.c_double()
        _check(lib().kg_mlp_train_step(self._m, ctypes.c_void_p(xp), ctypes.c_void_p(tp), int(x.shape[0]),
                                       float(lr), ctypes.byref(loss)))
        return loss.value

    def launches(self) -> int:
        n = ctypes.c_int64()
        _check(lib().kg_mlp_launches(self._m, ctypes.byref(n)))
        return n.value

    def timing_enable(self, enable: bool = True):
        _check(lib().kg_mlp_timing_enable(self._m, 1 if enable else 0))

    def timing_read(self) -> dict:
        ms, n, fl = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
        _check(lib().kg_mlp_timing_read(self._m, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(fl)))
        return {"gemm_ms": ms.value, "gemm_launches": n.value, "gemm_flop": fl.value}


def mlp_gemm_test(a_dev, b_dev, out_dev):
    """kg_mlp_gemm_test: out [rows][256] fp32 = a [rows][k] bf16 @ b [256][k]^T (device tensors)."""
    rows, k = int(a_dev.shape[0]), int(a_dev.shape[1])
    _check(lib().kg_mlp_gemm_test(ctypes.c_void_p(a_dev.data_ptr()), ctypes.c_void_p(b_dev.data_ptr()),
                                  rows, k, ctypes.c_void_p(out_dev.data_ptr())))
    return out_dev


def timing_enable(h: Hamiltonian, enable: bool = True):
    _check(lib().kg_timing_enable(h.handle, 1 if enable else 0))


def timing_read(h: Hamiltonian) -> dict:
    t = _Timing()
    _check(lib().kg_timing_read(h.handle, ctypes.byref(t)))
    return {k: getattr(t, k) for k, _ in _Timing._fields_}


# ----------------------------------------------------------------- host helpers

def bessel_series(tau: float, tol: float = 1e-15, max_terms: int = 1000) -> np.ndarray:
    """kg_bessel_series -> J_m(tau), m < N_p."""
    j = np.zeros(max_terms)
    n = ctypes.c_int()
    _check(lib().kg_bessel_series(float(tau), float(tol), max_terms, j.ctypes.data, ctypes.byref(n)))
    return j[:n.value].copy()


def jackson(n_moments: int) -> np.ndarray:
    g = np.zeros(n_moments)
    _check(lib().kg_jackson(int(n_moments), g.ctypes.data))
    return g


def kpm_sum(mu, energies_ev, emax_ev: float, area_nm2: float) -> np.ndarray:
    """kg_kpm_sum: mu real [..., M] -> [..., n_E] (Eqs. 29-31)."""
    mu = np.ascontiguousarray(np.real(mu), dtype=np.float64)
    lead, m = mu.shape[:-1], mu.shape[-1]
    e = np.ascontiguousarray(energies_ev, dtype=np.float64)
    sets = int(np.prod(lead)) if lead else 1
    out = np.zeros((sets, len(e)))
    _check(lib().kg_kpm_sum(mu.ctypes.data, sets, m, e.ctypes.data, len(e), float(emax_ev),
                            float(area_nm2), out.ctypes.data))
    return out.reshape(*lead, len(e))


def conductivity(formula: int, density, dt_fs: float) -> np.ndarray:
    """kg_conductivity: density [N_c][n_E] -> sigma [N_c][n_E] in e^2/h."""
    d = np.ascontiguousarray(density, dtype=np.float64)
    out = np.zeros_like(d)
    _check(lib().kg_conductivity(int(formula), d.ctypes.data, d.shape[0], d.shape[1],
                                 float(dt_fs), out.ctypes.data))
    return out


def ballistic(rho, rho_dx2, dt_fs: float, width_nm: float):
    """kg_ballistic -> (L [N_c][n_E] nm, G [N_c][n_E] e^2/h)  (Eqs. 50-51)."""
    r = np.ascontiguousarray(rho, dtype=np.float64)
    d = np.ascontiguousarray(rho_dx2, dtype=np.float64)
    length = np.zeros_like(d)
    g = np.zeros_like(d)
    _check(lib().kg_ballistic(r.ctypes.data, d.ctypes.data, d.shape[0], d.shape[1], float(dt_fs),
                              float(width_nm), length.ctypes.data, g.ctypes.data))
    return length, g


def sigma_sc(sigma, dt_fs: float, t1_fs: float, t2_fs: float):
    """kg_sigma_sc -> (max over t > 0 [n_E], block average over [t1, t2] [n_E])  (Eqs. 53-54)."""
    s = np.ascontiguousarray(sigma, dtype=np.float64)
    mx = np.zeros(s.shape[1])
    av = np.zeros(s.shape[1])
    _check(lib().kg_sigma_sc(s.ctypes.data, s.shape[0], s.shape[1], float(dt_fs), float(t1_fs), float(t2_fs),
                             mx.ctypes.data, av.ctypes.data))
    return mx, av


def pade_fit(t, y, m: int = 2, n: int = 2, positive: bool = False) -> np.ndarray:
    """kg_pade_fit (or kg_pade_fit_positive: every b_k >= 0) -> (a_0..a_m, b_1..b_n)  (Eq. 58)."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    c = np.zeros(m + 1 + n)
    fn = lib().kg_pade_fit_positive if positive else lib().kg_pade_fit
    _check(fn(t.ctypes.data, y.ctypes.data, len(t), m, n, c.ctypes.data))
    return c


def pade_eval(coef, t, m: int = 2, n: int = 2):
    """kg_pade_eval -> (value, derivative) of the fitted approximant at t."""
    c = np.ascontiguousarray(coef, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    v = np.zeros(len(t))
    d = np.zeros(len(t))
    _check(lib().kg_pade_eval(c.ctypes.data, m, n, t.ctypes.data, len(t), v.ctypes.data, d.ctypes.data))
    return v, d
