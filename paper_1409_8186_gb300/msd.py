"""Thin Python binding of libmsd's C ABI (include/msd.h).

Functions named ``msd_*`` mirror the C entry points one to one and only
marshal arguments (NumPy arrays for host data, torch tensors for device
memory and the current CUDA stream).  ``Problem`` bundles the handle with
the geometry it was created from.  Every computation runs in the CUDA
library; if ``libmsd.so`` cannot be loaded this module raises at import.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libmsd.so")

MSD_OK = 0
MSD_NOT_CONVERGED = 1
MSD_STAGNATED = 3
MSD_ERR_ARG, MSD_ERR_OVERLAP, MSD_ERR_CUDA, MSD_ERR_OOM, MSD_ERR_NONFINITE, MSD_ERR_RANGE = -1, -2, -3, -4, -5, -6
MSD_DIRICHLET, MSD_NEUMANN = 0, 1
MSD_FP64, MSD_MIXED, MSD_FP32 = 0, 1, 2
MSD_GEN_AUTO, MSD_GEN_STREAMED, MSD_GEN_RECOMPUTE = 0, 1, 2
MSD_FORM_EFIE, MSD_FORM_MFIE, MSD_FORM_CFIE, MSD_FORM_BWIE = 0, 1, 2, 3
FORMULATION_KINDS = {"efie": MSD_FORM_EFIE, "mfie": MSD_FORM_MFIE, "cfie": MSD_FORM_CFIE, "bwie": MSD_FORM_BWIE}
MSD_MAX_N = 55
MSD_MAX_DORT = 2048

STATUS_NAMES = {0: "MSD_OK", 1: "MSD_NOT_CONVERGED", 3: "MSD_STAGNATED", -1: "MSD_ERR_ARG",
                -2: "MSD_ERR_OVERLAP", -3: "MSD_ERR_CUDA", -4: "MSD_ERR_OOM",
                -5: "MSD_ERR_NONFINITE", -6: "MSD_ERR_RANGE"}


class MsdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class msd_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int), ("maxit", ctypes.c_int),
                ("max_refine", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("precision", ctypes.c_int), ("gen_mode", ctypes.c_int), ("reorth", ctypes.c_double)]


class msd_stats(ctypes.Structure):
    _fields_ = [("flag", ctypes.c_int), ("iters", ctypes.c_int), ("refine_steps", ctypes.c_int),
                ("reserved", ctypes.c_int), ("relres", ctypes.c_double), ("true_relres", ctypes.c_double),
                ("solve_ms", ctypes.c_double)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libmsd.so not built ({_LIB_PATH}); run paper_1409_8186_gb300.build.build()")
    lib = ctypes.CDLL(_LIB_PATH)
    P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, None
    sig = {
        "msd_create": (I, [I, P, P, P, P, P, P, P, ctypes.POINTER(ctypes.c_void_p)]),
        "msd_destroy": (V, [P]),
        "msd_num_unknowns": (ctypes.c_int64, [P]),
        "msd_row_offset": (ctypes.c_int64, [P, I]),
        "msd_disk_diagonals": (I, [P, P]),
        "msd_pair_generators": (I, [P, I, P]),
        "msd_rhs_planewave": (I, [P, I, P, P]),
        "msd_matvec": (I, [P, I, I, P, P]),
        "msd_matvec_noalloc": (I, [P, I, I, P, P]),
        "msd_solve_planewaves": (I, [P, I, P, ctypes.POINTER(msd_opts), P, P]),
        "msd_farfield": (I, [P, P, I, I, P, P]),
        "msd_update_geometry": (I, [P, P, P, P]),
        "msd_grad_farfield_misfit": (I, [P, I, P, I, P, P, ctypes.POINTER(msd_opts), P, P, P, P]),
        "msd_matvec_timing": (I, [P, I, P, P, P, P]),
        "msd_plan_info": (I, [P, I, I, P, P]),
        "msd_set_tile": (I, [P, I, I, I, I]),
        "msd_set_generator_mode": (I, [P, I, ctypes.c_int64]),
        "msd_nearfield": (I, [P, I, P, I, ctypes.c_int64, P, P]),
        "msd_rhs_pointsource": (I, [P, I, P, P]),
        "msd_solve_pointsources": (I, [P, I, P, ctypes.POINTER(msd_opts), P, P]),
        "msd_dort": (I, [P, I, ctypes.POINTER(msd_opts), P, P, P, P]),
        "msd_dort_eigen": (I, [P, I, P, P, P]),
        "msd_set_formulation": (I, [P, P, P, P]),
        "msd_set_formulation_kind": (I, [P, I, D, P]),
        "msd_formulation_weights": (I, [I, D, P, D, P, P, P]),
        "msd_set_penetrable": (I, [P, P, P]),
        "msd_penetrable_matvec": (I, [P, I, I, P, P, P, P]),
        "msd_solve_penetrable": (I, [P, I, P, ctypes.POINTER(msd_opts), P, P, P]),
        "msd_solve_penetrable_pointsources": (I, [P, I, P, ctypes.POINTER(msd_opts), P, P, P]),
        "msd_kernel_launches": (ctypes.c_int64, []),
        "msd_test_expire_waits": (V, [I]),
        "msd_set_truncation": (I, [P, P]),
        "msd_penetrable_interior_field": (I, [P, I, P, I, ctypes.c_int64, P, P]),
        "msd_dort_eigenvectors": (I, [P, I, P, I, P, P]),
        "msd_herglotz_wave": (I, [P, I, I, I, P, ctypes.c_int64, P, P]),
        "msd_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()
EXPORTED = ("msd_create", "msd_destroy", "msd_num_unknowns", "msd_row_offset", "msd_disk_diagonals",
            "msd_pair_generators", "msd_rhs_planewave", "msd_matvec", "msd_solve_planewaves",
            "msd_farfield", "msd_update_geometry", "msd_matvec_timing", "msd_kernel_launches",
            "msd_matvec_noalloc", "msd_grad_farfield_misfit", "msd_plan_info", "msd_set_tile",
            "msd_set_generator_mode", "msd_nearfield", "msd_rhs_pointsource", "msd_solve_pointsources",
            "msd_dort", "msd_dort_eigen", "msd_set_formulation", "msd_set_formulation_kind",
            "msd_formulation_weights", "msd_test_expire_waits", "msd_set_truncation", "msd_penetrable_interior_field", "msd_dort_eigenvectors", "msd_herglotz_wave",
            "msd_set_penetrable",
            "msd_penetrable_matvec", "msd_solve_penetrable", "msd_solve_penetrable_pointsources",
            "msd_last_error")


def library_path() -> str:
    return _LIB_PATH


def _check(st: int, allow_positive: bool = False) -> int:
    if st < 0 or (st > 0 and not allow_positive):
        raise MsdError(st, msd_last_error())
    return st


def _ptr(a) -> int:
    """Address of a NumPy array or a torch tensor (host or device)."""
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


# ---------------------------------------------------------------- C entry points

def msd_last_error() -> str:
    return _lib.msd_last_error().decode()


def msd_create(disk_off, centres, radii, bc, k, N, stream=None) -> int:
    disk_off = np.ascontiguousarray(disk_off, dtype=np.int32)
    centres = np.ascontiguousarray(centres, dtype=np.float64)
    radii = np.ascontiguousarray(radii, dtype=np.float64)
    bc = np.ascontiguousarray(bc, dtype=np.int8)
    k = np.ascontiguousarray(k, dtype=np.float64)
    N = np.ascontiguousarray(N, dtype=np.int32)
    out = ctypes.c_void_p()
    _check(_lib.msd_create(len(k), _ptr(disk_off), _ptr(centres), _ptr(radii), _ptr(bc), _ptr(k),
                           _ptr(N), _stream_handle(stream), ctypes.byref(out)))
    return out.value


def msd_destroy(h) -> None:
    _lib.msd_destroy(h)


def msd_num_unknowns(h) -> int:
    return int(_lib.msd_num_unknowns(h))


def msd_row_offset(h, config: int) -> int:
    return int(_lib.msd_row_offset(h, config))


def msd_disk_diagonals(h, out) -> None:
    _check(_lib.msd_disk_diagonals(h, _ptr(out)))


def msd_pair_generators(h, config: int, out) -> None:
    _check(_lib.msd_pair_generators(h, config, _ptr(out)))


def msd_rhs_planewave(h, R: int, betas, out) -> None:
    betas = np.ascontiguousarray(betas, dtype=np.float64)
    _check(_lib.msd_rhs_planewave(h, R, _ptr(betas), _ptr(out)))


def msd_matvec(h, R: int, precision: int, x, y) -> None:
    _check(_lib.msd_matvec(h, R, precision, _ptr(x), _ptr(y)))


def msd_matvec_noalloc(h, R: int, precision: int, x, y) -> None:
    """msd_matvec without any device allocation in the call (work area in a
    fixed 32 MiB device array; see include/msd.h)."""
    _check(_lib.msd_matvec_noalloc(h, R, precision, _ptr(x), _ptr(y)))


def msd_solve_planewaves(h, R: int, betas, opts: msd_opts | None, rho_out, stats_out=None) -> int:
    betas = np.ascontiguousarray(betas, dtype=np.float64)
    return _check(_lib.msd_solve_planewaves(h, R, _ptr(betas), ctypes.byref(opts) if opts else None,
                                            _ptr(rho_out), ctypes.addressof(stats_out) if stats_out is not None else None),
                  allow_positive=True)


def msd_farfield(h, rho, R: int, thetas, F_out) -> None:
    thetas = np.ascontiguousarray(thetas, dtype=np.float64)
    _check(_lib.msd_farfield(h, _ptr(rho), R, len(thetas), _ptr(thetas), _ptr(F_out)))


def msd_update_geometry(h, centres=None, radii=None, k=None) -> None:
    def arg(a):
        if a is None:
            return None
        return a if hasattr(a, "data_ptr") else np.ascontiguousarray(a, dtype=np.float64)
    c, r, kk = arg(centres), arg(radii), arg(k)
    _check(_lib.msd_update_geometry(h, _ptr(c) if c is not None else None,
                                    _ptr(r) if r is not None else None,
                                    _ptr(kk) if kk is not None else None))


def msd_grad_farfield_misfit(h, R: int, betas, thetas, F_target, opts: msd_opts | None, J_out=None, dO=None,
                             da=None, dk=None) -> int:
    betas = np.ascontiguousarray(betas, dtype=np.float64)
    thetas = np.ascontiguousarray(thetas, dtype=np.float64)
    if not hasattr(F_target, "data_ptr"):
        F_target = np.ascontiguousarray(F_target, dtype=np.complex128)
    p = lambda a: _ptr(a) if a is not None else None  # noqa: E731
    return _check(_lib.msd_grad_farfield_misfit(h, R, _ptr(betas), len(thetas), _ptr(thetas), _ptr(F_target),
                                                ctypes.byref(opts) if opts else None, p(J_out), p(dO), p(da),
                                                p(dk)), allow_positive=True)


def msd_matvec_timing(h, enable: int):
    """Returns (kernel_ms, launches, flops, bytes) accumulated since the last start."""
    ms, n = ctypes.c_double(), ctypes.c_int64()
    fl, by = ctypes.c_double(), ctypes.c_double()
    _check(_lib.msd_matvec_timing(h, enable, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(fl),
                                  ctypes.byref(by)))
    return ms.value, n.value, fl.value, by.value


def msd_plan_info(h, R: int, precision: int):
    """Returns ({"KB", "RT", "nsplit", "candidates"}, tuned_ms) of the product plan for (R, precision)."""
    out = (ctypes.c_int * 4)()
    ms = ctypes.c_double()
    _check(_lib.msd_plan_info(h, R, precision, out, ctypes.byref(ms)))
    return {"KB": out[0], "RT": out[1], "nsplit": out[2], "candidates": out[3]}, ms.value


def msd_set_tile(h, R: int, precision: int, KB: int, RT: int) -> None:
    _check(_lib.msd_set_tile(h, R, precision, KB, RT))


def msd_set_generator_mode(h, mode: int, chunk_bytes: int = 0) -> None:
    _check(_lib.msd_set_generator_mode(h, mode, chunk_bytes))


def msd_rhs_pointsource(h, R: int, sources, out) -> None:
    src = np.ascontiguousarray(sources, dtype=np.float64)
    _check(_lib.msd_rhs_pointsource(h, R, _ptr(src), _ptr(out)))


def msd_solve_pointsources(h, R: int, sources, opts: msd_opts | None, rho_out, stats_out=None) -> int:
    src = np.ascontiguousarray(sources, dtype=np.float64)
    return _check(_lib.msd_solve_pointsources(h, R, _ptr(src), ctypes.byref(opts) if opts else None, _ptr(rho_out),
                                              ctypes.addressof(stats_out) if stats_out is not None else None),
                  allow_positive=True)


def msd_nearfield(h, config: int, rho, R: int, points, u_out) -> None:
    pts = points if hasattr(points, "data_ptr") else np.ascontiguousarray(points, dtype=np.float64)
    _check(_lib.msd_nearfield(h, config, _ptr(rho), R, int(pts.shape[0]), _ptr(pts), _ptr(u_out)))


def msd_dort(h, n_alpha: int, opts: msd_opts | None, F_out, T_out, eig_out, stats_out=None) -> int:
    p = lambda a: _ptr(a) if a is not None else None  # noqa: E731
    return _check(_lib.msd_dort(h, n_alpha, ctypes.byref(opts) if opts else None, p(F_out), p(T_out), _ptr(eig_out),
                                ctypes.addressof(stats_out) if stats_out is not None else None),
                  allow_positive=True)


def msd_dort_eigen(h, n_alpha: int, F, T_out, eig_out) -> None:
    if not hasattr(F, "data_ptr"):
        F = np.ascontiguousarray(F, dtype=np.complex128)
    _check(_lib.msd_dort_eigen(h, n_alpha, _ptr(F), _ptr(T_out) if T_out is not None else None, _ptr(eig_out)))


def msd_set_formulation(h, op_weights, rhs_weights, rep_weights) -> None:
    """op_weights complex [2][5] (I, L, M, N, D per boundary condition),
    rhs_weights complex [2][2] (U, dU), rep_weights complex [2] (L, M);
    op_weights None restores the default rows."""
    if op_weights is None:
        _check(_lib.msd_set_formulation(h, None, None, None))
        return
    ow = np.ascontiguousarray(np.asarray(op_weights, np.complex128).reshape(2, 5)).view(np.float64)
    rw = np.ascontiguousarray(np.asarray(rhs_weights, np.complex128).reshape(2, 2)).view(np.float64)
    pw = np.ascontiguousarray(np.asarray(rep_weights, np.complex128).reshape(2)).view(np.float64)
    _check(_lib.msd_set_formulation(h, _ptr(ow), _ptr(rw), _ptr(pw)))


def msd_set_penetrable(h, k_minus, mu=None) -> None:
    if k_minus is None:
        _check(_lib.msd_set_penetrable(h, None, None))
        return
    km = np.ascontiguousarray(np.atleast_1d(k_minus), dtype=np.float64)
    m = None if mu is None else np.ascontiguousarray(mu, dtype=np.float64)
    _check(_lib.msd_set_penetrable(h, _ptr(km), _ptr(m) if m is not None else None))


def msd_penetrable_matvec(h, R: int, precision: int, xp, xm, yp, ym) -> None:
    _check(_lib.msd_penetrable_matvec(h, R, precision, _ptr(xp), _ptr(xm), _ptr(yp), _ptr(ym)))


def msd_solve_penetrable(h, R: int, betas, opts: msd_opts | None, rho_plus, rho_minus, stats_out=None) -> int:
    b = np.ascontiguousarray(betas, dtype=np.float64)
    return _check(_lib.msd_solve_penetrable(h, R, _ptr(b), ctypes.byref(opts) if opts else None, _ptr(rho_plus),
                                            _ptr(rho_minus), ctypes.addressof(stats_out) if stats_out is not None
                                            else None), allow_positive=True)


def msd_solve_penetrable_pointsources(h, R: int, sources, opts: msd_opts | None, rho_plus, rho_minus,
                                      stats_out=None) -> int:
    src = np.ascontiguousarray(sources, dtype=np.float64)
    return _check(_lib.msd_solve_penetrable_pointsources(h, R, _ptr(src), ctypes.byref(opts) if opts else None,
                                                         _ptr(rho_plus), _ptr(rho_minus),
                                                         ctypes.addressof(stats_out) if stats_out is not None
                                                         else None), allow_positive=True)


def _eta_arg(eta):
    if eta is None:
        return None
    e = complex(eta)
    return np.array([e.real, e.imag], np.float64)


def _kind(kind) -> int:
    if kind not in FORMULATION_KINDS:
        raise ValueError(f"unknown formulation {kind!r}; one of {sorted(FORMULATION_KINDS)}")
    return FORMULATION_KINDS[kind]


def msd_set_formulation_kind(h, kind: str, alpha: float = 0.5, eta=None) -> None:
    """kind "efie", "mfie", "cfie" or "bwie"; eta None means i k of each
    configuration (include/msd.h)."""
    e = _eta_arg(eta)
    _check(_lib.msd_set_formulation_kind(h, _kind(kind), float(alpha), _ptr(e) if e is not None else None))


def msd_formulation_weights(kind: str, alpha: float = 0.5, eta=None, k: float = 0.0):
    """The library's weights of a named formulation: (op [2][5], rhs [2][2],
    rep [2]) complex, the layout of msd_set_formulation."""
    e = _eta_arg(eta)
    op = np.zeros((2, 5), np.complex128)
    rhs = np.zeros((2, 2), np.complex128)
    rep = np.zeros(2, np.complex128)
    _check(_lib.msd_formulation_weights(_kind(kind), float(alpha), _ptr(e) if e is not None else None,
                                        float(k), _ptr(op), _ptr(rhs), _ptr(rep)))
    return op, rhs, rep


def formulation(kind: str, alpha: float = 0.5, eta=None, k: float | None = None):
    """Weights (op [2][5], rhs [2][2], rep [2]) of a standard formulation
    (section 3), formed by the library (msd_formulation_weights); eta
    defaults to i k."""
    if eta is None and kind in ("cfie", "bwie") and k is None:
        raise ValueError("eta or k is needed")
    return msd_formulation_weights(kind, alpha, eta, 0.0 if k is None else k)


def msd_kernel_launches() -> int:
    return int(_lib.msd_kernel_launches())


def msd_penetrable_interior_field(h, config: int, rho_minus, R: int, points, u_out) -> None:
    pts = points if hasattr(points, "data_ptr") else np.ascontiguousarray(points, dtype=np.float64)
    _check(_lib.msd_penetrable_interior_field(h, config, _ptr(rho_minus), R, len(pts), _ptr(pts), _ptr(u_out)))


def msd_dort_eigenvectors(h, n_alpha: int, F, K: int, eig_out, vec_out) -> None:
    if not hasattr(F, "data_ptr"):
        F = np.ascontiguousarray(F, dtype=np.complex128)
    _check(_lib.msd_dort_eigenvectors(h, n_alpha, _ptr(F), K, _ptr(eig_out) if eig_out is not None else None,
                                      _ptr(vec_out)))


def msd_herglotz_wave(h, config: int, n_alpha: int, K: int, g, points, u_out) -> None:
    if not hasattr(g, "data_ptr"):
        g = np.ascontiguousarray(g, dtype=np.complex128)
    pts = points if hasattr(points, "data_ptr") else np.ascontiguousarray(points, dtype=np.float64)
    _check(_lib.msd_herglotz_wave(h, config, n_alpha, K, _ptr(g), len(pts), _ptr(pts), _ptr(u_out)))


def msd_set_truncation(h, Np) -> None:
    """Per-disk truncation orders N_p (host int [disk_off[C]]); None restores N."""
    if Np is None:
        _check(_lib.msd_set_truncation(h, None))
        return
    arr = np.ascontiguousarray(Np, dtype=np.int32)
    _check(_lib.msd_set_truncation(h, _ptr(arr)))


def msd_test_expire_waits(on: bool) -> None:
    """Test hook: bounded device waits take their expiry path (include/msd.h)."""
    _lib.msd_test_expire_waits(1 if on else 0)


# ---------------------------------------------------------------- convenience wrapper

@dataclass
class SolveResult:
    rho: object          # torch complex128 [N_tot, R] (device) or numpy (host)
    status: int
    flags: np.ndarray
    iters: np.ndarray
    refine_steps: np.ndarray
    relres: np.ndarray
    true_relres: np.ndarray = None   # ||b - A rho|| / ||b|| (unpreconditioned); -1 where not computed
    solve_ms: float = 0.0


class Problem:
    """A batch of clusters (objects with centres, radii, bc, k, N) on the GPU."""

    def __init__(self, clusters, stream=None):
        if not isinstance(clusters, (list, tuple)):
            clusters = [clusters]
        self.clusters = list(clusters)
        Ms = [len(c.radii) for c in self.clusters]
        self.disk_off = np.concatenate([[0], np.cumsum(Ms)]).astype(np.int32)
        cen = np.concatenate([np.asarray(c.centres, np.float64) for c in self.clusters])
        rad = np.concatenate([np.asarray(c.radii, np.float64) for c in self.clusters])
        bc = np.concatenate([np.asarray(c.bc, np.int8) for c in self.clusters])
        k = np.array([c.k for c in self.clusters], np.float64)
        N = np.array([c.N for c in self.clusters], np.int32)
        self.C = len(self.clusters)
        self.handle = msd_create(self.disk_off, cen, rad, bc, k, N, stream)
        self.ntot = msd_num_unknowns(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            msd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def row_offset(self, c: int) -> int:
        return msd_row_offset(self.handle, c)

    def _betas(self, betas):
        b = np.asarray(betas, np.float64)
        if b.ndim == 1:
            b = np.broadcast_to(b, (self.C, b.shape[0]))
        return np.ascontiguousarray(b)

    def diagonals(self):
        import torch
        out = torch.empty((4, self.ntot), dtype=torch.complex128, device="cuda")
        msd_disk_diagonals(self.handle, out)
        return out

    def generators(self, c: int = 0):
        import torch
        cl = self.clusters[c]
        M, L = len(cl.radii), 4 * cl.N + 1
        out = torch.empty((M, M, L), dtype=torch.complex128, device="cuda")
        msd_pair_generators(self.handle, c, out)
        return out

    def rhs(self, betas):
        import torch
        b = self._betas(betas)
        out = torch.empty((self.ntot, b.shape[1]), dtype=torch.complex128, device="cuda")
        msd_rhs_planewave(self.handle, b.shape[1], b, out)
        return out

    def matvec(self, x, precision: int = MSD_FP64, out=None):
        import torch
        R = x.shape[1] if x.dim() == 2 else 1
        want = torch.complex128 if precision == MSD_FP64 else torch.complex64
        if x.dtype != want or not x.is_contiguous() or not x.is_cuda:
            raise ValueError(f"x must be a contiguous CUDA {want} tensor of shape [N_tot, R]")
        y = torch.empty_like(x) if out is None else out
        msd_matvec(self.handle, R, precision, x, y)
        return y

    def plan_info(self, R: int, precision: int = MSD_FP64):
        return msd_plan_info(self.handle, R, precision)

    def set_tile(self, R: int, precision: int, KB: int, RT: int) -> None:
        msd_set_tile(self.handle, R, precision, KB, RT)

    def set_generator_mode(self, mode: int, chunk_bytes: int = 0) -> None:
        msd_set_generator_mode(self.handle, mode, chunk_bytes)

    def solve(self, betas, tol=1e-10, restart=0, maxit=3000, precision=MSD_FP64, max_refine=0,
              inner_tol=0.0, out=None, gen_mode=MSD_GEN_AUTO, reorth=0.0) -> SolveResult:
        import torch
        b = self._betas(betas)
        R = b.shape[1]
        o = msd_opts(tol, restart, maxit, max_refine, inner_tol, precision, gen_mode, reorth)
        rho = torch.empty((self.ntot, R), dtype=torch.complex128, device="cuda") if out is None else out
        stats = (msd_stats * (self.C * R))()
        st = msd_solve_planewaves(self.handle, R, b, o, rho, stats)
        return SolveResult(rho, st, np.array([s.flag for s in stats]), np.array([s.iters for s in stats]),
                           np.array([s.refine_steps for s in stats]), np.array([s.relres for s in stats]),
                           np.array([s.true_relres for s in stats]), float(stats[0].solve_ms) if len(stats) else 0.0)

    def farfield(self, rho, thetas, out=None):
        import torch
        th = np.ascontiguousarray(thetas, np.float64)
        R = rho.shape[1]
        F = torch.empty((self.C, len(th), R), dtype=torch.complex128, device="cuda") if out is None else out
        msd_farfield(self.handle, rho, R, th, F)
        return F

    def _sources(self, sources):
        src = np.asarray(sources, dtype=np.float64)
        if src.ndim == 2:  # [R, 2] shared by every configuration
            src = np.broadcast_to(src, (self.C,) + src.shape)
        return np.ascontiguousarray(src)

    def rhs_pointsource(self, sources):
        import torch
        src = self._sources(sources)
        out = torch.empty((self.ntot, src.shape[1]), dtype=torch.complex128, device="cuda")
        msd_rhs_pointsource(self.handle, src.shape[1], src, out)
        return out

    def solve_pointsources(self, sources, tol=1e-10, restart=0, maxit=3000, precision=MSD_FP64,
                           out=None) -> SolveResult:
        import torch
        src = self._sources(sources)
        R = src.shape[1]
        o = msd_opts(tol, restart, maxit, 0, 0.0, precision, MSD_GEN_AUTO)
        rho = torch.empty((self.ntot, R), dtype=torch.complex128, device="cuda") if out is None else out
        stats = (msd_stats * (self.C * R))()
        st = msd_solve_pointsources(self.handle, R, src, o, rho, stats)
        return SolveResult(rho, st, np.array([s.flag for s in stats]), np.array([s.iters for s in stats]),
                           np.array([s.refine_steps for s in stats]), np.array([s.relres for s in stats]),
                           np.array([s.true_relres for s in stats]), float(stats[0].solve_ms) if len(stats) else 0.0)

    def nearfield(self, rho, points, config: int = 0, out=None):
        """Scattered field at points [P, 2] outside the disks of `config`
        (complex128 [P, R] on the device; 0 inside a disk)."""
        import torch
        R = rho.shape[1]
        pts = np.ascontiguousarray(points, dtype=np.float64)
        u = torch.empty((pts.shape[0], R), dtype=torch.complex128, device="cuda") if out is None else out
        msd_nearfield(self.handle, config, rho, R, pts, u)
        return u

    def interior_field(self, rho_minus, points, config: int = 0, out=None):
        """Penetrable obstacles: u- = L- rho- at points [P, 2] inside the disks
        of `config` (complex128 [P, R] on the device; 0 outside every disk)."""
        import torch
        R = rho_minus.shape[1]
        pts = np.ascontiguousarray(points, dtype=np.float64)
        u = torch.empty((pts.shape[0], R), dtype=torch.complex128, device="cuda") if out is None else out
        msd_penetrable_interior_field(self.handle, config, rho_minus, R, pts, u)
        return u

    def dort(self, n_alpha: int, tol=1e-12, precision=MSD_FP64, restart=0, maxit=3000, want_F=True,
             want_T=True):
        """Time reversal (section 7): returns (eig [C, n_alpha] largest first,
        F [C, n_alpha, n_alpha] or None, T [C, n_alpha, n_alpha] or None,
        status), device tensors."""
        import torch
        o = msd_opts(tol, restart, maxit, 0, 0.0, precision, MSD_GEN_AUTO)
        shape = (self.C, n_alpha, n_alpha)
        F = torch.empty(shape, dtype=torch.complex128, device="cuda") if want_F else None
        T = torch.empty(shape, dtype=torch.complex128, device="cuda") if want_T else None
        eig = torch.empty((self.C, n_alpha), dtype=torch.float64, device="cuda")
        st = msd_dort(self.handle, n_alpha, o, F, T, eig)
        return eig, F, T, st

    def set_formulation(self, kind=None, **kw):
        """Use a standard formulation ("efie", "mfie", "cfie", "bwie"; see
        formulation()), explicit weights (op=, rhs=, rep=), or the default
        rows (kind None)."""
        if kind is None and "op" not in kw:
            msd_set_formulation(self.handle, None, None, None)
        elif kind is None:
            msd_set_formulation(self.handle, kw["op"], kw["rhs"], kw["rep"])
        else:
            kw.pop("k", None)      # eta = i k of each configuration is the library's default
            msd_set_formulation_kind(self.handle, kind, **kw)

    def set_penetrable(self, k_minus, mu=None):
        """Penetrable obstacles (section 7): interior wavenumber(s) k_minus
        (scalar or [C]) and per-disk contrasts mu (None: 1); k_minus None
        switches back to sound-soft/sound-hard disks."""
        if k_minus is not None:
            k_minus = np.broadcast_to(np.asarray(k_minus, np.float64), (self.C,))
        msd_set_penetrable(self.handle, k_minus, mu)

    def penetrable_matvec(self, xp, xm):
        """(y+, y-) = B^-1 A (x+, x-) of the transmission system (FP64)."""
        R = xp.shape[1] if xp.dim() == 2 else 1
        yp, ym = xp.new_empty(xp.shape), xm.new_empty(xm.shape)
        msd_penetrable_matvec(self.handle, R, MSD_FP64, xp, xm, yp, ym)
        return yp, ym

    def solve_penetrable(self, betas=None, tol=1e-10, restart=0, maxit=3000, precision=MSD_FP64, sources=None):
        """Plane waves (betas) or point sources ([R, 2] or [C, R, 2]).
        Returns (rho_plus, rho_minus, SolveResult); the exterior field is
        farfield / nearfield of rho_plus."""
        import torch
        if sources is not None:
            b = self._sources(sources)
        else:
            b = self._betas(betas)
        R = b.shape[1]
        o = msd_opts(tol, restart, maxit, 0, 0.0, precision, MSD_GEN_AUTO)
        rp = torch.empty((self.ntot, R), dtype=torch.complex128, device="cuda")
        rm = torch.empty_like(rp)
        stats = (msd_stats * (self.C * R))()
        if sources is not None:
            st = msd_solve_penetrable_pointsources(self.handle, R, b, o, rp, rm, stats)
        else:
            st = msd_solve_penetrable(self.handle, R, b, o, rp, rm, stats)
        res = SolveResult(rp, st, np.array([s.flag for s in stats]), np.array([s.iters for s in stats]),
                          np.array([s.refine_steps for s in stats]), np.array([s.relres for s in stats]),
                          np.array([s.true_relres for s in stats]), float(stats[0].solve_ms) if len(stats) else 0.0)
        return rp, rm, res

    def dort_eigen(self, F, want_T=False):
        """T = conj(F)^T F and its eigenvalues (largest first) for caller
        far-field matrices F [C, n, n]; returns (eig, T or None)."""
        import torch
        n = F.shape[-1]
        T = torch.empty((self.C, n, n), dtype=torch.complex128, device="cuda") if want_T else None
        eig = torch.empty((self.C, n), dtype=torch.float64, device="cuda")
        msd_dort_eigen(self.handle, n, F, T, eig)
        return eig, T

    def dort_eigenvectors(self, F, K: int):
        """Eigenvalues [C, n] and the eigenvectors [C, K, n] of the K largest
        eigenvalues of T = conj(F)^T F, for far-field matrices F [C, n, n]."""
        import torch
        n = F.shape[-1]
        eig = torch.empty((self.C, n), dtype=torch.float64, device="cuda")
        vec = torch.empty((self.C, K, n), dtype=torch.complex128, device="cuda")
        msd_dort_eigenvectors(self.handle, n, F, K, eig, vec)
        return eig, vec

    def herglotz_wave(self, g, points, config: int = 0):
        """Discrete Herglotz waves of parameter vectors g [K, n_alpha] at points
        [P, 2] (complex128 [P, K] on the device)."""
        import torch
        g = g if hasattr(g, "data_ptr") else np.ascontiguousarray(g, dtype=np.complex128)
        K, na = g.shape
        pts = np.ascontiguousarray(points, dtype=np.float64)
        u = torch.empty((pts.shape[0], K), dtype=torch.complex128, device="cuda")
        msd_herglotz_wave(self.handle, config, na, K, g, pts, u)
        return u

    def update_geometry(self, centres=None, radii=None, k=None):
        msd_update_geometry(self.handle, centres, radii, k)

    def set_truncation(self, Np=None):
        """Per-disk truncation orders N_p <= N (None: N on every disk)."""
        msd_set_truncation(self.handle, Np)

    def grad_farfield_misfit(self, betas, thetas, F_target, tol=1e-12, precision=MSD_FP64, restart=0,
                             maxit=3000):
        """J [C], dJ/dO [sum M, 2], dJ/da [sum M], dJ/dk [C] (NumPy arrays)."""
        b = self._betas(betas)
        Mtot = int(self.disk_off[-1])
        J = np.zeros(self.C)
        dO = np.zeros((Mtot, 2))
        da = np.zeros(Mtot)
        dk = np.zeros(self.C)
        o = msd_opts(tol, restart, maxit, 0, 0.0, precision, MSD_GEN_AUTO)
        st = msd_grad_farfield_misfit(self.handle, b.shape[1], b, np.asarray(thetas, np.float64), F_target, o, J,
                                      dO, da, dk)
        if st != MSD_OK:
            raise MsdError(st, "a solve of the gradient did not converge")
        return J, dO, da, dk


def _autograd_function():
    import torch

    class FarFieldMisfit(torch.autograd.Function):
        """J = sum_c sum_{t,r} |F - F*|^2 as a differentiable function of the
        centres [sum M, 2], radii [sum M] and wavenumbers [C] (float64
        tensors), evaluated by the CUDA library: the forward pass runs the
        solve and the adjoint solve, the backward pass scales the stored
        gradients."""

        @staticmethod
        def forward(ctx, centres, radii, k, problem, betas, thetas, F_target, tol, precision):
            problem.update_geometry(centres.detach().contiguous().cpu().numpy(),
                                    radii.detach().contiguous().cpu().numpy(),
                                    k.detach().contiguous().cpu().numpy())
            J, dO, da, dk = problem.grad_farfield_misfit(betas, thetas, F_target, tol=tol, precision=precision)
            dev = centres.device
            ctx.save_for_backward(torch.from_numpy(dO).to(dev), torch.from_numpy(da).to(dev),
                                  torch.from_numpy(dk).to(dev))
            return torch.tensor(float(J.sum()), dtype=torch.float64, device=dev)

        @staticmethod
        def backward(ctx, gJ):
            dO, da, dk = ctx.saved_tensors
            return gJ * dO, gJ * da, gJ * dk, None, None, None, None, None, None

    return FarFieldMisfit


def farfield_misfit(problem, centres, radii, k, betas, thetas, F_target, tol=1e-12, precision=MSD_FP64):
    """Differentiable far-field misfit (torch.autograd), see FarFieldMisfit."""
    return _autograd_function().apply(centres, radii, k, problem, betas, thetas, F_target, tol, precision)
