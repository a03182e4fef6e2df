"""Thin ctypes binding of libnsstab.so (C ABI in include/nsstab.h).

Argument marshalling only: every step of the method runs in the library.
Device fields are ``torch.Tensor`` objects (CUDA, float64, contiguous,
shape ``[ny, nx]``); PyTorch supplies the device memory and the stream.  The
functions carry the C names; ``Stepper`` is a convenience owner of a
``nsstab_stepper*``.  There is no CPU fallback: if the library is missing
or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libnsstab.so")

OK = 0
NOT_CONVERGED = 1
DIVERGED = 2

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_long)


class Config(ctypes.Structure):
    """Mirror of ``nsstab_config``."""

    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("Lx", ctypes.c_double), ("Ly", ctypes.c_double),
        ("dt", ctypes.c_double), ("Re", ctypes.c_double), ("Uinf", ctypes.c_double),
        ("cyl_x", ctypes.c_double), ("cyl_y", ctypes.c_double), ("cyl_D", ctypes.c_double),
        ("eta", ctypes.c_double), ("mask_cells", ctypes.c_double),
        ("sponge_frac", ctypes.c_double), ("sponge_sigma", ctypes.c_double),
        ("precision", ctypes.c_int),
    ]


SERVE_MAX_EIG = 33   # NSSTAB_SERVE_MAX_EIG


class EigJob(ctypes.Structure):
    """Mirror of ``nsstab_eig_job``."""

    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("dt", ctypes.c_double), ("Re", ctypes.c_double), ("cyl_D", ctypes.c_double),
        ("base", ctypes.c_void_p), ("v0", ctypes.c_void_p),
    ]


class EigJobResult(ctypes.Structure):
    """Mirror of ``nsstab_eig_result``."""

    _fields_ = [
        ("status", ctypes.c_int), ("n_eig", ctypes.c_int), ("n_conv", ctypes.c_int), ("n_matvec", ctypes.c_int),
        ("group", ctypes.c_int), ("latency_s", ctypes.c_double),
        ("eig_re", ctypes.c_double * SERVE_MAX_EIG), ("eig_im", ctypes.c_double * SERVE_MAX_EIG),
        ("resid", ctypes.c_double * SERVE_MAX_EIG),
    ]


# (name, restype, argtypes) of every exported symbol declared in nsstab.h
SIGNATURES = [
    ("nsstab_config_default", None, [ctypes.POINTER(Config)]),
    ("stepper_create", ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    ("batch_create", ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_int, _dp, _dp, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.POINTER(ctypes.c_void_p)]),
    ("stepper_members", ctypes.c_int, [ctypes.c_void_p, _ip, _ip]),
    ("stepper_destroy", None, [ctypes.c_void_p]),
    ("stepper_poisson", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("step_nonlinear", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("stepper_set_base", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("apply_expTL", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double]),
    ("stepper_residual", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, _dp]),
    ("sfd_baseflow", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_long, ctypes.c_int, _dp, _lp]),
    ("newton_krylov_fixedpoint", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                                ctypes.c_double, ctypes.c_int, _dp, _ip, _ip]),
    ("newton_krylov_fixedpoint_ex", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                   ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                                   ctypes.c_double, ctypes.c_int, ctypes.c_int, _dp, _ip, _ip]),
    ("apply_tangent", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_double]),
    ("arnoldi_eigs", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_double, _dp, _dp, _dp,
                                    ctypes.c_void_p, _ip, _ip, _ip]),
    ("batch_arnoldi_eigs", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double, _dp, _dp,
                                          _dp, ctypes.c_void_p, _ip, _ip, _ip]),
    ("stepper_profile_linear", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, _dp]),
    ("stepper_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _ip]),
    ("stepper_set_plan", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    ("stepper_get_plan", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _ip, _ip]),
    ("stepper_set_fused_rows", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("stepper_get_fused_rows", ctypes.c_int, [ctypes.c_void_p, _ip]),
    ("block_arnoldi_eigs", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double, _dp, _dp,
                                          _dp, ctypes.c_void_p, _ip, _ip, _ip]),
    ("serve_eigs_persistent", ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_int, ctypes.POINTER(EigJob),
                                             ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                             ctypes.c_double, ctypes.c_longlong, ctypes.POINTER(EigJobResult), _ip]),
    ("serve_eigs", ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_int, ctypes.POINTER(EigJob), ctypes.c_int,
                                  ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_longlong,
                                  ctypes.c_int, ctypes.POINTER(EigJobResult), _ip]),
    ("unet_param_count", ctypes.c_long, [ctypes.c_int, ctypes.c_int]),
    ("unet_create", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    ("unet_destroy", None, [ctypes.c_void_p]),
    ("unet_set_params", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("unet_get_params", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("unet_forward", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("unet_gradient", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_void_p, _dp]),
    ("unet_train_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _dp]),
    ("cgs2_orthogonalize", ctypes.c_int, [ctypes.c_void_p, ctypes.c_long, ctypes.c_long, ctypes.c_int,
                                          ctypes.c_void_p, _dp, _dp, ctypes.c_void_p]),
    ("cgs2_orthogonalize_noalloc", ctypes.c_int, [ctypes.c_void_p, ctypes.c_long, ctypes.c_long, ctypes.c_int,
                                                  ctypes.c_void_p, _dp, _dp, ctypes.c_void_p]),
    ("nsstab_dense_eig", ctypes.c_int, [ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp, _dp]),
    ("nsstab_dense_schur_ordered", ctypes.c_int, [ctypes.c_int, _dp, ctypes.c_double, _dp, _dp, _ip]),
    ("nsstab_last_error", ctypes.c_char_p, []),
]

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libnsstab.so (build it with ``__graft_entry__.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} not found: build the CUDA library first (__graft_entry__.build())")
        lib = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class NsstabError(RuntimeError):
    pass


def _check(rc: int, what: str, allow_soft: bool = False) -> int:
    if rc < 0 or (rc > 0 and not allow_soft):
        msg = load_library().nsstab_last_error().decode(errors="replace")
        raise NsstabError(f"{what} failed with status {rc}: {msg}")
    return rc


def _field_ptr(t, shape, name):
    import torch

    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.device.type != "cuda" or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    if tuple(t.shape[-2:]) != tuple(shape) or t.numel() % (shape[0] * shape[1]) != 0:
        raise ValueError(f"{name} must have shape {shape}")
    return ctypes.c_void_p(t.data_ptr())


def _cfg_from(**kw) -> Config:
    cfg = Config()
    load_library().nsstab_config_default(ctypes.byref(cfg))
    for k, v in kw.items():
        if not hasattr(cfg, k):
            raise KeyError(k)
        setattr(cfg, k, v)
    return cfg


def config_default() -> Config:
    return _cfg_from()


def current_stream_handle():
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


# ------------------------------------------------ C-named thin wrappers

def stepper_create(cfg: Config, stream=None) -> ctypes.c_void_p:
    lib = load_library()
    h = ctypes.c_void_p()
    s = current_stream_handle() if stream is None else ctypes.c_void_p(stream)
    _check(lib.stepper_create(ctypes.byref(cfg), s, ctypes.byref(h)), "stepper_create")
    return h


def stepper_destroy(h) -> None:
    load_library().stepper_destroy(h)


def _gs_args(V, n: int, j: int, w, ldv):
    """Check the device tensors of a CGS2 call against the sizes the kernels
    will touch (V: j columns of length n, leading dimension ldv; w: n)."""
    import torch

    if w.dtype != torch.float64 or w.device.type != "cuda" or not w.is_contiguous():
        raise ValueError("w must be a contiguous float64 CUDA tensor")
    ldv = n if ldv is None else ldv
    if n < 1 or j < 0 or (j > 0 and ldv < n):
        raise ValueError("bad sizes: need n >= 1, j >= 0 and ldv >= n")
    if w.numel() < n:
        raise ValueError(f"w holds {w.numel()} elements, fewer than n = {n}")
    if j > 0:
        if V.dtype != torch.float64 or V.device.type != "cuda" or not V.is_contiguous():
            raise ValueError("V must be a contiguous float64 CUDA tensor")
        if V.numel() < (j - 1) * ldv + n:
            raise ValueError(f"V holds {V.numel()} elements, fewer than (j - 1) * ldv + n = {(j - 1) * ldv + n}")
    return ldv


def cgs2_orthogonalize(V, n: int, j: int, w, ldv: int | None = None, stream=None):
    """One CGS2 step on device tensors: returns (h as numpy array, beta)."""
    ldv = _gs_args(V, n, j, w, ldv)
    lib = load_library()
    h = np.zeros(max(j, 1))
    beta = ctypes.c_double()
    s = current_stream_handle() if stream is None else ctypes.c_void_p(stream)
    vp = ctypes.c_void_p(V.data_ptr()) if j > 0 else ctypes.c_void_p(0)
    _check(lib.cgs2_orthogonalize(vp, ldv, n, j, ctypes.c_void_p(w.data_ptr()),
                                  h.ctypes.data_as(_dp), ctypes.byref(beta), s), "cgs2_orthogonalize")
    return h[:j], beta.value


NOALLOC_MAX_COLS = 256


def cgs2_orthogonalize_noalloc(V, n: int, j: int, w, ldv: int | None = None, stream=None):
    """cgs2_orthogonalize without any device allocation (fixed static scratch;
    j <= NOALLOC_MAX_COLS).  For callers that cannot allocate at call time,
    such as frameworks whose memory pool owns the device memory."""
    ldv = _gs_args(V, n, j, w, ldv)
    lib = load_library()
    h = np.zeros(max(j, 1))
    beta = ctypes.c_double()
    s = current_stream_handle() if stream is None else ctypes.c_void_p(stream)
    vp = ctypes.c_void_p(V.data_ptr()) if j > 0 else ctypes.c_void_p(0)
    _check(lib.cgs2_orthogonalize_noalloc(vp, ldv, n, j, ctypes.c_void_p(w.data_ptr()),
                                          h.ctypes.data_as(_dp), ctypes.byref(beta), s),
           "cgs2_orthogonalize_noalloc")
    return h[:j], beta.value


def dense_eig(A: np.ndarray, is_hessenberg: bool = False, vectors: bool = True):
    """Host eigen-solver of the library on a small dense matrix (no GPU)."""
    lib = load_library()
    A = np.asfortranarray(np.asarray(A, dtype=np.float64))
    n = A.shape[0]
    wr, wi = np.zeros(n), np.zeros(n)
    vr = np.zeros((n, n), order="F") if vectors else None
    vi = np.zeros((n, n), order="F") if vectors else None
    _check(lib.nsstab_dense_eig(n, A.ctypes.data_as(_dp), int(is_hessenberg), wr.ctypes.data_as(_dp),
                                wi.ctypes.data_as(_dp), vr.ctypes.data_as(_dp) if vectors else None,
                                vi.ctypes.data_as(_dp) if vectors else None), "nsstab_dense_eig")
    w = wr + 1j * wi
    return (w, vr + 1j * vi) if vectors else w


def dense_schur_ordered(A: np.ndarray, thr: float):
    """Real Schur form with the eigenvalues |lambda| >= thr first: (T, Z, p)."""
    lib = load_library()
    A = np.asfortranarray(np.asarray(A, dtype=np.float64))
    n = A.shape[0]
    T = np.zeros((n, n), order="F")
    Z = np.zeros((n, n), order="F")
    p = ctypes.c_int()
    _check(lib.nsstab_dense_schur_ordered(n, A.ctypes.data_as(_dp), float(thr), T.ctypes.data_as(_dp),
                                          Z.ctypes.data_as(_dp), ctypes.byref(p)), "nsstab_dense_schur_ordered")
    return T, Z, p.value


def serve_eigs(jobs, m: int, nev: int, tol: float, T: float, max_restarts: int = 0, mem_budget: int = 0,
               max_concurrent: int = 0, persistent: bool = False, **cfg):
    """Many eigen-solves on mixed grids (C ``serve_eigs``, or with
    ``persistent=True`` C ``serve_eigs_persistent``: every grid advanced by
    one persistent launch per step kernel, FP32 only).

    ``jobs``: list of dicts with keys nx, ny, dt, Re, cyl_D, base, v0 (base
    and v0 device tensors of shape [ny, nx]).  ``cfg``: shared physical
    parameters of ``nsstab_config``.  Returns (status, results, ngroups),
    results a list of dicts (status, mu, residual, n_conv, n_matvec, group,
    latency_s) in job order; for the persistent form group is the wave and
    ngroups the number of waves."""
    import torch

    lib = load_library()
    arr = (EigJob * len(jobs))()
    for i, j in enumerate(jobs):
        shape = (int(j["ny"]), int(j["nx"]))
        arr[i] = EigJob(int(j["nx"]), int(j["ny"]), float(j["dt"]), float(j["Re"]), float(j["cyl_D"]),
                        _field_ptr(j["base"], shape, "base").value, _field_ptr(j["v0"], shape, "v0").value)
    out = (EigJobResult * len(jobs))()
    ng = ctypes.c_int()
    c = _cfg_from(**cfg)
    torch.cuda.current_stream().synchronize()   # the call's own streams do not wait on torch's
    if persistent:
        rc = lib.serve_eigs_persistent(ctypes.byref(c), len(jobs), arr, int(m), int(nev), float(tol),
                                       int(max_restarts), float(T), int(mem_budget), out, ctypes.byref(ng))
    else:
        rc = lib.serve_eigs(ctypes.byref(c), len(jobs), arr, int(m), int(nev), float(tol), int(max_restarts),
                            float(T), int(mem_budget), int(max_concurrent), out, ctypes.byref(ng))
    if rc < 0 and all(out[i].status == 0 and out[i].n_eig == 0 for i in range(len(jobs))):
        _check(rc, "serve_eigs_persistent" if persistent else "serve_eigs")
    res = []
    for r in out:
        k = r.n_eig
        res.append({"status": r.status, "mu": np.array(r.eig_re[:k]) + 1j * np.array(r.eig_im[:k]),
                    "residual": np.array(r.resid[:k]), "n_conv": r.n_conv, "n_matvec": r.n_matvec,
                    "group": r.group, "latency_s": r.latency_s})
    return rc, res, ng.value


def _f32_ptr(t, numel, name):
    import torch

    if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.dtype != torch.float32 \
            or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if t.numel() != numel:
        raise ValueError(f"{name} must hold {numel} values")
    return ctypes.c_void_p(t.data_ptr())


class UNet:
    """Owner of a ``nsstab_unet*`` (the learned base-flow initial guess)."""

    def __init__(self, in_ch: int, width: int, ny: int, nx: int, max_batch: int):
        self._lib = load_library()
        self.in_ch, self.width, self.ny, self.nx, self.max_batch = in_ch, width, ny, nx, max_batch
        self.count = int(self._lib.unet_param_count(in_ch, width))
        h = ctypes.c_void_p()
        _check(self._lib.unet_create(in_ch, width, ny, nx, max_batch, current_stream_handle(), ctypes.byref(h)),
               "unet_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.unet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _batch(self, x):
        B = x.numel() // (self.in_ch * self.ny * self.nx)
        return B, _f32_ptr(x, B * self.in_ch * self.ny * self.nx, "x")

    def unet_set_params(self, theta):
        _check(self._lib.unet_set_params(self._h, _f32_ptr(theta, self.count, "theta")), "unet_set_params")

    def unet_get_params(self, theta):
        _check(self._lib.unet_get_params(self._h, _f32_ptr(theta, self.count, "theta")), "unet_get_params")

    def unet_forward(self, x, y):
        B, xp = self._batch(x)
        _check(self._lib.unet_forward(self._h, xp, B, _f32_ptr(y, B * self.ny * self.nx, "y")), "unet_forward")

    def unet_gradient(self, x, target, grad) -> float:
        B, xp = self._batch(x)
        loss = ctypes.c_double()
        _check(self._lib.unet_gradient(self._h, xp, _f32_ptr(target, B * self.ny * self.nx, "target"), B,
                                       _f32_ptr(grad, self.count, "grad"), ctypes.byref(loss)), "unet_gradient")
        return loss.value

    def unet_train_step(self, x, target, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                        eps: float = 1e-8) -> float:
        B, xp = self._batch(x)
        loss = ctypes.c_double()
        _check(self._lib.unet_train_step(self._h, xp, _f32_ptr(target, B * self.ny * self.nx, "target"), B,
                                         float(lr), float(beta1), float(beta2), float(eps), ctypes.byref(loss)),
               "unet_train_step")
        return loss.value


@dataclass
class EigResult:
    mu: np.ndarray          # Ritz values (eigenvalues of M)
    residual: np.ndarray    # |b^T y|
    n_conv: int
    n_matvec: int
    status: int

    def growth(self, T: float) -> np.ndarray:
        """lambda = log(mu)/T (eigenvalues of the linearised operator)."""
        return np.log(self.mu.astype(complex)) / T


class Stepper:
    """Owner of one ``nsstab_stepper`` bound to the current torch stream.

    ``Stepper(**cfg)`` is a single stepper; ``Stepper(Re=[...], cyl_D=[...],
    per_set=b, **cfg)`` with a list of Reynolds numbers (and optionally of
    diameters) is a batch of len(Re) * b members (``batch_create``): field
    arguments are then [B, ny, nx] tensors and base flows [S, ny, nx].
    """

    def __init__(self, per_set: int = 1, **cfg):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("nsstab needs a CUDA GPU")
        Re = cfg.pop("Re", None)
        D = cfg.pop("cyl_D", None)
        batched = np.ndim(Re) == 1 or np.ndim(D) == 1 or per_set != 1
        if not batched:
            if Re is not None:
                cfg["Re"] = Re
            if D is not None:
                cfg["cyl_D"] = D
        self.cfg = _cfg_from(**cfg)
        self.shape = (self.cfg.ny, self.cfg.nx)
        self._stream = torch.cuda.current_stream()
        self._lib = load_library()
        if not batched:
            self._h = stepper_create(self.cfg, self._stream.cuda_stream)
            self.members, self.sets = 1, 1
            return
        nsets = len(Re) if np.ndim(Re) == 1 else (len(D) if np.ndim(D) == 1 else 1)
        re = np.ascontiguousarray(np.broadcast_to(self.cfg.Re if Re is None else Re, (nsets,)), dtype=np.float64)
        dd = np.ascontiguousarray(np.broadcast_to(self.cfg.cyl_D if D is None else D, (nsets,)), dtype=np.float64)
        h = ctypes.c_void_p()
        _check(self._lib.batch_create(ctypes.byref(self.cfg), nsets, re.ctypes.data_as(_dp), dd.ctypes.data_as(_dp),
                                      int(per_set), ctypes.c_void_p(self._stream.cuda_stream), ctypes.byref(h)),
               "batch_create")
        self._h = h
        mem, sets = ctypes.c_int(), ctypes.c_int()
        _check(self._lib.stepper_members(self._h, ctypes.byref(mem), ctypes.byref(sets)), "stepper_members")
        self.members, self.sets = mem.value, sets.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.stepper_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _p(self, t, name, count=None):
        count = self.members if count is None else count
        p = _field_ptr(t, self.shape, name)
        if t.numel() != count * self.shape[0] * self.shape[1]:
            raise ValueError(f"{name} must hold {count} fields of shape {self.shape}")
        return p

    def stepper_poisson(self, omega, psi):
        _check(self._lib.stepper_poisson(self._h, self._p(omega, "omega"), self._p(psi, "psi")), "stepper_poisson")

    def step_nonlinear(self, omega, nsteps: int):
        _check(self._lib.step_nonlinear(self._h, self._p(omega, "omega"), int(nsteps)), "step_nonlinear")

    def stepper_set_base(self, base):
        _check(self._lib.stepper_set_base(self._h, self._p(base, "base", self.sets)), "stepper_set_base")

    def apply_expTL(self, base, v_in, v_out, T: float):
        bp = self._p(base, "base", self.sets) if base is not None else None
        _check(self._lib.apply_expTL(self._h, bp, self._p(v_in, "v_in"), self._p(v_out, "v_out"), float(T)),
               "apply_expTL")

    def stepper_residual(self, q):
        """Base-flow residual r(q); a float for a single stepper, an array for a batch."""
        r = np.zeros(self.members)
        _check(self._lib.stepper_residual(self._h, self._p(q, "q"), r.ctypes.data_as(_dp)), "stepper_residual",
               allow_soft=True)
        return float(r[0]) if self.members == 1 else r

    def sfd_baseflow(self, omega, chi: float, Delta: float, tol: float, max_steps: int, check_every: int = 100):
        r = np.zeros(self.members)
        steps = ctypes.c_long()
        rc = _check(self._lib.sfd_baseflow(self._h, self._p(omega, "omega"), float(chi), float(Delta), float(tol),
                                           int(max_steps), int(check_every), r.ctypes.data_as(_dp),
                                           ctypes.byref(steps)),
                    "sfd_baseflow", allow_soft=True)
        return rc, (float(r[0]) if self.members == 1 else r), steps.value

    JACOBIANS = {"tangent": 0, "frozen": 1}

    def newton_krylov_fixedpoint(self, omega, T: float, gmres_m: int, tol: float, max_newton: int,
                                 lin=None, gmres_rtol: float = 1e-3, gmres_restarts: int = 2,
                                 jacobian: str = "tangent"):
        """Newton-Krylov base flow; lin: optional second Stepper whose
        arithmetic the Jacobian products use; jacobian: "tangent" (exact
        discrete tangent, co-integrated) or "frozen" (linearised about the
        current iterate)."""
        r = ctypes.c_double()
        it, mv = ctypes.c_int(), ctypes.c_int()
        rc = _check(self._lib.newton_krylov_fixedpoint_ex(self._h, lin._h if lin is not None else None,
                                                          self._p(omega, "omega"), float(T), int(gmres_m),
                                                          float(gmres_rtol), int(gmres_restarts), float(tol),
                                                          int(max_newton), self.JACOBIANS[jacobian],
                                                          ctypes.byref(r), ctypes.byref(it), ctypes.byref(mv)),
                    "newton_krylov_fixedpoint", allow_soft=True)
        return rc, r.value, it.value, mv.value

    def apply_tangent(self, q, v_in, v_out, T: float):
        """v_out = dPhi_T(q)/dq v_in (a Stepper(per_set=2, ...) of one parameter set)."""
        _check(self._lib.apply_tangent(self._h, self._p(q, "q", 1), self._p(v_in, "v_in", 1),
                                       self._p(v_out, "v_out", 1), float(T)), "apply_tangent")

    def batch_arnoldi_eigs(self, bases, v0, m: int, nev: int, tol: float, T: float, max_restarts: int = 0,
                           eigvecs=None) -> list:
        """One eigenproblem per member (batched stepper): a list of EigResult."""
        B = self.members
        re, im, res = (np.zeros((B, nev + 1)) for _ in range(3))
        n_eig, n_conv, n_mv = (np.zeros(B, dtype=np.int32) for _ in range(3))
        bp = self._p(bases, "bases", self.sets) if bases is not None else None
        ev = None
        if eigvecs is not None:
            if eigvecs.numel() != B * (nev + 1) * self.shape[0] * self.shape[1]:
                raise ValueError("eigvecs must hold B * (nev + 1) fields")
            ev = _field_ptr(eigvecs, self.shape, "eigvecs")
        ip = lambda a: a.ctypes.data_as(_ip)
        rc = _check(self._lib.batch_arnoldi_eigs(self._h, bp, self._p(v0, "v0"), int(m), int(nev), float(tol),
                                                 int(max_restarts), float(T), re.ctypes.data_as(_dp),
                                                 im.ctypes.data_as(_dp), res.ctypes.data_as(_dp), ev, ip(n_eig),
                                                 ip(n_conv), ip(n_mv)),
                    "batch_arnoldi_eigs", allow_soft=True)
        out = []
        for b in range(B):
            k = int(n_eig[b])
            status = OK if n_conv[b] >= k else NOT_CONVERGED
            out.append(EigResult(re[b, :k] + 1j * im[b, :k], res[b, :k], int(n_conv[b]), int(n_mv[b]), status))
        return out

    def arnoldi_eigs(self, base, v0, m: int, nev: int, tol: float, T: float, max_restarts: int = 0,
                     eigvecs=None) -> EigResult:
        re, im, res = np.zeros(nev + 1), np.zeros(nev + 1), np.zeros(nev + 1)
        n_eig, n_conv, n_mv = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        bp = self._p(base, "base") if base is not None else None
        ev = None
        if eigvecs is not None:
            if eigvecs.shape[0] < nev + 1:
                raise ValueError("eigvecs must hold nev + 1 fields")
            ev = _field_ptr(eigvecs, self.shape, "eigvecs")
        rc = _check(self._lib.arnoldi_eigs(self._h, bp, self._p(v0, "v0"), int(m), int(nev), float(tol),
                                           int(max_restarts), float(T), re.ctypes.data_as(_dp),
                                           im.ctypes.data_as(_dp), res.ctypes.data_as(_dp), ev,
                                           ctypes.byref(n_eig), ctypes.byref(n_conv), ctypes.byref(n_mv)),
                    "arnoldi_eigs", allow_soft=True)
        k = n_eig.value
        return EigResult(re[:k] + 1j * im[:k], res[:k], n_conv.value, n_mv.value, rc)

    def block_arnoldi_eigs(self, base, v0, m: int, nev: int, tol: float, T: float, max_restarts: int = 0,
                           eigvecs=None):
        """Block Krylov-Schur with b = ``per_set`` vectors per product with M,
        one eigenproblem per parameter set (a stepper made as
        ``Stepper(per_set=b, Re=..., ...)``); v0: [sets * b, ny, nx], set s's
        start block in rows s*b .. s*b + b - 1.  Returns an EigResult for a
        single parameter set, else a list of them (one per set)."""
        S = self.sets
        re, im, res = (np.zeros((S, nev + 1)) for _ in range(3))
        n_eig, n_conv, n_mv = (np.zeros(S, dtype=np.int32) for _ in range(3))
        bp = self._p(base, "base", S) if base is not None else None
        ev = None
        if eigvecs is not None:
            if eigvecs.numel() < S * (nev + 1) * self.shape[0] * self.shape[1]:
                raise ValueError("eigvecs must hold sets * (nev + 1) fields")
            ev = _field_ptr(eigvecs, self.shape, "eigvecs")
        ip = lambda a: a.ctypes.data_as(_ip)
        rc = _check(self._lib.block_arnoldi_eigs(self._h, bp, self._p(v0, "v0"), int(m), int(nev), float(tol),
                                                 int(max_restarts), float(T), re.ctypes.data_as(_dp),
                                                 im.ctypes.data_as(_dp), res.ctypes.data_as(_dp), ev, ip(n_eig),
                                                 ip(n_conv), ip(n_mv)),
                    "block_arnoldi_eigs", allow_soft=True)
        out = []
        for s in range(S):
            k = int(n_eig[s])
            status = OK if n_conv[s] >= k else NOT_CONVERGED
            out.append(EigResult(re[s, :k] + 1j * im[s, :k], res[s, :k], int(n_conv[s]), int(n_mv[s]),
                                 rc if S == 1 else status))
        return out[0] if S == 1 else out

    KERNELS = ("col_poisson", "row_inverse_psi", "row_forward_rhs", "col_update", "row_inverse_star",
               "row_forward_pen")

    def stepper_profile_linear(self, v, nsteps: int) -> dict:  # noqa: D401
        """Per-kernel milliseconds (summed over nsteps linearised steps)."""
        ms = np.zeros(6)
        _check(self._lib.stepper_profile_linear(self._h, self._p(v, "v"), int(nsteps), ms.ctypes.data_as(_dp)),
               "stepper_profile_linear")
        return dict(zip(self.KERNELS, ms.tolist()))

    def stepper_autotune(self, reps: int = 10) -> dict:
        """Time every valid launch plan of each kernel and keep the fastest."""
        plans = (ctypes.c_int * 12)()
        _check(self._lib.stepper_autotune(self._h, int(reps), plans), "stepper_autotune")
        return {k: (plans[2 * i], plans[2 * i + 1]) for i, k in enumerate(self.KERNELS)}

    def stepper_set_plan(self, kernel: int, log2_elems: int, per_block: int):
        _check(self._lib.stepper_set_plan(self._h, int(kernel), int(log2_elems), int(per_block)), "stepper_set_plan")

    def stepper_get_plan(self, kernel: int):
        le, per = ctypes.c_int(), ctypes.c_int()
        _check(self._lib.stepper_get_plan(self._h, int(kernel), ctypes.byref(le), ctypes.byref(per)),
               "stepper_get_plan")
        return le.value, per.value

    def stepper_set_fused_rows(self, rows_per_strip: int):
        """FP32: four-kernel step with fused row passes over strips of
        rows_per_strip rows (0: the six-kernel step)."""
        _check(self._lib.stepper_set_fused_rows(self._h, int(rows_per_strip)), "stepper_set_fused_rows")

    def stepper_get_fused_rows(self) -> int:
        r = ctypes.c_int()
        _check(self._lib.stepper_get_fused_rows(self._h, ctypes.byref(r)), "stepper_get_fused_rows")
        return r.value

    def plans(self) -> dict:
        return {k: self.stepper_get_plan(i) for i, k in enumerate(self.KERNELS)}

    def steps_for(self, T: float) -> int:
        k = int(round(T / self.cfg.dt))
        if k < 1 or not math.isclose(k * self.cfg.dt, T, rel_tol=1e-9):
            raise ValueError("T must be a whole number of steps")
        return k
