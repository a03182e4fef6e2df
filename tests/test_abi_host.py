"""CPU-side checks of the C-ABI library: it loads, exports every symbol that
include/nsstab.h declares, validates arguments before touching a GPU, and its
host dense eigen-solver (the Ritz-value / Schur step of the Krylov layer)
agrees with LAPACK.  No compute call here needs a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest
import scipy.linalg

from paper_1804_03859_gb300 import build, nsstab

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return nsstab.load_library()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "nsstab.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:void|int|long|char)\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(n for n, _, _ in nsstab.SIGNATURES) == names


def test_config_defaults_match_the_cylinder_case(lib):
    from oracle import ns2d

    cfg = nsstab.config_default()
    ref = ns2d.Config()
    for k in ("nx", "ny", "Lx", "Ly", "dt", "Re", "Uinf", "cyl_x", "cyl_y", "cyl_D", "eta", "mask_cells",
              "sponge_frac", "sponge_sigma"):
        assert getattr(cfg, k) == getattr(ref, k), k
    assert cfg.precision == 64


@pytest.mark.parametrize("field,value", [("nx", 100), ("ny", 4), ("nx", 8192), ("dt", 0.0), ("Re", -1.0),
                                         ("precision", 16), ("eta", 0.0)])
def test_bad_configs_are_rejected_before_any_device_call(lib, field, value):
    cfg = nsstab.config_default()
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    rc = lib.stepper_create(ctypes.byref(cfg), None, ctypes.byref(h))
    assert rc == -1
    assert h.value is None
    assert len(lib.nsstab_last_error()) > 0


def test_null_arguments_are_rejected(lib):
    assert lib.step_nonlinear(None, None, 1) == -1
    assert lib.apply_expTL(None, None, None, None, 1.0) == -1
    assert lib.cgs2_orthogonalize(None, 1, 1, 1, None, None, None, None) == -1


@pytest.mark.parametrize("job,kw,what", [
    (dict(nx=30), {}, "job 1"),             # grid not a power of two
    (dict(dt=0.03), {}, "job 1"),           # T = 2 is not a whole number of steps
    (dict(Re=0.0), {}, "job 1"),
    ({}, dict(nev=40), "nev"),              # nev >= m
    ({}, dict(T=0.0), "T > 0"),
])
def test_serve_eigs_validates_every_job_before_any_device_call(lib, job, kw, what):
    """The pointers below are never dereferenced: validation fails first."""
    good = dict(nx=32, ny=16, dt=0.02, Re=50.0, cyl_D=1.0, base=16, v0=16)
    bad = dict(good, **job)
    jobs = (nsstab.EigJob * 2)()
    for i, j in enumerate((good, bad)):
        jobs[i] = nsstab.EigJob(j["nx"], j["ny"], j["dt"], j["Re"], j["cyl_D"], j["base"], j["v0"])
    out = (nsstab.EigJobResult * 2)()
    ng = ctypes.c_int(-7)
    a = dict(m=40, nev=4, tol=1e-8, max_restarts=1, T=2.0)
    a.update(kw)
    cfg = nsstab.config_default()
    rc = lib.serve_eigs(ctypes.byref(cfg), 2, jobs, a["m"], a["nev"], a["tol"], a["max_restarts"], a["T"], 0, 0,
                        out, ctypes.byref(ng))
    assert rc == -1
    assert what in lib.nsstab_last_error().decode()
    assert ng.value == -7


@pytest.mark.parametrize("job,kw,what", [
    (dict(nx=30), {}, "job 1"),             # grid not a power of two
    (dict(dt=0.03), {}, "job 1"),           # T = 2 is not a whole number of steps
    ({}, dict(nev=40), "nev"),              # nev >= m
    ({}, dict(precision=64), "precision 32"),   # the persistent launch runs the FP32 stepper
])
def test_serve_eigs_persistent_validates_before_any_device_call(lib, job, kw, what):
    """As serve_eigs, plus the FP32-only rule; no pointer is dereferenced."""
    good = dict(nx=32, ny=16, dt=0.02, Re=50.0, cyl_D=1.0, base=16, v0=16)
    bad = dict(good, **job)
    jobs = (nsstab.EigJob * 2)()
    for i, j in enumerate((good, bad)):
        jobs[i] = nsstab.EigJob(j["nx"], j["ny"], j["dt"], j["Re"], j["cyl_D"], j["base"], j["v0"])
    out = (nsstab.EigJobResult * 2)()
    nw = ctypes.c_int(-7)
    a = dict(m=40, nev=4, precision=32)
    a.update(kw)
    cfg = nsstab.config_default()
    cfg.precision = a["precision"]
    rc = lib.serve_eigs_persistent(ctypes.byref(cfg), 2, jobs, a["m"], a["nev"], 1e-6, 1, 2.0, 0, out,
                                   ctypes.byref(nw))
    assert rc == -1
    assert what in lib.nsstab_last_error().decode()
    assert nw.value == -7


def _match(a, b):
    return max(np.min(np.abs(b - x)) for x in a)


@pytest.mark.parametrize("n,seed", [(5, 0), (24, 1), (80, 2), (150, 3)])
def test_dense_eig_matches_lapack(lib, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    w, V = nsstab.dense_eig(A)
    wl = np.linalg.eigvals(A)
    scale = np.abs(wl).max()
    assert _match(w, wl) < 1e-10 * scale and _match(wl, w) < 1e-10 * scale
    for k in range(n):
        v = V[:, k]
        assert abs(np.linalg.norm(v) - 1) < 1e-12
        assert np.linalg.norm(A @ v - w[k] * v) < 1e-9 * scale


def test_dense_eig_on_hessenberg_input_and_repeated_values(lib):
    rng = np.random.default_rng(5)
    H = np.triu(rng.standard_normal((40, 40)), -1)
    w = nsstab.dense_eig(H, is_hessenberg=True, vectors=False)
    assert _match(w, np.linalg.eigvals(H)) < 1e-10 * np.abs(w).max()
    # a rotation-like matrix with conjugate pairs of equal modulus
    B = scipy.linalg.block_diag(*[np.array([[np.cos(t), -np.sin(t)], [np.sin(t), np.cos(t)]]) * r
                                  for t, r in [(0.3, 1.0), (1.1, 0.9), (2.0, 0.5)]])
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    w = nsstab.dense_eig(Q @ B @ Q.T, vectors=False)
    assert _match(w, np.linalg.eigvals(B)) < 1e-12


@pytest.mark.parametrize("n,seed", [(12, 0), (40, 1), (100, 2)])
def test_ordered_schur_puts_the_wanted_values_first(lib, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) / np.sqrt(n)
    mags = np.sort(np.abs(np.linalg.eigvals(A)))[::-1]
    thr = 0.5 * (mags[n // 3] + mags[n // 3 + 1])
    T, Z, p = nsstab.dense_schur_ordered(A, thr)
    assert np.abs(Z.T @ Z - np.eye(n)).max() < 1e-12
    assert np.linalg.norm(Z @ T @ Z.T - A) < 1e-12 * np.linalg.norm(A)
    assert np.abs(np.tril(T, -2)).max() == 0.0
    lead = np.linalg.eigvals(T[:p, :p])
    tail = np.linalg.eigvals(T[p:, p:])
    assert np.all(np.abs(lead) >= thr) and np.all(np.abs(tail) < thr)
    assert p == int(np.sum(mags >= thr))
    # same invariant subspace as scipy's sorted Schur form
    _, Zs, sdim = scipy.linalg.schur(A, output="real", sort=lambda x, y: np.hypot(x, y) >= thr)
    assert sdim == p
    s = np.linalg.svd(Z[:, :p].T @ Zs[:, :p], compute_uv=False)
    assert s.min() > 1 - 1e-10


class _FakeCudaTensor:
    """Stands in for a float64 CUDA tensor of a given size (no GPU needed):
    the CGS2 wrappers must reject undersized buffers before any call."""

    def __init__(self, numel):
        import torch

        self.dtype = torch.float64
        self.device = torch.device("cuda", 0)
        self._n = numel

    def is_contiguous(self):
        return True

    def numel(self):
        return self._n

    def data_ptr(self):
        raise AssertionError("an undersized buffer reached the C call")


@pytest.mark.parametrize("fn", [nsstab.cgs2_orthogonalize, nsstab.cgs2_orthogonalize_noalloc])
@pytest.mark.parametrize("vsize,wsize,j,ldv", [
    (4 * 1000 - 1, 1000, 4, None),      # V one element short of j columns
    (3 * 1200 + 999, 1000, 4, 1200),    # with a leading dimension: (j-1) ldv + n - 1
    (4 * 1000, 999, 4, None),           # w short
    (4 * 1000, 1000, 4, 999),           # ldv < n
])
def test_cgs2_wrappers_reject_undersized_tensors(fn, vsize, wsize, j, ldv):
    with pytest.raises(ValueError):
        fn(_FakeCudaTensor(vsize), 1000, j, _FakeCudaTensor(wsize), ldv=ldv)
