"""The serving batch (many eigen-solves on mixed grids, grouped into batched
steppers that run concurrently under a device-memory budget): every solve
gives the Ritz values of the same solve run alone, one of them pinned to the
dense eigendecomposition of the assembled propagator; a small budget splits
the groups and still gives the same values; a budget below one solve
fails those solves cleanly."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense, krylov, ns2d  # noqa: E402
from paper_1804_03859_gb300 import inputs, nsstab  # noqa: E402

pytestmark = pytest.mark.gpu

T, M, NEV, TOL = 2.0, 40, 4, 1e-9
# (nx, ny, dt, Re, D): two grids, three and two solves
SPECS = [(32, 16, 0.02, 50.0, 1.0), (64, 32, 0.01, 50.0, 1.0), (32, 16, 0.02, 40.0, 0.8),
         (64, 32, 0.01, 70.0, 0.9), (32, 16, 0.02, 60.0, 1.2)]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _match(a, b):
    return max(np.min(np.abs(b - x)) for x in a)


@pytest.fixture(scope="module")
def jobs():
    out = []
    for i, (nx, ny, dt, re, d) in enumerate(SPECS):
        out.append(dict(nx=nx, ny=ny, dt=dt, Re=re, cyl_D=d,
                        base=_dev(inputs.wake_like_field(ny, nx, seed=60 + i)),
                        v0=_dev(inputs.gaussian_field(ny, nx, seed=70 + i))))
    return out


@pytest.fixture(scope="module")
def alone(jobs):
    """Each solve on its own single stepper (arnoldi_eigs)."""
    res = []
    for j in jobs:
        st = nsstab.Stepper(nx=j["nx"], ny=j["ny"], dt=j["dt"], Re=j["Re"], cyl_D=j["cyl_D"])
        r = st.arnoldi_eigs(j["base"], j["v0"], m=M, nev=NEV, tol=TOL, T=T, max_restarts=60)
        assert r.n_conv == len(r.mu)
        res.append(r.mu)
    return res


def test_serving_batch_matches_solves_run_alone(jobs, alone):
    t0 = time.perf_counter()
    rc, res, ngroups = nsstab.serve_eigs(jobs, m=M, nev=NEV, tol=TOL, T=T, max_restarts=60)
    wall = time.perf_counter() - t0
    assert rc == nsstab.OK
    assert ngroups == 2
    groups = {}
    for j, r, mu in zip(jobs, res, alone):
        assert r["status"] == nsstab.OK and r["n_conv"] == len(r["mu"]) == len(mu)
        assert _match(r["mu"], mu) <= 1e-8
        assert 0.0 < r["latency_s"] <= wall
        groups.setdefault((j["nx"], j["ny"]), set()).add(r["group"])
    assert all(len(g) == 1 for g in groups.values())
    assert groups[(64, 32)] != groups[(32, 16)]


def test_serving_pinned_to_the_dense_propagator(jobs):
    """Job 0 is the 32x16 cylinder case at Re 50: its Ritz values are
    eigenvalues of the explicitly assembled M = exp(T A)."""
    j = jobs[0]
    cfg = ns2d.Config(nx=32, ny=16, dt=0.02, Re=50.0, cyl_D=1.0)
    base = j["base"].cpu().numpy()
    mu = np.linalg.eigvals(dense.assemble_M(ns2d.Base.from_omega(base, cfg), T, cfg))
    mu = mu[krylov.leading_order(mu)]
    rc, res, _ = nsstab.serve_eigs(jobs[:1], m=M, nev=NEV, tol=TOL, T=T, max_restarts=60)
    assert rc == nsstab.OK
    assert _match(res[0]["mu"], mu[:6]) <= 1e-8


def test_small_budget_splits_groups_with_the_same_results(jobs, alone):
    # room for one 64x32 solve at a time, not two (the estimate is about
    # 67.8 MB fixed + 1.0 MB per 64x32 solve)
    rc, res, ngroups = nsstab.serve_eigs(jobs, m=M, nev=NEV, tol=TOL, T=T, max_restarts=60,
                                         mem_budget=69_000_000, max_concurrent=3)
    assert rc == nsstab.OK
    assert ngroups >= 3
    for r, mu in zip(res, alone):
        assert _match(r["mu"], mu) <= 1e-8


def test_budget_below_one_solve_fails_those_solves(jobs):
    rc, res, ngroups = nsstab.serve_eigs(jobs, m=M, nev=NEV, tol=TOL, T=T, mem_budget=1 << 20)
    assert rc == -3
    assert ngroups == 0
    assert all(r["status"] == -3 for r in res)


def test_double_float_serving_batch(jobs, alone):
    rc, res, _ = nsstab.serve_eigs(jobs, m=M, nev=NEV, tol=TOL, T=T, max_restarts=60, precision=48)
    assert rc == nsstab.OK
    for r, mu in zip(res, alone):
        assert _match(r["mu"], mu) <= 1e-8


def test_one_job_and_a_single_group(jobs, alone):
    rc, res, ngroups = nsstab.serve_eigs(jobs[3:4], m=M, nev=NEV, tol=TOL, T=T, max_restarts=60)
    assert rc == nsstab.OK and ngroups == 1 and res[0]["group"] == 0
    assert _match(res[0]["mu"], alone[3]) <= 1e-8


def test_fp32_serving_batch(jobs, alone):
    """FP32 steppers in the serving batch: leading values within 1e-5 relative."""
    rc, res, _ = nsstab.serve_eigs(jobs, m=M, nev=NEV, tol=1e-6, T=T, max_restarts=60, precision=32)
    assert rc == nsstab.OK
    for r, mu in zip(res, alone):
        for x in r["mu"]:
            assert np.min(np.abs(mu - x)) <= 1e-5 * abs(x)


def test_concurrent_groups_on_four_grids_raise_no_error():
    """Groups on grids with different launch plans run at once in separate
    threads (launch attributes are shared per kernel function)."""
    jobs = []
    for i, (nx, ny) in enumerate([(32, 16), (64, 32), (128, 64), (256, 128)] * 3):
        dt = 0.01 * 128 / nx
        jobs.append(dict(nx=nx, ny=ny, dt=dt, Re=50.0 + i, cyl_D=1.0,
                         base=_dev(inputs.wake_like_field(ny, nx, seed=80 + i)),
                         v0=_dev(inputs.gaussian_field(ny, nx, seed=90 + i))))
    for _ in range(3):
        rc, res, ngroups = nsstab.serve_eigs(jobs, m=24, nev=2, tol=1e-6, T=0.32, max_restarts=2, precision=32,
                                             max_concurrent=4)
        assert rc >= 0, nsstab.load_library().nsstab_last_error()
        assert ngroups == 4
        assert all(r["status"] >= 0 and r["n_matvec"] > 0 for r in res)


# ------------------------------------------------- one persistent launch

RAG_SPECS = [(64, 32, 0.02, 50.0, 1.0), (128, 64, 0.01, 45.0, 0.9), (64, 32, 0.02, 70.0, 1.1),
             (256, 128, 0.005, 60.0, 1.0), (128, 64, 0.01, 80.0, 1.2)]
RT, RM, RNEV, RTOL = 0.4, 48, 4, 1e-6


@pytest.fixture(scope="module")
def rag_jobs():
    out = []
    for i, (nx, ny, dt, re, d) in enumerate(RAG_SPECS):
        out.append(dict(nx=nx, ny=ny, dt=dt, Re=re, cyl_D=d,
                        base=_dev(inputs.wake_like_field(ny, nx, seed=80 + i)),
                        v0=_dev(inputs.gaussian_field(ny, nx, seed=90 + i))))
    return out


def test_persistent_launch_matches_per_grid_batches(rag_jobs):
    """Three grids with three time steps (20, 40 and 80 steps per product)
    advanced by the same launches: every solve's leading eigenvalues equal
    those of the per-grid batched steppers (both FP32; 1e-5 relative)."""
    rc0, ref, ng0 = nsstab.serve_eigs(rag_jobs, m=RM, nev=RNEV, tol=RTOL, T=RT, max_restarts=80, precision=32)
    rc1, got, nwaves = nsstab.serve_eigs(rag_jobs, m=RM, nev=RNEV, tol=RTOL, T=RT, max_restarts=80, precision=32,
                                         persistent=True)
    assert rc0 == nsstab.OK and rc1 == nsstab.OK
    assert ng0 == 3 and nwaves == 1
    for a, b in zip(ref, got):
        assert b["status"] == nsstab.OK and b["n_conv"] == len(b["mu"]) == len(a["mu"])
        assert b["group"] == 0 and b["latency_s"] > 0
        for x in b["mu"]:
            assert np.min(np.abs(a["mu"] - x)) <= 1e-5 * abs(x)


def test_persistent_launch_pinned_to_the_dense_propagator(rag_jobs):
    """The 64x32 solve at Re 50 through the persistent launch (alongside a
    128x64 one): its Ritz values are eigenvalues of the assembled M."""
    j = rag_jobs[0]
    cfg = ns2d.Config(nx=64, ny=32, dt=0.02, Re=50.0, cyl_D=1.0)
    mu = np.linalg.eigvals(dense.assemble_M(ns2d.Base.from_omega(j["base"].cpu().numpy(), cfg), RT, cfg))
    mu = mu[krylov.leading_order(mu)][:6]
    rc, res, _ = nsstab.serve_eigs([j, rag_jobs[1]], m=RM, nev=RNEV, tol=RTOL, T=RT, max_restarts=80,
                                   precision=32, persistent=True)
    assert rc == nsstab.OK
    for x in res[0]["mu"]:
        assert np.min(np.abs(mu - x)) <= 1e-5 * abs(x)


def test_persistent_waves_under_a_small_budget_give_the_same_values(rag_jobs):
    rc0, ref, _ = nsstab.serve_eigs(rag_jobs, m=RM, nev=RNEV, tol=RTOL, T=RT, max_restarts=80, precision=32,
                                    persistent=True)
    rc1, got, nwaves = nsstab.serve_eigs(rag_jobs, m=RM, nev=RNEV, tol=RTOL, T=RT, max_restarts=80, precision=32,
                                         persistent=True, mem_budget=100 << 20)
    assert rc0 == nsstab.OK and rc1 == nsstab.OK and nwaves >= 2
    for a, b in zip(ref, got):
        for x in b["mu"]:
            assert np.min(np.abs(a["mu"] - x)) <= 1e-5 * abs(x)


def test_persistent_launch_needs_the_fp32_stepper(rag_jobs):
    with pytest.raises(nsstab.NsstabError, match="precision 32"):
        nsstab.serve_eigs(rag_jobs[:1], m=RM, nev=RNEV, tol=RTOL, T=RT, precision=64, persistent=True)
