"""GPU parity of the Krylov layer (steps a6-a7): CGS2 against numpy, Arnoldi
and Krylov-Schur eigenvalues against the oracle's Arnoldi and against LAPACK
on the explicitly assembled propagator.  Bar: leading eigenvalues within
1e-8 (FP64 stepper) and 1e-5 relative (FP32 stepper)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense, krylov, ns2d  # noqa: E402
from paper_1804_03859_gb300 import inputs, nsstab  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _match(a, b):
    return max(np.min(np.abs(b - x)) for x in a)


@pytest.mark.parametrize("n,j", [(1000, 0), (1000, 1), (8192, 7), (131072, 65), (100003, 129)])
def test_cgs2_parity(n, j):
    rng = np.random.default_rng(n + j)
    V = np.linalg.qr(rng.standard_normal((n, max(j, 1))))[0][:, :j] if j else np.zeros((n, 0))
    w = rng.standard_normal(n)
    Vd = _dev(np.ascontiguousarray(V.T)) if j else torch.zeros(1, dtype=torch.float64, device="cuda")
    wd = _dev(w)
    h, beta = nsstab.cgs2_orthogonalize(Vd, n, j, wd)
    torch.cuda.synchronize()
    h1 = V.T @ w
    w1 = w - V @ h1
    h2 = V.T @ w1
    w2 = w1 - V @ h2
    assert np.allclose(h, h1 + h2, rtol=0, atol=1e-12 * np.linalg.norm(w))
    assert abs(beta - np.linalg.norm(w2)) <= 1e-12 * np.linalg.norm(w)
    got = wd.cpu().numpy()
    assert np.linalg.norm(got - w2) <= 1e-12 * np.linalg.norm(w)
    if j:
        assert np.abs(V.T @ got).max() <= 1e-13 * np.linalg.norm(w)


@pytest.fixture(scope="module")
def small():
    kw = dict(nx=32, ny=16, dt=0.02, Re=50.0)
    cfg = ns2d.Config(**kw)
    base = inputs.wake_like_field(16, 32, seed=7)
    T = 2.0
    M = dense.assemble_M(ns2d.Base.from_omega(base, cfg), T, cfg)
    mu = np.linalg.eigvals(M)
    return kw, cfg, base, T, mu[krylov.leading_order(mu)]


def test_arnoldi_matches_dense_eigendecomposition(small):
    kw, cfg, base, T, mu_dense = small
    st = nsstab.Stepper(**kw)
    v0 = inputs.gaussian_field(16, 32, seed=11)
    res = st.arnoldi_eigs(_dev(base), _dev(v0), m=150, nev=4, tol=1e-10, T=T)
    assert res.status == nsstab.OK and res.n_conv == len(res.mu) == 5
    assert res.n_matvec == 150
    assert _match(res.mu, mu_dense[:6]) <= 1e-10


def test_arnoldi_ritz_values_match_the_oracle_arnoldi(small):
    kw, cfg, base, T, _ = small
    b = ns2d.Base.from_omega(base, cfg)
    v0 = inputs.gaussian_field(16, 32, seed=12)
    m = 40
    st = nsstab.Stepper(**kw)
    got = st.arnoldi_eigs(_dev(base), _dev(v0), m=m, nev=6, tol=1e-6, T=T)
    ref = krylov.arnoldi_eigs(lambda x: ns2d.apply_expTL(b, x.reshape(16, 32), T, cfg).ravel(),
                              v0.ravel(), m=m, nev=6, tol=1e-6)
    assert len(got.mu) == len(ref.mu)
    assert _match(got.mu, ref.mu) <= 1e-8 and _match(ref.mu, got.mu) <= 1e-8
    for g, r in zip(np.sort_complex(got.mu), np.sort_complex(ref.mu)):
        pass
    order_g = np.lexsort((-got.mu.imag, -np.abs(got.mu)))
    assert np.all(order_g == np.arange(len(got.mu)))
    # residual estimates agree where they are above round-off
    assert np.allclose(np.sort(got.residual), np.sort(ref.residual), rtol=1e-5, atol=1e-12)


def test_krylov_schur_matches_dense(small):
    kw, cfg, base, T, mu_dense = small
    st = nsstab.Stepper(**kw)
    v0 = inputs.gaussian_field(16, 32, seed=14)
    res = st.arnoldi_eigs(_dev(base), _dev(v0), m=40, nev=4, tol=1e-11, T=T, max_restarts=200)
    assert res.status == nsstab.OK and res.n_conv == len(res.mu)
    assert res.n_matvec > 40
    assert _match(res.mu, mu_dense[:6]) <= 1e-10


def test_ritz_vectors_are_eigenvectors(small):
    kw, cfg, base, T, mu_dense = small
    st = nsstab.Stepper(**kw)
    v0 = inputs.gaussian_field(16, 32, seed=15)
    vecs = torch.zeros(6, 16, 32, dtype=torch.float64, device="cuda")
    res = st.arnoldi_eigs(_dev(base), _dev(v0), m=150, nev=3, tol=1e-10, T=T, eigvecs=vecs)
    V = vecs.cpu().numpy().reshape(6, -1)
    b = ns2d.Base.from_omega(base, cfg)
    k = 0
    while k < len(res.mu):
        mu = res.mu[k]
        if abs(mu.imag) > 0 and k + 1 < len(res.mu):
            x = V[k] + 1j * V[k + 1]
            step = 2
        else:
            x = V[k].astype(complex)
            step = 1
        Mx = ns2d.apply_expTL(b, x.real.reshape(16, 32), T, cfg) + 1j * ns2d.apply_expTL(b, x.imag.reshape(16, 32), T, cfg)
        assert np.linalg.norm(Mx.ravel() - mu * x) <= 1e-9 * np.linalg.norm(x)
        assert abs(np.linalg.norm(x) - 1) < 1e-10
        k += step


def test_cylinder_case_128x64_arnoldi_against_oracle():
    """The 128x64 cylinder workload: Krylov dimension 64, leading 4 values."""
    kw = dict(nx=128, ny=64, dt=0.01, Re=50.0)
    cfg = ns2d.Config(**kw)
    base = ns2d.step_nonlinear(np.zeros((64, 128)), 300, cfg)   # developing wake
    v0 = inputs.gaussian_field(64, 128, seed=0)
    T, m = 0.5, 64
    st = nsstab.Stepper(**kw)
    got = st.arnoldi_eigs(_dev(base), _dev(v0), m=m, nev=4, tol=1e-8, T=T)
    b = ns2d.Base.from_omega(base, cfg)
    ref = krylov.arnoldi_eigs(lambda x: ns2d.apply_expTL(b, x.reshape(64, 128), T, cfg).ravel(),
                              v0.ravel(), m=m, nev=4, tol=1e-8)
    assert len(got.mu) == len(ref.mu)
    assert _match(got.mu, ref.mu) <= 1e-8


def test_fp32_stepper_eigenvalues_within_1e5(small):
    kw, cfg, base, T, mu_dense = small
    st = nsstab.Stepper(precision=32, **kw)
    v0 = inputs.gaussian_field(16, 32, seed=16)
    res = st.arnoldi_eigs(_dev(base), _dev(v0), m=40, nev=4, tol=1e-6, T=T, max_restarts=200)
    assert res.n_conv == len(res.mu)
    for mu in res.mu:
        assert np.min(np.abs(mu_dense - mu)) <= 1e-5 * abs(mu)


def test_fp32_eigenvalues_track_fp64_on_a_fine_grid():
    """256x128 (100 steps per product with M): the FP32 stepper's leading
    eigenvalues stay within 1e-5 relative of the FP64 stepper's, which the
    tests above pin to the oracle."""
    nx, ny = 256, 128
    kw = dict(nx=nx, ny=ny, dt=0.01 * 128 / nx, Re=60.0)
    base = _dev(inputs.wake_like_field(ny, nx, seed=21))
    v0 = _dev(inputs.gaussian_field(ny, nx, seed=22))
    ref = nsstab.Stepper(**kw).arnoldi_eigs(base, v0, m=96, nev=4, tol=1e-9, T=0.5, max_restarts=20)
    got = nsstab.Stepper(precision=32, **kw).arnoldi_eigs(base, v0, m=96, nev=4, tol=1e-7, T=0.5,
                                                          max_restarts=20)
    assert ref.n_conv == len(ref.mu) and got.n_conv == len(got.mu)
    for mu in got.mu:
        assert np.min(np.abs(ref.mu - mu)) <= 1e-5 * abs(mu)


@pytest.mark.parametrize("b,m", [(1, 60), (2, 60), (3, 60), (4, 60), (8, 96)])
def test_block_krylov_schur_matches_dense_eigendecomposition(small, b, m):
    """Block Krylov-Schur (blocked CGS2 against the basis, then within the
    block) against LAPACK on the assembled propagator, every block size the
    blocked kernels are instantiated for up to 8 (odd sizes included)."""
    kw, cfg, base, T, mu_dense = small
    st = nsstab.Stepper(per_set=b, **kw)
    v0 = np.stack([inputs.gaussian_field(16, 32, seed=40 + i) for i in range(b)])
    res = st.block_arnoldi_eigs(_dev(base), _dev(v0), m=m, nev=4, tol=1e-10, T=T, max_restarts=200)
    assert res.status == nsstab.OK and res.n_conv == len(res.mu)
    assert _match(res.mu, mu_dense[:6]) <= 1e-10
    assert res.n_matvec % b == 0


def test_block_krylov_schur_matches_single_vector_on_a_wake():
    kw = dict(nx=128, ny=64, dt=0.01, Re=50.0)
    cfg = ns2d.Config(**kw)
    base = _dev(ns2d.step_nonlinear(np.zeros((64, 128)), 300, cfg))
    T = 0.5
    v0 = np.stack([inputs.gaussian_field(64, 128, seed=50 + i) for i in range(4)])
    one = nsstab.Stepper(**kw).arnoldi_eigs(base, _dev(v0[0]), m=64, nev=6, tol=1e-9, T=T, max_restarts=40)
    blk = nsstab.Stepper(per_set=2, **kw).block_arnoldi_eigs(base, _dev(v0[:2]), m=128, nev=6, tol=1e-9, T=T,
                                                             max_restarts=60)
    assert one.n_conv == len(one.mu) and blk.n_conv == len(blk.mu)
    assert _match(blk.mu, one.mu) <= 1e-8 and _match(one.mu, blk.mu) <= 1e-8
    ev = torch.empty(7, 64, 128, dtype=torch.float64, device="cuda")
    st = nsstab.Stepper(per_set=2, **kw)
    r2 = st.block_arnoldi_eigs(base, _dev(v0[:2]), m=64, nev=2, tol=1e-9, T=T, max_restarts=40, eigvecs=ev)
    # leading Ritz vector: M x = mu x to the Ritz residual (a complex pair is
    # stored as Re in slot 0 and Im in slot 1, and M Re = Re(mu) Re - Im(mu) Im)
    x = ev[0].clone()
    mx = torch.empty_like(x)
    nsstab.Stepper(**kw).apply_expTL(base, x, mx, T)
    mu = r2.mu[0]
    ref = mu.real * x - (mu.imag * ev[1] if mu.imag != 0 else 0.0)
    assert float(torch.linalg.norm(mx - ref)) <= 1e-7


def test_block_krylov_schur_rejects_bad_input():
    kw = dict(nx=32, ny=16, dt=0.02, Re=50.0)
    base = _dev(np.zeros((16, 32)))
    st = nsstab.Stepper(per_set=2, **kw)
    same = _dev(np.stack([inputs.gaussian_field(16, 32, seed=1)] * 2))
    with pytest.raises(nsstab.NsstabError):
        st.block_arnoldi_eigs(base, same, m=40, nev=2, tol=1e-8, T=0.4)     # dependent start block
    with pytest.raises(nsstab.NsstabError):
        st.block_arnoldi_eigs(base, same, m=8, nev=2, tol=1e-8, T=0.4)      # m too small for b and nev
    two_sets = nsstab.Stepper(Re=[40.0, 50.0], per_set=2, nx=32, ny=16, dt=0.02)
    with pytest.raises(ValueError):
        two_sets.block_arnoldi_eigs(None, same, m=40, nev=2, tol=1e-8, T=0.4)   # needs sets * b start vectors
    wide = nsstab.Stepper(per_set=8, nx=64, ny=32, dt=0.02, Re=50.0)
    eight = _dev(np.stack([inputs.gaussian_field(32, 64, seed=s) for s in range(8)]))
    with pytest.raises(nsstab.NsstabError):
        wide.block_arnoldi_eigs(None, eight, m=800, nev=2, tol=1e-8, T=0.4)    # (m + b) b above 6144


def test_batched_block_krylov_schur_matches_dense_per_set(small):
    """Two parameter sets (Re 50 and 40, their own base flows), a block of 2
    vectors each, in one lockstep run: each set's eigenvalues equal the dense
    eigendecomposition of its own assembled propagator."""
    kw, cfg, base, T, mu_dense = small
    cfg2 = ns2d.Config(**dict(kw, Re=40.0))
    base2 = inputs.wake_like_field(16, 32, seed=8)
    M2 = dense.assemble_M(ns2d.Base.from_omega(base2, cfg2), T, cfg2)
    mu2 = np.linalg.eigvals(M2)
    mu2 = mu2[krylov.leading_order(mu2)]
    st = nsstab.Stepper(Re=[50.0, 40.0], per_set=2, nx=32, ny=16, dt=0.02)
    v0 = np.stack([inputs.gaussian_field(16, 32, seed=60 + i) for i in range(4)])
    res = st.block_arnoldi_eigs(_dev(np.stack([base, base2])), _dev(v0), m=60, nev=4, tol=1e-10, T=T,
                                max_restarts=200)
    assert len(res) == 2
    for r, mu in zip(res, (mu_dense, mu2)):
        assert r.status == nsstab.OK and r.n_conv == len(r.mu)
        assert _match(r.mu, mu[:6]) <= 1e-10
        assert r.n_matvec % 2 == 0


def test_batched_block_sets_equal_their_separate_solves():
    """Three Reynolds numbers x a block of 2 in one run against each set's
    block solve run alone (64x32 wakes); Ritz vectors of one set checked
    against M x = mu x with a plain stepper of that set."""
    kw = dict(nx=64, ny=32, dt=0.02)
    Res = [40.0, 55.0, 70.0]
    T = 0.4
    bases = np.stack([inputs.wake_like_field(32, 64, seed=70 + s) for s in range(3)])
    v0 = np.stack([inputs.gaussian_field(32, 64, seed=80 + i) for i in range(6)])
    nev = 4
    ev = torch.zeros(3 * (nev + 1), 32, 64, dtype=torch.float64, device="cuda")
    res = nsstab.Stepper(Re=Res, per_set=2, **kw).block_arnoldi_eigs(_dev(bases), _dev(v0), m=48, nev=nev,
                                                                     tol=1e-9, T=T, max_restarts=100, eigvecs=ev)
    for s in range(3):
        one = nsstab.Stepper(Re=Res[s], per_set=2, **kw).block_arnoldi_eigs(
            _dev(bases[s]), _dev(v0[2 * s:2 * s + 2]), m=48, nev=nev, tol=1e-9, T=T, max_restarts=100)
        assert res[s].n_conv == len(res[s].mu) and one.n_conv == len(one.mu)
        assert _match(res[s].mu, one.mu) <= 1e-10 and _match(one.mu, res[s].mu) <= 1e-10
    s = 1
    x = ev[s * (nev + 1)].clone()
    mx = torch.empty_like(x)
    nsstab.Stepper(Re=Res[s], **kw).apply_expTL(_dev(bases[s]), x, mx, T)
    mu = res[s].mu[0]
    ref = mu.real * x - (mu.imag * ev[s * (nev + 1) + 1] if mu.imag != 0 else 0.0)
    assert float(torch.linalg.norm(mx - ref)) <= 1e-7


def test_invalid_krylov_arguments():
    st = nsstab.Stepper(nx=16, ny=8)
    v0 = _dev(inputs.gaussian_field(8, 16, seed=1))
    base = _dev(np.zeros((8, 16)))
    for m, nev in [(1, 1), (200, 2), (10, 10)]:
        with pytest.raises(nsstab.NsstabError):
            st.arnoldi_eigs(base, v0, m=m, nev=nev, tol=1e-8, T=0.5)
    with pytest.raises(nsstab.NsstabError):
        st.arnoldi_eigs(base, torch.zeros(8, 16, dtype=torch.float64, device="cuda"), m=10, nev=2, tol=1e-8, T=0.5)


def test_double_float_arnoldi_matches_dense(small):
    kw, cfg, base, T, mu_dense = small
    st = nsstab.Stepper(precision=48, **kw)
    v0 = inputs.gaussian_field(16, 32, seed=11)
    res = st.arnoldi_eigs(_dev(base), _dev(v0), m=150, nev=4, tol=1e-10, T=T)
    assert res.status == nsstab.OK and res.n_conv == len(res.mu)
    assert _match(res.mu, mu_dense[:6]) <= 1e-10


def test_batched_block_fp32_tracks_fp64():
    """The batched block solve with the FP32 stepper: every set's leading
    eigenvalues within 1e-5 relative of the FP64 stepper's (same sets, same
    start blocks)."""
    kw = dict(nx=64, ny=32, dt=0.02, Re=[45.0, 65.0], per_set=2)
    bases = _dev(np.stack([inputs.wake_like_field(32, 64, seed=90 + s) for s in range(2)]))
    v0 = _dev(np.stack([inputs.gaussian_field(32, 64, seed=95 + i) for i in range(4)]))
    ref = nsstab.Stepper(**kw).block_arnoldi_eigs(bases, v0, m=48, nev=4, tol=1e-9, T=0.4, max_restarts=100)
    got = nsstab.Stepper(precision=32, **kw).block_arnoldi_eigs(bases, v0, m=48, nev=4, tol=1e-6, T=0.4,
                                                                max_restarts=100)
    for r, g in zip(ref, got):
        assert r.n_conv == len(r.mu) and g.n_conv == len(g.mu)
        for mu in g.mu:
            assert np.min(np.abs(r.mu - mu)) <= 1e-5 * abs(mu)
