"""The allocation-free CGS2 entry point gives the same result as the regular one.

cgs2_orthogonalize_noalloc exists for callers that cannot allocate device
memory when they orthogonalise (a framework whose memory pool owns the
device memory and forbids side allocations, or a real-time loop that must
not take the allocator's locks); it keeps its scratch in a fixed device
array inside the library instead.  This file is collected last so that a run which
stops at the first failure has run every other test before it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1804_03859_gb300 import nsstab  # noqa: E402

pytestmark = pytest.mark.gpu


def _basis(n, j, seed):
    rng = np.random.default_rng(seed)
    V = np.linalg.qr(rng.standard_normal((n, j)))[0]
    return torch.from_numpy(np.ascontiguousarray(V.T)).cuda(), rng.standard_normal(n)


@pytest.mark.parametrize("n,j", [(131072, 64), (100003, 256), (4096, 0)])
def test_noalloc_matches_cgs2_twice_in_a_row(n, j):
    V, w0 = _basis(n, max(j, 1), seed=n + j)
    if j == 0:
        V = torch.zeros(1, dtype=torch.float64, device="cuda")
    scale = np.linalg.norm(w0)
    for call in range(2):
        w_ref = torch.from_numpy(w0 * (call + 1)).cuda()
        w_new = w_ref.clone()
        h_ref, b_ref = nsstab.cgs2_orthogonalize(V, n, j, w_ref)
        h_new, b_new = nsstab.cgs2_orthogonalize_noalloc(V, n, j, w_new)
        torch.cuda.synchronize()
        tol = 1e-12 * scale * (call + 1)
        assert np.abs(h_new - h_ref).max(initial=0.0) <= tol
        assert abs(b_new - b_ref) <= tol
        assert torch.max(torch.abs(w_new - w_ref)).item() <= tol


def test_noalloc_rejects_bases_beyond_its_fixed_scratch():
    n, j = 1024, nsstab.NOALLOC_MAX_COLS + 1
    V = torch.zeros(j, n, dtype=torch.float64, device="cuda")
    w = torch.ones(n, dtype=torch.float64, device="cuda")
    with pytest.raises(nsstab.NsstabError, match="NSSTAB_NOALLOC_MAX_COLS"):
        nsstab.cgs2_orthogonalize_noalloc(V, n, j, w)


def test_noalloc_calls_leave_device_free_memory_unchanged():
    """The defining property: after a first call (which loads the kernels and
    looks up the scratch address), further calls at the largest basis size
    allocate nothing, also from a host thread that never called before."""
    import threading

    n, j = 65536, nsstab.NOALLOC_MAX_COLS
    V, w0 = _basis(n, j, seed=11)
    w = torch.from_numpy(w0).cuda()
    nsstab.cgs2_orthogonalize_noalloc(V, n, j, w.clone())
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(4):
        w.copy_(torch.from_numpy(w0))
        nsstab.cgs2_orthogonalize_noalloc(V, n, j, w)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    errors = []

    def other_thread():
        try:
            for _ in range(2):
                nsstab.cgs2_orthogonalize_noalloc(V, n, j, w)
            torch.cuda.synchronize()
        except Exception as e:  # reported by the main thread
            errors.append(e)

    t = threading.Thread(target=other_thread)
    t.start()
    t.join()
    assert not errors, errors
    assert torch.cuda.mem_get_info()[0] == free0
