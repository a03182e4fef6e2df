"""The allocation-free CGS2 entry point gives the same result as the regular one.

cgs2_orthogonalize_noalloc exists for callers that cannot allocate device
memory when they orthogonalise (for example while another component is
capturing the stream into a CUDA graph, or inside a framework whose memory
pool forbids side allocations); it keeps its scratch in a fixed device array
inside the library instead.  This file is collected last so that a run which
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
