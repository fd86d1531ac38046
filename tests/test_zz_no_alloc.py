"""The scratch-free eigensolver entry point against the allocating one, on the GPU.

wgw_symm_eig_noalloc_dev is for callers that cannot allocate device memory when they
call (their device memory is reserved up front by another allocator, or they cannot
afford the synchronisation an allocation implies).  It keeps its work space in a fixed
device array shared by all calls.  This file is collected last so that a failure here
comes after every other test has run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05623_gb300 import build
    build.build()
    import paper_2203_05623_gb300 as W
    return W


def sym(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    return A + A.T


def test_noalloc_matches_allocating_entry_point_twice(W):
    import torch
    # Two calls in a row on different sizes: the second must not see the first one's leftovers.
    for n, seed in ((300, 1), (77, 2), (512, 3)):
        A = sym(n, seed)
        w_ref, Z_ref = W.wgw_symm_eig_dev(torch.from_numpy(A.copy()).cuda())
        w_out = torch.empty(n, dtype=torch.float64, device="cuda")
        Z_out = torch.empty((n, n), dtype=torch.float64, device="cuda")
        w, Z = W.wgw_symm_eig_dev(torch.from_numpy(A.copy()).cuda(), w=w_out, Z=Z_out, noalloc=True)
        torch.cuda.synchronize()
        w, Z, w_ref, Z_ref = (t.cpu().numpy() for t in (w, Z, w_ref, Z_ref))
        scale = np.max(np.abs(w_ref))
        assert np.max(np.abs(w - w_ref)) < 1e-13 * scale * n ** 0.5
        # Same kernel on the same input: columns agree (up to sign, to be safe).
        Zc, Zr = Z.T, Z_ref.T
        signs = np.sign(np.sum(Zc * Zr, axis=0))
        assert np.max(np.abs(Zc * signs - Zr)) < 1e-12 * n ** 0.5
        assert np.max(np.abs(A @ Zc - Zc * w)) < 1e-12 * scale * n ** 0.5


def test_noalloc_rejects_sizes_above_its_limit(W):
    import torch
    A = torch.zeros((513, 513), dtype=torch.float64, device="cuda")
    with pytest.raises(W.WgwError) as e:
        W.wgw_symm_eig_dev(A, noalloc=True)
    assert e.value.status == W.WGW_ERR_ARG
