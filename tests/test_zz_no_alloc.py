"""The allocation-free Gram entry point (oqr_gram_noalloc) against oqr_gram.

oqr_gram_noalloc is for callers that cannot allocate device memory: a plug-in
whose host framework's caching allocator already owns the GPU's memory, or a
real-time or embedded host that fixes its memory at start-up.  It keeps its
scratch in a fixed file-scope device array instead of a context workspace.
This file is collected last so that a failure here leaves every other test
already run; it passes both alone in a fresh process and after the rest.
"""
import ctypes

import numpy as np
import pytest

from paper_1401_5171_gb300 import inputs

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_5171_gb300 import oqr
    return torch, oqr, oqr.load()


def _call_noalloc(lib, torch, oqr, A, Z, G):
    m, n = Z.shape
    return lib.oqr_gram_noalloc(m, n, ctypes.c_void_p(A.data_ptr()), A.stride(1), ctypes.c_void_p(Z.data_ptr()),
                                Z.stride(1), ctypes.c_void_p(G.data_ptr()), G.stride(1),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_existing_gram_two_calls(env):
    torch, oqr, lib = env
    ctx = oqr.Oqr(0)
    # two calls in a row with different shapes: the second must not see the first's scratch
    for (m, n, seed) in [(3000, 300, 1), (1777, 40, 2)]:
        A_np, Z_np = inputs.paper_case(4, m, n, 1e4, 1e2, seed=seed)
        A = oqr.colmajor(torch.as_tensor(A_np).cuda())
        Z = oqr.colmajor(torch.as_tensor(Z_np).cuda())
        G_ref = ctx.oqr_gram(A, Z)
        G = oqr.empty_colmajor(n, n, A.device)
        G.fill_(float("nan"))
        assert _call_noalloc(lib, torch, oqr, A, Z, G) == oqr.OQR_OK
        torch.cuda.synchronize()
        Gh, Gr = G.cpu().numpy(), G_ref.cpu().numpy()
        scale = np.abs(Z_np).T @ np.abs(A_np) @ np.abs(Z_np)
        assert np.all(np.isfinite(Gh))
        assert np.array_equal(Gh, Gh.T)
        assert np.all(np.abs(Gh - Gr) <= 8 * m * U * scale)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, oqr, lib = env
    m, n = 1100, 1025
    A = oqr.empty_colmajor(m, m, "cuda")
    Z = oqr.empty_colmajor(m, n, "cuda")
    G = oqr.empty_colmajor(n, n, "cuda")
    assert _call_noalloc(lib, torch, oqr, A, Z, G) == oqr.OQR_ERR_UNSUPPORTED


def _padded(torch, X, pad):
    """A column-major copy of X whose leading dimension is rows + pad (an odd pad: a byte stride that
    is not a multiple of 16, which TMA cannot address, so the kernel takes its plain-load path)."""
    rows, cols = X.shape
    buf = torch.zeros((cols, rows + pad), dtype=torch.float64, device="cuda")
    buf[:, :rows] = torch.as_tensor(X.T)
    return buf.t()[:rows]


def test_noalloc_padded_leading_dimensions_plain_path(env):
    """lda, ldz and ldg padded by an odd count of doubles: the Gram kernel's plain-load path and a G
    with ldg > n, against oqr_gram on the same padded operands (same tolerance)."""
    torch, oqr, lib = env
    ctx = oqr.Oqr(0)
    m, n = 1201, 70
    A_np, Z_np = inputs.paper_case(4, m, n, 1e3, 1e2, seed=5)
    A, Z = _padded(torch, A_np, 3), _padded(torch, Z_np, 1)
    assert A.stride(1) == m + 3 and Z.stride(1) == m + 1
    G_ref = ctx.oqr_gram(A, Z)
    Gbuf = torch.full((n, n + 5), float("nan"), dtype=torch.float64, device="cuda")
    G = Gbuf.t()[:n]                                   # ldg = n + 5
    for _ in range(2):                                 # two calls in a row
        assert _call_noalloc(lib, torch, oqr, A, Z, G) == oqr.OQR_OK
        torch.cuda.synchronize()
        Gh, Gr = G.cpu().numpy(), G_ref.cpu().numpy()
        scale = np.abs(Z_np).T @ np.abs(A_np) @ np.abs(Z_np)
        assert np.all(np.isfinite(Gh)) and np.array_equal(Gh, Gh.T)
        assert np.all(np.abs(Gh - Gr) <= 8 * m * U * scale)
    ctx.close()


def test_noalloc_leaves_free_device_memory_unchanged(env):
    """After a first call (which looks up the array's address), further calls change the device's free
    memory by nothing: the entry point allocates no device memory."""
    torch, oqr, lib = env
    m, n = 2048, 128
    A_np, Z_np = inputs.paper_case(4, m, n, 1e3, 1e2, seed=6)
    A = oqr.colmajor(torch.as_tensor(A_np).cuda())
    Z = oqr.colmajor(torch.as_tensor(Z_np).cuda())
    G = oqr.empty_colmajor(n, n, "cuda")
    assert _call_noalloc(lib, torch, oqr, A, Z, G) == oqr.OQR_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _call_noalloc(lib, torch, oqr, A, Z, G) == oqr.OQR_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
