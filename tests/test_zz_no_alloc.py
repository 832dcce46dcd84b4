"""The SVD entry point that allocates nothing (mpo_svd_static).

Some callers cannot call cudaMalloc when they need a factorisation, for
example code running inside an allocator's own callbacks (allocating again
would re-enter the allocator) or under a fixed memory budget granted up
front. mpo_svd_static keeps its scratch in a device array built into the
library. Here it is called through the C ABI and compared with the allocating
entry point (mpo_svd, block form) on the same inputs, twice in a row, since
every call reuses the same scratch. This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2003_13163_gb300.circuits import random_complex
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    return need_gpu()


def _matrix(r, c, seed):
    k = min(r, c)
    U = np.linalg.qr(random_complex((r, k), seed=seed))[0]
    Vh = np.linalg.qr(random_complex((c, k), seed=seed + 1))[0].conj().T
    return (U * np.exp(-0.02 * np.arange(k))[None, :]) @ Vh


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_static_scratch_svd_matches_allocating_entry(M, prec):
    import torch
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    eps = 2.2e-16 if prec == "fp64" else 1.2e-7
    for call, (r, c, seed) in enumerate([(200, 700, 1), (130, 256, 7)]):
        X = torch.tensor(_matrix(r, c, seed), dtype=dt, device="cuda")
        Xa, Xs = X.clone(), X.clone()
        wa, Ua = M.svd_rows(Xa, prec, block=True)
        ws, Us = M.svd_rows_static(Xs, prec)
        tol = 50 * eps * np.sqrt(c)
        sa = np.sort(wa.cpu().numpy().astype(np.float64))
        ss = np.sort(ws.cpu().numpy().astype(np.float64))
        np.testing.assert_allclose(np.sqrt(np.maximum(ss, 0)), np.sqrt(np.maximum(sa, 0)), atol=tol)
        # same factorisation: X = U (U^H X) with U from either entry point
        Um = Us.cpu().numpy().astype(np.complex128).T
        np.testing.assert_allclose(Um @ Xs.cpu().numpy().astype(np.complex128),
                                   X.cpu().numpy().astype(np.complex128), atol=tol)
        np.testing.assert_allclose(Xs.cpu().numpy(), Xa.cpu().numpy(), atol=tol)
        np.testing.assert_allclose(Us.cpu().numpy(), Ua.cpu().numpy(), atol=tol)


def test_static_scratch_svd_rejects_oversize(M):
    import torch
    X = torch.zeros((600, 64), dtype=torch.complex128, device="cuda")
    with pytest.raises(M.MPOError) as e:
        M.svd_rows_static(X, "fp64")
    assert e.value.code == -1 and "scratch limit" in str(e.value)


@pytest.mark.parametrize("r,c", [(512, 2048), (512, 1537)])
def test_static_scratch_svd_at_the_limit(M, r, c):
    """At the built-in limit (512 rows, 2048 columns), where the pair and
    chunk counts fill the static array exactly, and with a ragged last
    column chunk: the same factorisation as the allocating entry point."""
    import torch
    X = torch.tensor(_matrix(r, c, 11), dtype=torch.complex128, device="cuda")
    Xa, Xs = X.clone(), X.clone()
    wa, Ua = M.svd_rows(Xa, "fp64", block=True)
    ws, Us = M.svd_rows_static(Xs, "fp64")
    tol = 50 * 2.2e-16 * np.sqrt(c)
    np.testing.assert_allclose(Xs.cpu().numpy(), Xa.cpu().numpy(), atol=tol)
    np.testing.assert_allclose(Us.cpu().numpy(), Ua.cpu().numpy(), atol=tol)
    np.testing.assert_allclose(ws.cpu().numpy(), wa.cpu().numpy(), rtol=1e-12, atol=1e-14)


def test_static_scratch_svd_rejects_oversize_columns(M):
    import torch
    X = torch.zeros((64, 2049), dtype=torch.complex128, device="cuda")
    with pytest.raises(M.MPOError) as e:
        M.svd_rows_static(X, "fp64")
    assert e.value.code == -1 and "scratch limit" in str(e.value)


def test_static_scratch_svd_allocates_nothing_after_warm_up(M):
    """After a first call (which loads the module and maps the array), a call
    leaves the free device memory unchanged and updates the statistics that
    mpo_svd_last_stats reports."""
    import ctypes
    import torch
    lib = M.load_library()
    X0 = torch.tensor(_matrix(8, 16, 3), dtype=torch.complex128, device="cuda")
    M.svd_rows_static(X0.clone(), "fp64")                       # warm-up
    r, c = 300, 900
    X = torch.tensor(_matrix(r, c, 5), dtype=torch.complex128, device="cuda")
    w = torch.empty(r, dtype=torch.float64, device="cuda")
    Ut = torch.empty((r, r), dtype=torch.complex128, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    rc = lib.mpo_svd_static(r, c, X.data_ptr(), w.data_ptr(), Ut.data_ptr(), M.MPO_FP64, 0, st)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert rc == 0 and free1 == free0
    stats = M.svd_last_stats()
    assert stats["sweeps"] > 0 and stats["gram_ms"] + stats["pair_eig_ms"] + stats["apply_ms"] > 0
