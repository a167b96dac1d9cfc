"""rbgs_tall_update_noalloc: the tall update for callers that cannot let a
library allocate device memory (their own allocator owns HBM, or an allocation
or free on their latency path may synchronise the device).  It takes its
scratch from a fixed buffer inside the library instead of cudaMalloc.

This file is named so that pytest collects it last: a run that stops at the
first failure has then already run every other test.  The GPU test calls the
entry point through the C ABI twice in a row (the buffer keeps the first
call's contents) and checks each result against rbgs_tall_update, the
allocating entry point, on the same inputs."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2111_14641_gb300 as rbpkg
from paper_2111_14641_gb300 import rbgs as rbmod

ETOOLARGE = 9
EINVAL = 1


def _lib():
    from paper_2111_14641_gb300 import build

    build.build()
    return rbmod.load()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    """c + mb above the fixed scratch's limit is refused before any CUDA call
    (the pointers below are never dereferenced), so this runs without a GPU."""
    lib = _lib()
    kmax = rbpkg.NOALLOC_MAX_K
    fake = ctypes.c_void_p(1 << 20)
    for prec in (0, 1, 2):
        n, mb = 128, 16
        c = kmax - mb + 1
        code = lib.rbgs_tall_update_noalloc(prec, n, c, mb, fake, n, fake, n, fake, c + mb, fake, n, None, 1)
        assert code == ETOOLARGE
        # argument errors keep their own code
        assert lib.rbgs_tall_update_noalloc(prec, 0, c, mb, fake, n, fake, n, fake, c + mb, fake, n, None, 1) == EINVAL


def _dev_ld(A, dtype, ld):
    """numpy (n x m) -> column-major CUDA tensor with leading dimension ld."""
    n, m = A.shape
    buf = torch.zeros((m, ld), dtype=dtype, device="cuda")
    buf[:, :n] = torch.from_numpy(np.ascontiguousarray(A.T)).to("cuda", dtype)
    return buf.t()[:n]


def _host(T):
    return T.detach().double().cpu().numpy()


def _call_noalloc(lib, prec, Qd, Xd, Gd, out):
    n, mb = Xd.shape
    c = 0 if Qd is None else Qd.shape[1]
    code = lib.rbgs_tall_update_noalloc(rbpkg.PREC[prec], n, c, mb, 0 if Qd is None else Qd.data_ptr(),
                                        n if Qd is None else Qd.stride(1), Xd.data_ptr(), Xd.stride(1),
                                        Gd.data_ptr(), Gd.stride(1), out.data_ptr(), out.stride(1), None, 1)
    assert code == 0, rbmod.STATUS.get(code, code)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
def test_noalloc_matches_allocating_entry_point(prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = _lib()
    kmax = rbpkg.NOALLOC_MAX_K
    td = torch.float64 if prec == "fp64" else torch.float32
    # two calls in a row: the first at the largest accepted c + mb, the second
    # smaller (ragged row tail, odd block size) on the buffer the first filled
    shapes = [(1000, kmax - 50, 50), (2051, 37, 13)]
    for call, (n, c, mb) in enumerate(shapes):
        rng = np.random.default_rng(100 * call + mb)
        ld = (n + 3) // 4 * 4 + 4
        Qp = rng.standard_normal((n, c))
        X = rng.standard_normal((n, mb))
        G = rng.standard_normal((c + mb, mb))
        if prec != "fp64":
            Qp = Qp.astype(np.float32).astype(np.float64)
            X = X.astype(np.float32).astype(np.float64)
        Qd = _dev_ld(Qp, td, ld)
        Xd = _dev_ld(X, td, ld)
        Gd = _dev_ld(G, torch.float64, c + mb)
        out_na = _dev_ld(np.zeros((n, mb)), td, ld)
        out_ref = _dev_ld(np.zeros((n, mb)), td, ld)
        _call_noalloc(lib, prec, Qd, Xd, Gd, out_na)
        rbpkg.tall_update(Qd, Xd, torch.from_numpy(G), prec=prec, out=out_ref)
        torch.cuda.synchronize()
        res, ref = _host(out_na), _host(out_ref)
        scale = np.abs(np.hstack([Qp, X])).sum(axis=1, keepdims=True) * np.abs(G).max() + 1e-300
        tol = {"fp64": 1e-15 * (c + mb), "fp32": 2e-7 * (c + mb), "tf32x3": 2e-6}[prec]
        assert (np.abs(res - ref) / scale).max() <= tol, f"call {call}"
        exact = np.hstack([Qp, X]) @ G
        assert (np.abs(res - exact) / scale).max() <= tol, f"call {call}"
    # the same call once more: device memory in use must not change across it
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    _call_noalloc(lib, prec, Qd, Xd, Gd, out_na)
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0
    assert np.array_equal(_host(out_na), res)
