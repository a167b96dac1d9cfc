"""The C-ABI library builds, loads and exports every symbol include/rbgs.h declares.
No compute call here: this file runs without a GPU."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def lib():
    from paper_2111_14641_gb300 import build as b

    path = b.build()
    return ctypes.CDLL(str(path))


def _declared():
    txt = (ROOT / "include" / "rbgs.h").read_text()
    return sorted(set(re.findall(r"^RBGS_API\s+(?:rbgs_status|void|const char\*)\s+(rbgs_\w+)\s*\(", txt, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("rbgs_qr", "rbgs_sketch_apply", "rbgs_tall_update", "rbgs_philox", "rbgs_opts_default",
                 "rbgs_release_workspace", "rbgs_version"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_matches_header():
    from paper_2111_14641_gb300 import rbgs

    assert rbgs.header_functions() == _declared()


def _struct_fields(name):
    """(type, field) pairs of `typedef struct { ... } name;` in the header, comments dropped."""
    txt = (ROOT / "include" / "rbgs.h").read_text()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", txt).group(1)
    return re.findall(r"(double|int32_t|int64_t|uint64_t|void\*|const void\*)\s+(\w+)\s*;", body)


@pytest.mark.parametrize("cname,pyname", [("rbgs_stats", "Stats"), ("rbgs_opts", "Opts")])
def test_binding_structs_match_header(cname, pyname):
    """The ctypes structures lay out the header's fields in order, with the same types."""
    from paper_2111_14641_gb300 import rbgs

    ctype = {"double": ctypes.c_double, "int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64,
             "uint64_t": ctypes.c_uint64, "void*": ctypes.c_void_p, "const void*": ctypes.c_void_p}
    want = [(f, ctype[t]) for t, f in _struct_fields(cname)]
    got = list(getattr(rbgs, pyname)._fields_)
    assert [f for f, _ in got] == [f for f, _ in want]
    assert [ctypes.sizeof(t) for _, t in got] == [ctypes.sizeof(t) for _, t in want]


def test_opts_default_and_version(lib):
    from paper_2111_14641_gb300.rbgs import Opts

    o = Opts()
    lib.rbgs_opts_default(ctypes.byref(o))
    assert (o.prec, o.ls_iters, o.reorth, o.certify, o.sync) == (0, 2, 0, 0, 1)
    assert o.reorth_tol == 1e-8
    lib.rbgs_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.rbgs_version()


def test_argument_checks_need_no_device(lib):
    """Invalid sizes are rejected before any CUDA call (RBGS_EINVAL == 1)."""
    i64 = ctypes.c_int64
    lib.rbgs_qr.argtypes = [ctypes.c_void_p, i64, i64, i64, i64, ctypes.c_int, i64, ctypes.c_uint64,
                            ctypes.c_void_p, i64, ctypes.c_void_p, i64, ctypes.c_void_p, ctypes.c_void_p]
    fake = ctypes.c_void_p(0x1000)
    other = ctypes.c_void_p(0x10000000)
    rr = ctypes.c_void_p(0x20000000)
    # no block width
    assert lib.rbgs_qr(fake, 100, 10, 100, 0, 0, 20, 0, other, 100, rr, 10, None, None) == 1
    # k < m
    assert lib.rbgs_qr(fake, 100, 8, 100, 4, 0, 4, 0, other, 100, rr, 8, None, None) == 1
    # k > n for a dense sketch
    assert lib.rbgs_qr(fake, 100, 8, 100, 4, 0, 101, 0, other, 100, rr, 8, None, None) == 1
    # ld too small
    assert lib.rbgs_qr(fake, 100, 8, 99, 4, 0, 16, 0, other, 100, rr, 8, None, None) == 1
    # null pointer
    assert lib.rbgs_qr(None, 100, 8, 100, 4, 0, 16, 0, other, 100, rr, 8, None, None) == 1
    # block size above 64
    assert lib.rbgs_qr(fake, 1000, 128, 1000, 128, 0, 256, 0, other, 1000, rr, 128, None, None) == 1
    # W and Q overlap
    assert lib.rbgs_qr(fake, 100, 8, 100, 4, 0, 16, 0, fake, 100, rr, 8, None, None) == 1
    # steps 4-5 variant other than 0, 1, 3, 4, 5 or 6
    from paper_2111_14641_gb300 import rbgs as rbmod

    o = rbmod.Opts()
    lib.rbgs_opts_default(ctypes.byref(o))
    for bad in (2, 7, -1):
        o.interblock = bad
        assert lib.rbgs_qr(fake, 100, 8, 100, 4, 0, 16, 0, other, 100, rr, 8, ctypes.byref(o), None) == 1
    # step-2 solver other than Richardson, CG or Householder
    o.interblock = 5
    for bad in (3, -1):
        o.ls = bad
        assert lib.rbgs_qr(fake, 100, 8, 100, 4, 0, 16, 0, other, 100, rr, 8, ctypes.byref(o), None) == 1


def test_krylov_argument_checks_need_no_device(lib):
    """The Sec. 5 entry points refuse bad descriptors before any CUDA call."""
    import ctypes

    from paper_2111_14641_gb300 import rbgs as rbmod

    lib = rbmod.load()  # the binding's handle: argument types declared
    bad = rbmod.Op(5, 0, 8, 8, 1.0, 1.0)          # unknown operator kind
    empty = rbmod.Op(0, 0, 0, 8, 1.0, 1.0)        # empty grid
    fake = ctypes.c_void_p(1 << 20)
    assert lib.rbgs_op_apply(ctypes.byref(bad), 0, fake, 64, 1, fake, 64, None, 1) == 1
    assert lib.rbgs_op_apply(None, 0, fake, 64, 1, fake, 64, None, 1) == 1
    assert lib.rbgs_block_arnoldi(ctypes.byref(empty), fake, 64, 2, 4, 0, 16, 0, fake, 64, fake, 8, None, None) == 1
    cyc = ctypes.c_int64(0)
    rel = (ctypes.c_double * 2)()
    good = rbmod.Op(0, 0, 8, 8, 1.0, 1.0)
    # p < 2, then k < m
    assert lib.rbgs_block_gmres(ctypes.byref(good), fake, 64, fake, 64, 2, 1, 1e-8, 10, 0, 16, 0, None,
                                ctypes.byref(cyc), ctypes.cast(rel, ctypes.c_void_p)) == 1
    assert lib.rbgs_block_fom(ctypes.byref(good), fake, 64, fake, 64, 2, 8, 1e-8, 10, 0, 8, 0, None,
                              ctypes.byref(cyc), ctypes.cast(rel, ctypes.c_void_p)) == 1


def test_rayleigh_ritz_argument_checks_need_no_device(lib):
    """rbgs_rayleigh_ritz refuses bad arguments before any CUDA call."""
    import ctypes

    from paper_2111_14641_gb300 import rbgs as rbmod

    lib = rbmod.load()
    good = rbmod.Op(0, 0, 8, 8, 1.0, 1.0)
    fake = ctypes.c_void_p(1 << 20)
    out = [(ctypes.c_double * 2)() for _ in range(3)]
    ptrs = [ctypes.cast(o, ctypes.c_void_p) for o in out]

    def call(op, mb, p, n_iter, which, k, ldx=64):
        return lib.rbgs_rayleigh_ritz(ctypes.byref(op), fake, 64, mb, p, n_iter, which, 0, k, 0, None, fake, ldx,
                                      *ptrs)

    assert call(good, 2, 1, 1, 0, 16) == 1            # p < 2
    assert call(good, 2, 4, 0, 0, 16) == 1            # no iteration
    assert call(good, 2, 4, 1, 2, 16) == 1            # which is 0 or 1
    assert call(good, 2, 4, 1, 0, 4) == 1             # k < p mb
    assert call(good, 2, 4, 1, 0, 16, ldx=10) == 1    # ldx < n
    big = rbmod.Op(0, 0, 256, 256, 1.0, 1.0)          # (p - 1) mb > RBGS_RITZ_MAX_N
    assert lib.rbgs_rayleigh_ritz(ctypes.byref(big), fake, 65536, 64, 18, 1, 0, 0, 2048, 0, None, fake, 65536,
                                  *ptrs) == 1
    assert lib.rbgs_rayleigh_ritz(None, fake, 64, 2, 4, 1, 0, 0, 16, 0, None, fake, 64, *ptrs) == 1


def test_embedding_check_argument_checks_need_no_device(lib):
    """rbgs_embedding_check refuses a missing output and bad sizes first."""
    import ctypes

    from paper_2111_14641_gb300 import rbgs as rbmod

    lib = rbmod.load()
    fake = ctypes.c_void_p(1 << 20)
    out = ctypes.c_double(0.0)
    outp = ctypes.cast(ctypes.pointer(out), ctypes.c_void_p)
    assert lib.rbgs_embedding_check(fake, 100, 8, 100, 4, 0, 16, 0, 1, None, None) == 1     # no output
    assert lib.rbgs_embedding_check(fake, 100, 8, 100, 4, 0, 101, 0, 1, None, outp) == 1    # k > n
    assert lib.rbgs_embedding_check(fake, 100, 8, 99, 4, 0, 16, 0, 1, None, outp) == 1      # ldz < n


@pytest.mark.parametrize("seed,k", [(0, 1), (6, 5), (11, 8), ((9 << 33) + 5, 2001), (3, 200)])
def test_sparse_sign_generator_matches_the_oracle(lib, seed, k):
    """The sparse-sign Theta the sketch kernels evaluate (run here on the host
    through the C ABI) has the oracle's nonzeros exactly, columns beyond 2^32
    included; the two sides implement the definition independently."""
    import numpy as np

    import oracle
    from paper_2111_14641_gb300 import rbgs as rbmod

    for j0, count in ((0, 300), ((5 << 32) + 7, 40)):
        rows, neg = rbmod.sparse_sign_columns(seed, k, j0, count)
        r_ref, s_ref = oracle.sparse_columns(seed, k, j0, count)
        assert np.array_equal(rows, r_ref)
        assert np.array_equal(neg == 1, s_ref < 0)
    with pytest.raises(rbmod.RbgsError):
        rbmod.sparse_sign_columns(seed, 0, 0, 1)


@pytest.mark.parametrize("seed", [0, 12345, (7 << 40) + 3])
def test_gaussian_generator_matches_the_oracle(lib, seed):
    """The Gaussian Theta the dense sketch kernels evaluate (their double-FP32
    Box-Muller, compiled here for the host and called through the C ABI)
    against the oracle's libm Box-Muller in FP64, entry by entry: within
    3e-14 of the pair's radius, over 640,000 entries of the leading columns
    and 4,000 entries of columns beyond 2^32."""
    import numpy as np

    import oracle
    from paper_2111_14641_gb300 import rbgs as rbmod

    k, n = 64, 10000
    T = oracle.theta_dense("gauss", k, n, seed)
    r, j = np.meshgrid(np.arange(k), np.arange(n), indexing="ij")
    G = rbmod.gaussian_entries(seed, k, r, j)
    rad = np.sqrt(T[0::2] ** 2 + T[1::2] ** 2)
    err = np.maximum(np.abs(G[0::2] - T[0::2]), np.abs(G[1::2] - T[1::2])) / rad
    assert err.max() <= 3e-14, err.max()
    # columns past 2^32 (counter word 3 holds j >> 32), both rows of each pair
    rng = np.random.default_rng(seed & 0xffff)
    jb = (1 << 32) + rng.integers(0, 1 << 40, 2000)
    rp = rng.integers(0, k // 2, 2000)
    rb2 = np.stack([2 * rp, 2 * rp + 1], axis=1).ravel()
    jb2 = np.repeat(jb, 2)
    Gb = rbmod.gaussian_entries(seed, k, rb2, jb2).reshape(-1, 2)
    Tb = oracle.theta_gauss_entries(k, seed, rb2, jb2).reshape(-1, 2)
    radb = np.sqrt((Tb ** 2).sum(axis=1))
    assert (np.abs(Gb - Tb).max(axis=1) / radb).max() <= 3e-14
    # argument checks (through the binding's declared argument types)
    lib = rbmod.load()
    assert lib.rbgs_gaussian_entries(seed, 0, None, None, 0, None) == 1           # k < 1
    bad = np.array([k], dtype=np.int64)
    out = np.zeros(1)
    assert lib.rbgs_gaussian_entries(seed, k, bad.ctypes.data, bad.ctypes.data, 1, out.ctypes.data) == 1  # r >= k
