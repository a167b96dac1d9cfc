"""Pins of the CPU oracle against things other than itself (CPU only).

Each test checks the oracle against a textbook/library routine, a closed form,
an invariant or a bound that the paper states, chosen so that a plausible slip
(a dropped term, a wrong sign, a transposed operand, a wrong index) fails one
of them.  Paper references are to Balabanov & Grigori, arXiv 2111.14641.
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.stats as sst

import oracle
import synth

U64 = 2.0 ** -53


# ---------------------------------------------------------------- generator --

def _curand_host():
    for cand in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if cand and os.path.exists(cand) if cand.startswith("/") else cand:
            try:
                return ctypes.CDLL(cand)
            except OSError:
                continue
    return None


@pytest.mark.parametrize("seed", [0, 123456789, (5 << 40) + 17])
def test_philox_matches_curand_host_generator(seed):
    """Philox4x32-10 bits equal cuRAND's host PHILOX4_32_10 generator.  Its
    output block b is philox(counter = (b div 65536, 0, b mod 65536, 0),
    key = (seed_lo, seed_hi)), which exercises counter words 0 and 2 and
    both key words."""
    lib = _curand_host()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0
    nblk = 2 * 65536 + 8
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        buf = (ctypes.c_uint * (4 * nblk))()
        assert lib.curandGenerate(gen, buf, ctypes.c_size_t(4 * nblk)) == 0
        ref = np.frombuffer(buf, dtype=np.uint32).reshape(nblk, 4)
    finally:
        lib.curandDestroyGenerator(gen)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    blocks = list(range(0, 40)) + list(range(65530, 65560)) + [99991, 131072, nblk - 1]
    for b in blocks:
        got = oracle.philox([b // 65536, 0, b % 65536, 0], key)
        np.testing.assert_array_equal(got, ref[b])


def test_philox_uniform_bytes():
    """Chi-square test of byte frequencies over the purpose-word streams."""
    words = np.concatenate([oracle.philox([i, 0, p, 0], [7, 9]) for p in range(4) for i in range(2048)])
    bytes_ = words.view(np.uint8)
    counts = np.bincount(bytes_, minlength=256)
    _, pval = sst.chisquare(counts)
    assert pval > 1e-4


# ------------------------------------------------------------------ sketches --

@pytest.mark.parametrize("q", range(0, 9))
def test_fwht_equals_dense_hadamard(q):
    """Sylvester-ordered H of order 2^q (scipy.linalg.hadamard) times x."""
    n = 2 ** q
    x = np.random.default_rng(q).standard_normal(n)
    np.testing.assert_allclose(oracle.fwht(x), sla.hadamard(n) @ x, rtol=0, atol=1e-12 * max(1, n))


@pytest.mark.parametrize("n,k,seed", [(100, 32, 5), (128, 128, 1), (1000, 60, 9), (33, 64, 2)])
def test_srht_three_ways(n, k, seed):
    """Sec. 2.3: Theta = (1/sqrt k) Samp H D with zero padding.  The entry
    definition, the fast-transform path and an explicit build from
    scipy.linalg.hadamard must all agree."""
    npad = oracle.srht_padded(n)
    assert npad >= n and npad & (npad - 1) == 0 and npad < 2 * max(n, 1)
    T = oracle.theta_dense("srht", k, n, seed)
    s = oracle.srht_samples(seed, n, k)
    assert np.all(np.diff(s) > 0) and s[0] >= 0 and s[-1] < npad
    D = oracle.srht_signs(seed, n)
    assert set(np.unique(D)) <= {-1.0, 1.0}
    Texp = sla.hadamard(npad)[s][:, :n] * D / np.sqrt(k)
    np.testing.assert_array_equal(T, Texp)
    X = np.random.default_rng(1).standard_normal((n, 3))
    np.testing.assert_allclose(oracle.theta_apply("srht", k, seed, X), T @ X, rtol=0, atol=1e-12)


def test_srht_samples_uniform_without_replacement():
    """Uniform subsampling: over many seeds every row is kept with frequency k/n'."""
    n, k, trials = 64, 16, 4000
    hits = np.zeros(n)
    for seed in range(trials):
        s = oracle.srht_samples(seed, n, k)
        assert len(np.unique(s)) == k
        hits[s] += 1
    _, pval = sst.chisquare(hits)
    assert pval > 1e-4
    assert abs(hits.sum() - trials * k) == 0


def test_gaussian_theta_distribution():
    """Gaussian sketch: i.i.d. N(0, 1/k) entries."""
    k, n = 64, 3000
    T = oracle.theta_dense("gauss", k, n, 11)
    z = (T * np.sqrt(k)).ravel()
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 0.03
    assert sst.kstest(z, "norm").pvalue > 1e-4
    # the cosine and sine branches of one Box-Muller pair are uncorrelated
    assert abs(np.corrcoef(T[0::2].ravel(), T[1::2].ravel())[0, 1]) < 0.02


def test_rademacher_theta_distribution():
    """Sec. 2.3: P(theta = 1/sqrt k) = P(theta = -1/sqrt k) = 1/2."""
    k, n = 200, 2000
    T = oracle.theta_dense("rademacher", k, n, 3)
    assert set(np.unique(T * np.sqrt(k)).round(12)) == {-1.0, 1.0}
    frac = (T > 0).mean()
    assert abs(frac - 0.5) < 5 * 0.5 / np.sqrt(T.size)
    X = np.random.default_rng(0).standard_normal((n, 4))
    np.testing.assert_allclose(oracle.theta_apply("rademacher", k, 3, X), T @ X, rtol=0, atol=1e-12)
    Tg = oracle.theta_dense("gauss", 40, 300, 5)
    Xg = np.random.default_rng(0).standard_normal((300, 2))
    np.testing.assert_allclose(oracle.theta_apply("gauss", 40, 5, Xg), Tg @ Xg, rtol=0, atol=1e-12)


def _segments(k):
    z = min(8, k)
    return z, [(s * k // z, (s + 1) * k // z) for s in range(z)]


@pytest.mark.parametrize("k", [1, 5, 8, 19, 200, 2001])
def test_sparse_sign_theta_structure(k):
    """The block construction of the sparse JL transform (Kane and Nelson
    2014): z = min(8, k) row segments, exactly one nonzero +-1/sqrt(z) per
    segment and column, so every column has unit norm.  k <= 8 leaves one row
    per segment: a dense +-1/sqrt(k) sign matrix."""
    n = 300
    z, seg = _segments(k)
    T = oracle.theta_dense("sparse", k, n, 11)
    for s, (lo, hi) in enumerate(seg):
        block = T[lo:hi]
        assert np.all((block != 0).sum(axis=0) == 1)
    assert set(np.unique(np.abs(T[T != 0]) * np.sqrt(z)).round(14)) == {1.0}
    np.testing.assert_allclose(np.linalg.norm(T, axis=0), 1.0, rtol=0, atol=1e-15)
    if k <= 8:
        assert np.all(T != 0)
    # columns beyond 2^32 take the high counter word: they differ from their low twins
    r_lo, s_lo = oracle.sparse_columns(11, k, 5, 3)
    r_hi, s_hi = oracle.sparse_columns(11, k, 5 + (1 << 32), 3)
    if k > 8:
        assert not (np.array_equal(r_lo, r_hi) and np.array_equal(s_lo, s_hi))
    for (lo, hi), col in zip(seg, r_hi.T):
        assert np.all((col >= lo) & (col < hi))


def test_sparse_sign_theta_distribution():
    """Within each segment the nonzero's row is uniform and its sign is a fair
    coin, independently over columns (chi-square and binomial bounds at about
    five standard deviations)."""
    k, n = 200, 20000
    z, seg = _segments(k)
    rows, signs = oracle.sparse_columns(3, k, 0, n)
    for s, (lo, hi) in enumerate(seg):
        size = hi - lo
        cnt = np.bincount(rows[:, s] - lo, minlength=size)
        expect = n / size
        chi2 = ((cnt - expect) ** 2 / expect).sum()
        assert chi2 < (size - 1) + 5 * np.sqrt(2 * (size - 1))
    neg = (signs < 0).mean()
    assert abs(neg - 0.5) < 5 * 0.5 / np.sqrt(signs.size)
    off = rows - np.array([lo for lo, _ in seg])[None, :]
    assert abs(np.corrcoef(off[:-1].ravel(), off[1:].ravel())[0, 1]) < 0.02
    # E[Theta^T Theta] = I: the off-diagonal inner products of distinct columns average to 0
    T = oracle.theta_dense("sparse", k, 2000, 3)
    G = T.T @ T
    off_diag = G[~np.eye(2000, dtype=bool)]
    assert abs(off_diag.mean()) < 5 * off_diag.std() / np.sqrt(off_diag.size)


def test_sparse_sign_columns_follow_the_written_definition():
    """The nonzeros restated from the raw Philox blocks (word s & 3 of the
    block with counter (j_lo, s >> 2, 4, j_hi)), for low and high column
    indices; the raw generator is pinned by the cuRAND known answers."""
    seed, k = (9 << 33) + 5, 2001
    z, seg = _segments(k)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for j0 in (0, 777, (3 << 32) + 11):
        rows, signs = oracle.sparse_columns(seed, k, j0, 4)
        for t in range(4):
            j = j0 + t
            for s, (lo, hi) in enumerate(seg):
                x = oracle.philox([j & 0xFFFFFFFF, s >> 2, 4, j >> 32], key)
                w = int(x[s & 3])
                assert rows[t, s] == lo + (w >> 1) % (hi - lo)
                assert signs[t, s] == (-1.0 if w & 1 else 1.0)


@pytest.mark.parametrize("kind", ["gauss", "rademacher", "srht", "sparse"])
def test_subspace_embedding(kind):
    """Def. 2.1: with k large against d, Theta is an eps-embedding of a fixed
    d-dimensional subspace with eps < 1/2; by Cor. 2.4 the sketch then keeps
    the singular values within (1 -+ eps)^{1/2}."""
    n, d, k = 4096, 10, 400
    U, _ = np.linalg.qr(np.random.default_rng(4).standard_normal((n, d)))
    SU = oracle.theta_apply(kind, k, 21, U)
    eps = np.linalg.norm(SU.T @ SU - np.eye(d), 2)
    assert eps < 0.5
    sv = np.linalg.svd(SU, compute_uv=False)
    assert sv.min() >= np.sqrt(1 - eps) - 1e-12 and sv.max() <= np.sqrt(1 + eps) + 1e-12


# ----------------------------------------------------------- dense routines --

@pytest.mark.parametrize("m,n", [(7, 7), (50, 13), (300, 40)])
def test_householder_qr_matches_numpy(m, n):
    A = np.random.default_rng(m).standard_normal((m, n))
    Q, R, rc = oracle.householder_qr(A)
    assert rc == 0
    Qn, Rn = np.linalg.qr(A)
    s = np.sign(np.diag(Rn))
    np.testing.assert_allclose(Q, Qn * s, atol=1e-12)
    np.testing.assert_allclose(R, s[:, None] * Rn, atol=1e-12)
    assert np.all(np.diag(R) > 0) and np.allclose(np.tril(R, -1), 0)
    np.testing.assert_allclose(Q.T @ Q, np.eye(n), atol=1e-13)


def _near_orthonormal(k, c, pert, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((k, c)))
    return U + pert * rng.standard_normal((k, c)) / np.sqrt(k)


def test_ls_householder_equals_lstsq():
    rng = np.random.default_rng(3)
    S = rng.standard_normal((80, 20))
    P = rng.standard_normal((80, 5))
    X = oracle.ls_solve(S, P, "householder")
    Xr = np.linalg.lstsq(S, P, rcond=None)[0]
    np.testing.assert_allclose(X, Xr, atol=1e-12)


@pytest.mark.parametrize("iters", [1, 2, 3, 5])
def test_ls_richardson_error_bound(iters):
    """Supplement, Richardson: ||x_j - y_j|| <= Delta^l ||y_j|| with
    Delta = ||I - S^T S||_F, y the exact normal-equation solution."""
    S = _near_orthonormal(200, 30, 0.05, 1)
    P = np.random.default_rng(2).standard_normal((200, 4))
    Y = np.linalg.lstsq(S, P, rcond=None)[0]
    delta = np.linalg.norm(np.eye(30) - S.T @ S, "fro")
    assert delta < 1
    X = oracle.ls_solve(S, P, "richardson", iters)
    for j in range(4):
        assert np.linalg.norm(X[:, j] - Y[:, j]) <= delta ** iters * np.linalg.norm(Y[:, j]) * (1 + 1e-10) + 1e-14
    # l = 1 is the sketched BCGS coefficient S^T P
    np.testing.assert_allclose(oracle.ls_solve(S, P, "richardson", 1), S.T @ P, atol=1e-13)


@pytest.mark.parametrize("iters", [1, 2, 4])
def test_ls_cg_error_bound(iters):
    """Supplement, CG on the normal equations:
    ||S (x_j - y_j)|| <= 2 Delta^l ||y_j||."""
    S = _near_orthonormal(200, 30, 0.08, 5)
    P = np.random.default_rng(6).standard_normal((200, 3))
    Y = np.linalg.lstsq(S, P, rcond=None)[0]
    delta = np.linalg.norm(np.eye(30) - S.T @ S, "fro")
    X = oracle.ls_solve(S, P, "cg", iters)
    for j in range(3):
        assert np.linalg.norm(S @ (X[:, j] - Y[:, j])) <= 2 * delta ** iters * np.linalg.norm(Y[:, j]) + 1e-13


# ---------------------------------------------------------------- RBGS ------

@pytest.mark.parametrize("variant", [1, 3, 4, 5, 6])
def test_rbgs_identity_sketch_is_householder_qr(variant):
    """With Theta = I (k = n) the sketched inner product is the l2 one, so the
    RBGS output is the thin QR of W with a positive diagonal."""
    W = synth.svd_matrix(96, 24, 1e3, 3)
    out = oracle.rbgs(W, 6, "identity", 96, 0, variant=variant)
    Qn, Rn = np.linalg.qr(W)
    s = np.sign(np.diag(Rn))
    np.testing.assert_allclose(out["Q"], Qn * s, atol=1e-10)
    np.testing.assert_allclose(out["R"], s[:, None] * Rn, atol=1e-12)


@pytest.mark.parametrize("kind", ["gauss", "rademacher", "srht", "sparse"])
@pytest.mark.parametrize("variant", [1, 3, 4, 5, 6])
def test_rbgs_reaches_closed_form(kind, variant):
    """In exact arithmetic R = R(Theta W) with a positive diagonal and
    Q = W R^{-1} (Theta Q orthonormal, W = QR, R upper triangular positive)."""
    n, m, mp, k = 1500, 24, 6, 120
    W = synth.svd_matrix(n, m, 1e3, 8)
    out = oracle.rbgs(W, mp, kind, k, 5, variant=variant, ls="householder")
    Qc, Rc, rc = oracle.rcholqr(W, kind, k, 5)
    assert rc == 0 and out["rc"] == 0
    # closed form against numpy's QR of the explicitly built Theta W
    T = oracle.theta_dense(kind, k, n, 5)
    Rn = np.linalg.qr(T @ W)[1]
    Rn = np.sign(np.diag(Rn))[:, None] * Rn
    np.testing.assert_allclose(Rc, Rn, rtol=0, atol=1e-12 * np.abs(Rn).max())
    np.testing.assert_allclose(out["R"], Rc, rtol=0, atol=1e-11 * np.abs(Rc).max())
    np.testing.assert_allclose(out["Q"], Qc, rtol=0, atol=1e-9 * np.abs(Qc).max())


@pytest.mark.parametrize("variant", [1, 3, 4, 5, 6])
@pytest.mark.parametrize("reorth", [False, True])
@pytest.mark.parametrize("m,mp", [(23, 6), (25, 8), (7, 4)])
def test_rbgs_ragged_last_block_reaches_closed_form(variant, reorth, m, mp):
    """m not a multiple of m_p: the last block holds the remaining columns.
    The closed form (R of Theta W, Q = W R^{-1}) does not depend on the
    blocking, so the ragged factorization must reach it; with Theta = I it is
    numpy's QR."""
    n, k = 1200, 100
    W = synth.svd_matrix(n, m, 1e3, m + mp)
    out = oracle.rbgs(W, mp, "srht", k, 3, variant=variant, ls="householder", reorth=reorth)
    Qc, Rc, rc = oracle.rcholqr(W, "srht", k, 3)
    assert rc == 0 and out["rc"] == 0
    np.testing.assert_allclose(out["R"], Rc, rtol=0, atol=1e-11 * np.abs(Rc).max())
    np.testing.assert_allclose(out["Q"], Qc, rtol=0, atol=1e-9 * np.abs(Qc).max())
    if reorth:
        assert out["passes2"] == (m + mp - 1) // mp - 1
    ident = oracle.rbgs(W[:200], mp, "identity", 200, 0, variant=variant)
    Qn, Rn = np.linalg.qr(W[:200])
    sg = np.sign(np.diag(Rn))
    np.testing.assert_allclose(ident["R"], sg[:, None] * Rn, atol=1e-12 * np.abs(Rn).max())


@pytest.mark.parametrize("ls,iters", [("householder", 0), ("richardson", 5), ("cg", 20)])
def test_rbgs_invariants(ls, iters):
    n, m, mp, k = 4000, 40, 8, 200
    W = synth.svd_matrix(n, m, 1e6, 2)
    out = oracle.rbgs(W, mp, "gauss", k, 1, variant=5, ls=ls, ls_iters=iters)
    Q, R = out["Q"], out["R"]
    assert np.allclose(np.tril(R, -1), 0) and np.all(np.diag(R) > 0)
    assert oracle.factorization_error(W, Q, R) < 1e-14
    fro, two = oracle.sketched_orthogonality(Q, "gauss", k, 1)
    assert fro < 1e-7
    # the oracle's own step-6 Delta is the same number
    assert abs(out["delta"] - fro) < 1e-12 + 1e-6 * fro
    # range(Q) = range(W): principal angles vanish
    ang = sla.subspace_angles(Q, W)
    assert ang.max() < 1e-8


def test_thm41_certification():
    """Thm. 4.1: if Delta, Delta~ <= 0.1 and Theta is an eps-embedding
    (eps <= 1/2) for Q and W, then
      (1+eps)^{-1/2}(1 - Delta - 0.1u) <= sigma(Q) <= (1-eps)^{-1/2}(1 + Delta + 0.1u)
    and ||W - QR||_F <= 4 u m^{3/2} ||W||_F."""
    n, m, mp, k = 6000, 48, 8, 2000
    W = synth.svd_matrix(n, m, 1e8, 12)
    out = oracle.rbgs(W, mp, "rademacher", k, 3, variant=6, ls="householder")
    Q, R = out["Q"], out["R"]
    assert out["delta"] <= 0.1 and out["delta_tilde"] <= 0.1
    Ub, _ = np.linalg.qr(W)
    SU = oracle.theta_apply("rademacher", k, 3, Ub)
    eps = np.linalg.norm(SU.T @ SU - np.eye(m), 2)
    assert eps <= 0.5
    u = 2 * U64  # unique FP64 arithmetic; the theorem's u_crs = F(m, n) u >= u
    sv = np.linalg.svd(Q, compute_uv=False)
    d = out["delta"]
    assert sv.min() >= (1 + eps) ** -0.5 * (1 - d - 0.1 * u)
    assert sv.max() <= (1 - eps) ** -0.5 * (1 + d + 0.1 * u)
    assert np.linalg.norm(W - Q @ R) <= 4 * u * m ** 1.5 * np.linalg.norm(W) * 10


def test_thm42_a_priori_bounds():
    """Thm. 4.2: Delta~ <= 6 u m^{3/2} and Delta <= 20 u m^2 cond(W) for a
    backward-stable step 2 (u_crs of unique FP64 taken as 16 u)."""
    n, m, mp, k = 5000, 40, 10, 240
    for cnd in (1e2, 1e5, 1e9):
        W = synth.svd_matrix(n, m, cnd, 31)
        out = oracle.rbgs(W, mp, "srht", k, 4, variant=5, ls="householder")
        u = 16 * U64
        assert out["delta_tilde"] <= 6 * u * m ** 1.5
        assert out["delta"] <= 20 * u * m ** 2 * cnd


@pytest.mark.parametrize("variant,two_pass_tol", [(4, 1e-12), (5, 1e-12), (6, 1e-13)])
def test_single_pass_loss_grows_with_cond_and_second_pass_removes_it(variant, two_pass_tol):
    """Single-pass RBGS loses sketched orthogonality ~ u cond(W) (MGS-like,
    Sec. 6.1); the optional second pass (an extension: re-orthogonalization,
    Sec. 1.2) brings Delta back near O(u); the l2 pre-orthogonalization of
    Alg. 6 also removes the within-block term."""
    n, m, mp, k = 3000, 30, 6, 150
    losses = []
    for cnd in (1e6, 1e9, 1e12):
        W = synth.svd_matrix(n, m, cnd, 5)
        one = oracle.rbgs(W, mp, "gauss", k, 2, variant=variant, ls="householder")
        two = oracle.rbgs(W, mp, "gauss", k, 2, variant=variant, ls="householder", reorth=True)
        losses.append(one["delta"])
        assert 1e-2 * U64 * cnd < one["delta"] < 1e3 * U64 * cnd
        assert two["delta"] < two_pass_tol
        assert two["passes2"] == m // mp - 1
        for out in (one, two):
            assert oracle.factorization_error(W, out["Q"], out["R"]) < 1e-14
    assert losses[0] < losses[1] < losses[2]


def test_ex1_matrix_factorization_error_near_machine_precision():
    """Sec. 6.1: on the numerically rank-deficient parametric matrix the
    relative error ||W - QR|| / ||W|| of RBGS stays near machine precision."""
    n, m, mp, k = 4096, 60, 10, 600
    W = synth.ex1_matrix(n, m)
    out = oracle.rbgs(W, mp, "srht", k, 1, variant=6, ls="householder")
    assert np.linalg.norm(W - out["Q"] @ out["R"], 2) / np.linalg.norm(W, 2) < 1e-14
    assert np.all(np.isfinite(out["Q"]))


def test_bad_arguments_rejected():
    W = np.zeros((10, 6))
    with pytest.raises(ValueError):
        oracle.rbgs(W, 0, "gauss", 6, 0)  # no block width
    with pytest.raises(ValueError):
        oracle.rbgs(W, 3, "gauss", 5, 0)  # k < m
    with pytest.raises(ValueError):
        oracle.rbgs(W, 3, "gauss", 11, 0)  # k > n for a dense sketch
    with pytest.raises(ValueError):
        oracle.srht_samples(0, 10, 17)  # k > n'


@pytest.mark.parametrize("fname,kind,k,n,seed", [
    ("theta_srht_k5_n12_seed3.txt", "srht", 5, 12, 3),
    ("theta_rademacher_k6_n9_seed4.txt", "rademacher", 6, 9, 4),
    ("theta_gauss_k4_n7_seed5.txt", "gauss", 4, 7, 5),
    ("theta_sparse_k19_n6_seed6.txt", "sparse", 19, 6, 6),
])
def test_theta_golden(fname, kind, k, n, seed):
    """Stored Theta entries (tests/golden, written by make_golden.py from the
    oracle) guard the sketch convention that the CUDA side re-implements."""
    ref = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", fname))
    T = oracle.theta_dense(kind, k, n, seed)
    tol = 0.0 if kind != "gauss" else 1e-15
    np.testing.assert_allclose(T, ref, rtol=tol, atol=tol)


# ------------------------------------------- Sec. 5: Arnoldi, GMRES, FOM --

def _kron_stencil(nx, ny, bx, by):
    """The convection-diffusion matrix written as a Kronecker sum of the 1-D
    central-difference operators (independent of the oracle's loop)."""
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)

    def one_d(nn, h, b):
        T = np.zeros((nn, nn))
        for i in range(nn):
            T[i, i] = 2.0 / h ** 2
            if i > 0:
                T[i, i - 1] = -1.0 / h ** 2 - b / (2 * h)
            if i + 1 < nn:
                T[i, i + 1] = -1.0 / h ** 2 + b / (2 * h)
        return T

    return np.kron(np.eye(ny), one_d(nx, hx, bx)) + np.kron(one_d(ny, hy, by), np.eye(nx))


@pytest.mark.parametrize("nx,ny,bx,by", [(6, 5, 100.0, 50.0), (9, 9, 3.0, 1.5), (4, 7, 0.0, 0.0)])
def test_stencil_matches_kronecker_form(nx, ny, bx, by):
    A = oracle.stencil5_dense(nx, ny, bx, by)
    np.testing.assert_allclose(A, _kron_stencil(nx, ny, bx, by), rtol=1e-14, atol=1e-10)


def test_stencil_eigenvalues_closed_form():
    """With cell Peclet numbers P = b h / 2 < 1 the spectrum is real:
    lambda_jl = (2/h^2) [2 - sqrt(1 - Px^2) cos(j pi h) - sqrt(1 - Py^2) cos(l pi h)]."""
    nx = ny = 12
    bx, by = 10.0, 5.0
    h = 1.0 / (nx + 1)
    px, py = bx * h / 2, by * h / 2
    ev = np.sort(np.linalg.eigvals(oracle.stencil5_dense(nx, ny, bx, by)).real)
    j = np.arange(1, nx + 1)
    lam = (2 / h ** 2) * (2 - np.sqrt(1 - px ** 2) * np.cos(j[:, None] * np.pi * h)
                          - np.sqrt(1 - py ** 2) * np.cos(j[None, :] * np.pi * h))
    np.testing.assert_allclose(ev, np.sort(lam.ravel()), rtol=1e-10)


def test_arnoldi_identity_and_sketched_orthonormality():
    """Alg. 7: A Q_(1:p-1) = Q H with H = R_(1:p,2:p), Theta Q orthonormal, B = Q_1 R_11."""
    nx, ny, mp, p = 10, 8, 3, 6
    B = synth.gaussian(nx * ny, mp, 4)
    out = oracle.rbgs_arnoldi(nx, ny, 30.0, 10.0, B, p, "gauss", 60, 2)
    Q, R = out["Q"], out["R"]
    A = _kron_stencil(nx, ny, 30.0, 10.0)
    AQ = A @ Q[:, : (p - 1) * mp]
    assert np.abs(AQ - Q @ R[:, mp:]).max() <= 1e-13 * np.abs(AQ).max()
    np.testing.assert_allclose(Q[:, :mp] @ R[:mp, :mp], B, atol=1e-13 * np.abs(B).max())
    assert np.allclose(np.tril(R, -1), 0.0)
    S = oracle.theta_apply("gauss", 60, 2, Q)
    assert np.abs(S.T @ S - np.eye(p * mp)).max() < 1e-12


def _krylov_basis(A, B, blocks):
    K = [B]
    for _ in range(blocks - 1):
        K.append(A @ K[-1])
    return np.hstack(K)


def test_gmres_identity_sketch_is_textbook_minimal_residual():
    """With Theta = I one cycle of randomized block GMRES is block GMRES: each
    column minimizes ||b - A u|| over K_(p-1)(A, B) (brute force on an
    explicit Krylov basis)."""
    nx, ny, mp, p = 6, 6, 2, 5
    n = nx * ny
    B = synth.gaussian(n, mp, 9)
    A = _kron_stencil(nx, ny, 20.0, 10.0)
    X, cyc, _ = oracle.block_krylov("gmres", nx, ny, 20.0, 10.0, B, np.zeros((n, mp)), p, "identity", n, 0, 0.0, 1)
    assert cyc == 1
    K = _krylov_basis(A, B, p - 1)
    for i in range(mp):
        y, *_ = np.linalg.lstsq(A @ K, B[:, i], rcond=None)
        u_star = K @ y
        assert np.linalg.norm(B[:, i] - A @ X[:, i]) <= np.linalg.norm(B[:, i] - A @ u_star) * (1 + 1e-8) + 1e-12
        np.testing.assert_allclose(X[:, i], u_star, rtol=1e-6, atol=1e-9 * np.abs(u_star).max())


def test_gmres_minimizes_the_sketched_residual():
    """Sec. 5.2: u_i = argmin over K_(p-1) of ||Theta (b_i - A u)||."""
    nx, ny, mp, p, k = 7, 6, 2, 5, 30
    n = nx * ny
    B = synth.gaussian(n, mp, 12)
    A = _kron_stencil(nx, ny, 15.0, 5.0)
    X, _, _ = oracle.block_krylov("gmres", nx, ny, 15.0, 5.0, B, np.zeros((n, mp)), p, "gauss", k, 5, 0.0, 1)
    T = oracle.theta_dense("gauss", k, n, 5)
    K = _krylov_basis(A, B, p - 1)
    for i in range(mp):
        y, *_ = np.linalg.lstsq(T @ A @ K, T @ B[:, i], rcond=None)
        r_star = np.linalg.norm(T @ (B[:, i] - A @ (K @ y)))
        r_got = np.linalg.norm(T @ (B[:, i] - A @ X[:, i]))
        assert r_got <= r_star * (1 + 1e-7)
        assert abs(r_got - r_star) <= 1e-7 * r_star


def test_fom_satisfies_sketched_galerkin():
    """Sec. 5.3: <Theta v, Theta r(u_i)> = 0 for all v in K_(p-1)."""
    nx, ny, mp, p, k = 7, 6, 2, 5, 30
    n = nx * ny
    B = synth.gaussian(n, mp, 13)
    A = _kron_stencil(nx, ny, 15.0, 5.0)
    X, _, _ = oracle.block_krylov("fom", nx, ny, 15.0, 5.0, B, np.zeros((n, mp)), p, "gauss", k, 6, 0.0, 1)
    T = oracle.theta_dense("gauss", k, n, 6)
    K = _krylov_basis(A, B, p - 1)
    Kq, _ = np.linalg.qr(T @ K)
    G = Kq.T @ (T @ (B - A @ X))
    assert np.abs(G).max() <= 1e-9 * np.linalg.norm(T @ B)


@pytest.mark.parametrize("method", ["gmres", "fom"])
def test_restarted_solver_reaches_direct_solution(method):
    nx, ny, mp = 10, 9, 2
    n = nx * ny
    B = synth.gaussian(n, mp, 21)
    X, cyc, rel = oracle.block_krylov(method, nx, ny, 12.0, 6.0, B, np.zeros((n, mp)), 8, "gauss", 64, 8, 1e-11, 200)
    assert rel.max() <= 1e-11 and cyc >= 1
    Xd = np.linalg.solve(_kron_stencil(nx, ny, 12.0, 6.0), B)
    assert np.abs(X - Xd).max() <= 1e-8 * np.abs(Xd).max()


# ------------------------------------------------ Alg. 8: Rayleigh-Ritz --

def _closed_form_eigs(nx, ny, bx, by):
    """Eigenvalues of the convection-diffusion stencil for cell Peclet
    numbers below 1 (separable: the 1-D tridiagonal Toeplitz spectra add)."""
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    px, py = bx * hx / 2, by * hy / 2
    ex = (2.0 - 2.0 * np.sqrt(1 - px ** 2) * np.cos(np.arange(1, nx + 1) * np.pi * hx)) / hx ** 2
    ey = (2.0 - 2.0 * np.sqrt(1 - py ** 2) * np.cos(np.arange(1, ny + 1) * np.pi * hy)) / hy ** 2
    return np.sort((ex[:, None] + ey[None, :]).ravel())


def _ritz_vectors(out, mp, p):
    """Complex Ritz pairs (mu, y) of the last iteration, recomputed from its H."""
    N = (p - 1) * mp
    H = out["R"][:, mp:]
    mu, V = np.linalg.eig(H[:N, :N])
    return oracle.ritz_select(mu, V, mp, "LR")


def test_rr_identity_sketch_is_classical_rayleigh_ritz():
    """With Theta = I the Ritz values are the eigenvalues of V^T A V for an
    orthonormal basis V of the block Krylov space K_(p-1)(A, B) (brute force
    on an explicit Krylov basis)."""
    nx, ny, bx, by, mp, p = 7, 6, 8.0, 4.0, 2, 6
    n = nx * ny
    B = synth.gaussian(n, mp, 41)
    A = _kron_stencil(nx, ny, bx, by)
    out = oracle.rayleigh_ritz(nx, ny, bx, by, B, p, 1, "LR", "identity", n, 0)
    V, _ = np.linalg.qr(_krylov_basis(A, B, p - 1))
    ev = np.linalg.eigvals(V.T @ A @ V)
    order = sorted(range(ev.size), key=lambda i: (-ev[i].real, -ev[i].imag))
    want = [ev[i] for i in order if ev[i].imag >= 0][:mp]
    got = [v for v in out["values"] if v.imag >= 0][: len(want)]
    np.testing.assert_allclose(np.array(got), np.array(want)[: len(got)], rtol=1e-9)


def test_rr_sketched_galerkin_and_residual_estimate():
    """Sec. 5.4: a Ritz pair (mu, u = Q_(1:p-1) y) satisfies the sketched
    Galerkin condition <Theta v, Theta (A u - mu u)> = 0 on range(Q_(1:p-1)),
    and ||H_(p,1:p-1) y|| equals ||Theta (A u - mu u)|| (Arnoldi identity with
    Theta Q orthonormal).  Checked with the dense Theta and operator."""
    nx, ny, bx, by, mp, p, k = 9, 7, 10.0, 5.0, 3, 6, 50
    n = nx * ny
    B = synth.gaussian(n, mp, 43)
    out = oracle.rayleigh_ritz(nx, ny, bx, by, B, p, 1, "LR", "gauss", k, 8)
    T = oracle.theta_dense("gauss", k, n, 8)
    A = _kron_stencil(nx, ny, bx, by)
    N = (p - 1) * mp
    Qn = out["Q"][:, :N]
    vals, _, vecs = _ritz_vectors(out, mp, p)
    np.testing.assert_allclose(vals, out["values"], rtol=1e-12)
    for j, (mu, y) in enumerate(zip(vals, vecs)):
        u = Qn @ y
        r = T @ (A @ u - mu * u)
        g = (T @ Qn).T @ r
        assert np.abs(g).max() <= 1e-9 * np.linalg.norm(T @ (A @ u))
        assert abs(np.linalg.norm(r) - out["resid"][j]) <= 1e-9 * np.linalg.norm(T @ (A @ u))


@pytest.mark.parametrize("which", ["LR", "SR"])
def test_rr_restarts_converge_to_closed_form_eigenvalues(which):
    """Restarted Alg. 8 on a small grid with cell Peclet numbers below 1: the
    leading Ritz value reaches the extreme eigenvalue of the closed form, its
    residual estimate vanishes, and its returned vector (unit 2-norm) is an
    eigenvector of the dense operator."""
    nx, ny, bx, by, mp, p = 10, 8, 12.0, 6.0, 3, 6
    n = nx * ny
    ev = _closed_form_eigs(nx, ny, bx, by)
    B = synth.gaussian(n, mp, 31)
    out = oracle.rayleigh_ritz(nx, ny, bx, by, B, p, 60, which, "gauss", 60, 4)
    target = ev[-1] if which == "LR" else ev[0]
    mu = out["values"][0]
    assert abs(mu.imag) == 0.0
    assert abs(mu.real - target) <= 1e-11 * ev[-1]
    assert out["resid"][0] <= 1e-9 * ev[-1]
    x = out["X"][:, 0]
    assert abs(np.linalg.norm(x) - 1.0) <= 1e-14
    A = _kron_stencil(nx, ny, bx, by)
    assert np.linalg.norm(A @ x - mu.real * x) <= 1e-8 * ev[-1]
    # the Ritz values ordered as requested, each extreme in its set
    re = [v.real for v in out["values"]]
    assert re == sorted(re, reverse=(which == "LR"))


def test_ritz_select_conventions():
    """The selection and scaling rules on a matrix with a known spectrum:
    a conjugate pair takes two columns (Re y, Im y), each y has unit norm and a
    real positive largest entry, and the last slot keeps only Re y."""
    rng = np.random.default_rng(5)
    S = rng.standard_normal((5, 5))
    D = np.zeros((5, 5))
    D[0, 0] = 5.0
    D[1:3, 1:3] = [[3.0, 2.0], [-2.0, 3.0]]     # 3 +- 2i
    D[3, 3], D[4, 4] = 1.0, -1.0
    M = S @ D @ np.linalg.inv(S)
    mu, V = np.linalg.eig(M)
    vals, Y, vecs = oracle.ritz_select(mu, V, 3, "LR")
    np.testing.assert_allclose(vals, [5.0, 3.0 + 2.0j, 3.0 - 2.0j], atol=1e-10)
    for y in vecs:
        assert abs(np.linalg.norm(y) - 1.0) < 1e-14
        j = int(np.argmax(np.abs(y)))
        assert abs(y[j].imag) < 1e-15 and y[j].real > 0
    np.testing.assert_allclose(Y[:, 1], vecs[1].real)
    np.testing.assert_allclose(Y[:, 2], vecs[1].imag)
    vals2, Y2, _ = oracle.ritz_select(mu, V, 2, "LR")
    np.testing.assert_allclose(vals2, [5.0, 3.0 + 2.0j], atol=1e-10)
    vals3, _, _ = oracle.ritz_select(mu, V, 2, "SR")
    np.testing.assert_allclose(vals3, [-1.0, 1.0], atol=1e-10)


# ------------------------------------------- the a posteriori Phi check --

@pytest.mark.parametrize("kind", ["gauss", "srht"])
def test_embedding_check_equals_dense_brute_force(kind):
    """||I - M^T M||_F with M = (Theta Z) R^{-1}, R the R factor of Phi Z, both
    sketches built as dense matrices (no RBGS involved)."""
    n, m, mp, k = 600, 12, 4, 80
    Z = synth.svd_matrix(n, m, 1e2, 71)
    got = oracle.embedding_check(Z, mp, kind, k, 5, 9)
    T = oracle.theta_dense(kind, k, n, 5)
    F = oracle.theta_dense(kind, k, n, 9)
    Rf = np.linalg.qr(F @ Z)[1]
    M = (T @ Z) @ np.linalg.inv(Rf)
    want = np.linalg.norm(np.eye(m) - M.T @ M, "fro")
    assert abs(got - want) <= 1e-10 * max(want, 1.0)
    assert 0.05 < want < 10.0   # two independent k = 80 sketches of a 12-dimensional space


def test_embedding_check_with_phi_equal_theta_is_sketched_orthogonality():
    """Phi = Theta: Theta Q_phi is orthonormal by construction, the check
    returns the sketched orthogonality of RBGS (FP64 rounding)."""
    n, m, mp, k = 800, 16, 4, 90
    Z = synth.svd_matrix(n, m, 1e3, 72)
    assert oracle.embedding_check(Z, mp, "gauss", k, 3, 3) < 1e-12


def test_embedding_check_shrinks_with_k():
    """A larger sketch embeds the same space better: the defect falls roughly
    like sqrt(m / k)."""
    n, m, mp = 4000, 10, 5
    Z = synth.svd_matrix(n, m, 1e2, 73)
    small = np.mean([oracle.embedding_check(Z, mp, "gauss", 40, s, s + 100) for s in range(4)])
    large = np.mean([oracle.embedding_check(Z, mp, "gauss", 1000, s, s + 100) for s in range(4)])
    assert large < small / 2.5


# ------------------------------------------------ Cholesky QR post-processing --

@pytest.mark.parametrize("kind", ["gauss", "srht"])
def test_cholqr_postprocess_gives_householder_qr(kind):
    """After the post-processing Q is l2-orthonormal and W = QR with a positive
    diagonal, which makes (Q, R) the unique thin QR of W: numpy's Householder
    QR up to the column signs."""
    n, m, mp, k = 2000, 24, 6, 120
    W = synth.svd_matrix(n, m, 1e4, 81)
    out = oracle.rbgs(W, mp, kind, k, 2)
    Q, R = oracle.cholqr_postprocess(out["Q"], out["R"])
    assert np.abs(Q.T @ Q - np.eye(m)).max() < 1e-13
    assert np.linalg.norm(W - Q @ R) / np.linalg.norm(W) < 1e-14
    Qn, Rn = np.linalg.qr(W)
    sg = np.sign(np.diag(Rn))
    np.testing.assert_allclose(R, sg[:, None] * Rn, atol=1e-11 * np.abs(Rn).max())
    np.testing.assert_allclose(Q, Qn * sg, atol=1e-8)


def test_cholqr_postprocess_keeps_an_orthonormal_q():
    """An l2-orthonormal Q (RBGS with Theta = I) gives R' = I."""
    W = synth.svd_matrix(300, 12, 1e2, 82)
    out = oracle.rbgs(W, 4, "identity", 300, 0)
    Q, R = oracle.cholqr_postprocess(out["Q"], out["R"])
    np.testing.assert_allclose(Q, out["Q"], atol=1e-13)
    np.testing.assert_allclose(R, out["R"], atol=1e-12 * np.abs(out["R"]).max())
