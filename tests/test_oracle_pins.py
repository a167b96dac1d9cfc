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


@pytest.mark.parametrize("kind", ["gauss", "rademacher", "srht"])
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

@pytest.mark.parametrize("variant", [4, 5, 6])
def test_rbgs_identity_sketch_is_householder_qr(variant):
    """With Theta = I (k = n) the sketched inner product is the l2 one, so the
    RBGS output is the thin QR of W with a positive diagonal."""
    W = synth.svd_matrix(96, 24, 1e3, 3)
    out = oracle.rbgs(W, 6, "identity", 96, 0, variant=variant)
    Qn, Rn = np.linalg.qr(W)
    s = np.sign(np.diag(Rn))
    np.testing.assert_allclose(out["Q"], Qn * s, atol=1e-10)
    np.testing.assert_allclose(out["R"], s[:, None] * Rn, atol=1e-12)


@pytest.mark.parametrize("kind", ["gauss", "rademacher", "srht"])
@pytest.mark.parametrize("variant", [4, 5, 6])
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
        oracle.rbgs(W, 4, "gauss", 6, 0)  # m not a multiple of mp
    with pytest.raises(ValueError):
        oracle.rbgs(W, 3, "gauss", 11, 0)  # k > n for a dense sketch
    with pytest.raises(ValueError):
        oracle.srht_samples(0, 10, 17)  # k > n'


@pytest.mark.parametrize("fname,kind,k,n,seed", [
    ("theta_srht_k5_n12_seed3.txt", "srht", 5, 12, 3),
    ("theta_rademacher_k6_n9_seed4.txt", "rademacher", 6, 9, 4),
    ("theta_gauss_k4_n7_seed5.txt", "gauss", 4, 7, 5),
])
def test_theta_golden(fname, kind, k, n, seed):
    """Stored Theta entries (tests/golden, written by make_golden.py from the
    oracle) guard the sketch convention that the CUDA side re-implements."""
    ref = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", fname))
    T = oracle.theta_dense(kind, k, n, seed)
    tol = 0.0 if kind != "gauss" else 1e-15
    np.testing.assert_allclose(T, ref, rtol=tol, atol=tol)
