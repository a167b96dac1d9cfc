"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.  Paper references: Balabanov & Grigori, arXiv 2111.14641."""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2111_14641_gb300 as rb
    from paper_2111_14641_gb300 import build

    build.build()
    rb.load()
    return rb


def dev(A, dtype=torch.float64):
    """numpy (n x m) -> column-major CUDA tensor."""
    A = np.asarray(A)
    return torch.from_numpy(np.ascontiguousarray(A.T)).to("cuda", dtype).t()


def host(T):
    return T.detach().double().cpu().numpy()


# Forward-error bound for the factors (derived in the design notes, "parity
# tolerance"): R = R(Theta W) and column j of R and of Q depend only on the
# leading columns W_{:,1:j}, so a computation that is backward stable to
# O(u) (||W - QR|| / ||W|| ~ u; Thm. 4.1 for RBGS) perturbs column j by at most
# about u kappa_j, kappa_j = cond(R_{1:j,1:j}) = cond(Theta W_{:,1:j}).  The
# tests allow C u sqrt(m) kappa_j with u the unit roundoff of the storage
# (2^-24 for FP32 W and Q, 2^-53 for FP64), sqrt(m) for the growth of the
# backward error with the number of columns, and C = PARITY_C; for the
# element-wise maximum over the n rows of a column of Q also sqrt(2 ln n),
# the size of the largest of n independent errors of one standard deviation.
U32 = 2.0 ** -24
U64 = 2.0 ** -53
PARITY_C = 4.0


def col_kappas(Rref, cols=None):
    """kappa_j = cond(R_{1:j,1:j}) for the columns j (all by default)."""
    m = Rref.shape[1]
    cols = range(m) if cols is None else cols
    out = {}
    for j in cols:
        sv = np.linalg.svd(Rref[: j + 1, : j + 1], compute_uv=False)
        out[j] = sv[0] / sv[-1]
    return out


def assert_factor_parity(Q, R, Qref, Rref, u, extra=0.0, label=""):
    """Column by column: max_i |R_ij - Rref_ij| <= tol_j ||Rref_:j|| and
    max_i |Q_ij - Qref_ij| <= tol_j sqrt(2 ln n) max_i |Qref_ij|, tol_j =
    PARITY_C u sqrt(m) kappa_j + extra kappa_j (extra: a tolerance the options
    allow, e.g. the adaptive second pass's threshold).  Returns the largest
    observed ratio err_j / (u sqrt(m) kappa_j) for R, and for Q divided by
    sqrt(2 ln n)."""
    m = Rref.shape[1]
    ev = np.sqrt(2.0 * np.log(max(Q.shape[0], 2)))
    kap = col_kappas(Rref)
    worst_r = worst_q = 0.0
    for j in range(m):
        unit = u * np.sqrt(m) * kap[j]
        tol = PARITY_C * unit + extra * kap[j]
        er = np.abs(R[:, j] - Rref[:, j]).max() / np.linalg.norm(Rref[:, j])
        eq = np.abs(Q[:, j] - Qref[:, j]).max() / np.abs(Qref[:, j]).max()
        assert er <= tol, f"{label} R column {j}: {er:.3e} > {tol:.3e} (kappa_j {kap[j]:.3e})"
        assert eq <= tol * ev, f"{label} Q column {j}: {eq:.3e} > {tol * ev:.3e} (kappa_j {kap[j]:.3e})"
        worst_r, worst_q = max(worst_r, er / unit), max(worst_q, eq / (unit * ev))
    print(f"[parity] {label} max err/(u sqrt(m) kappa_j): R {worst_r:.3f}, Q {worst_q:.3f}")
    return worst_r, worst_q


# ------------------------------------------------------------------ Philox --

def test_philox_bits_match_oracle(rb):
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(257, 4), dtype=np.uint64).astype(np.uint32)
    seed = (7 << 35) + 12345
    out = rb.philox(torch.from_numpy(ctr.view(np.int32)).cuda(), seed).cpu().numpy().view(np.uint32)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(ctr.shape[0]):
        np.testing.assert_array_equal(out[i], oracle.philox(ctr[i], key))


# ---------------------------------------------------------------- sketches --

SKETCH_CASES = [
    ("gauss", 1, 1, 1), ("gauss", 100, 3, 40), ("gauss", 1000, 65, 130), ("gauss", 5000, 5, 64),
    ("rademacher", 100, 3, 40), ("rademacher", 3001, 9, 200), ("rademacher", 777, 64, 129),
    ("srht", 1, 2, 1), ("srht", 100, 3, 40), ("srht", 1000, 65, 130), ("srht", 16384, 4, 300),
    ("srht", 16385, 3, 300), ("srht", 70000, 2, 500), ("srht", 4096, 1, 4096),
]


@pytest.mark.parametrize("kind,n,c,k", SKETCH_CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sketch_matches_oracle(rb, kind, n, c, k, prec):
    """Y = Theta X (Sec. 2.3) against the oracle's Theta X."""
    seed = 1234 + n
    X = synth.gaussian(n, c, seed=n + c)
    if prec == "fp32":
        X = X.astype(np.float32).astype(np.float64)
    Y = host(rb.sketch_apply(dev(X, torch.float64 if prec == "fp64" else torch.float32), kind, k, seed, prec=prec))
    Yr = oracle.theta_apply(kind, k, seed, X)
    scale = np.linalg.norm(X, axis=0)[None, :] + 1e-300
    err = np.abs(Y - Yr) / scale
    tol = 1e-13 if prec == "fp64" else 3e-6
    assert err.max() <= tol, f"max rel err {err.max():.3e}"


@pytest.mark.parametrize("n,k", [(4096, 512), (70001, 64)])
def test_gaussian_entries_match_oracle(rb, n, k):
    """Entries of the Gaussian Theta one by one (Box-Muller pairs): with X a
    set of identity columns, column t of Y = Theta X is column j_t of Theta on
    both sides exactly (one nonzero term per sum), so this compares the two
    generators entry by entry.  Bound: 3e-14 of the pair's radius
    sqrt(z_2r^2 + z_2r+1^2), about 200 ulps of FP64, well above the device's
    double-float evaluation error (about 2^-46 of the radius) and far below
    any wrong term of the logarithm or the angle."""
    rng = np.random.default_rng(n)
    cols = np.unique(np.concatenate([[0, 1, n - 1], rng.integers(0, n, 253)]))
    X = np.zeros((n, cols.size))
    X[cols, np.arange(cols.size)] = 1.0
    seed = 99 + n
    Y = host(rb.sketch_apply(dev(X), "gauss", k, seed, prec="fp64"))
    Yr = oracle.theta_apply("gauss", k, seed, X)
    rad = np.sqrt(Yr[0::2] ** 2 + Yr[1::2] ** 2)
    err = np.maximum(np.abs(Y[0::2] - Yr[0::2]), np.abs(Y[1::2] - Yr[1::2])) / rad
    assert np.isfinite(Y).all()
    assert err.max() <= 3e-14, f"max error {err.max():.3e} of the pair radius"


# --------------------------------------------------------------- tall ops ---

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,c,mb", [(1, 0, 1), (129, 5, 3), (1000, 64, 16), (4097, 200, 50), (300, 0, 64)])
@pytest.mark.parametrize("inplace", [False, True])
def test_tall_update_matches_numpy(rb, prec, n, c, mb, inplace):
    """Qout = [Qprev | X] G, the fused step 3 + triangular solve of Alg. 5."""
    rng = np.random.default_rng(n + c + mb)
    Qp = rng.standard_normal((n, c))
    X = rng.standard_normal((n, mb))
    G = rng.standard_normal((c + mb, mb))
    td = torch.float64 if prec == "fp64" else torch.float32
    if prec == "fp32":
        Qp = Qp.astype(np.float32).astype(np.float64)
        X = X.astype(np.float32).astype(np.float64)
    Qd = dev(Qp, td) if c > 0 else None
    Xd = dev(X, td)
    out = Xd if inplace else None
    res = host(rb.tall_update(Qd, Xd, torch.from_numpy(G), prec=prec, out=out))
    ref = np.hstack([Qp, X]) @ G
    scale = np.abs(np.hstack([Qp, X])).sum(axis=1, keepdims=True) * np.abs(G).max() + 1e-300
    tol = 1e-15 * (c + mb) if prec == "fp64" else 2e-7 * (c + mb)
    assert (np.abs(res - ref) / scale).max() <= tol


# ------------------------------------------------------------------ RBGS ----

def _check_qr_against_oracle(rb, W, mb, kind, k, seed, l, reorth, cond, prec="fp64"):
    td = torch.float64 if prec == "fp64" else torch.float32
    if prec != "fp64":
        W = W.astype(np.float32).astype(np.float64)
    Qd, Rd, st = rb.rbgs_qr(dev(W, td), mb, kind, k, seed, prec=prec, ls_iters=l, reorth=int(reorth), certify=True)
    Q, R = host(Qd), host(Rd)
    ref = oracle.rbgs(W, mb, kind, k, seed, variant=5, ls="richardson", ls_iters=l, reorth=reorth, ls_iters_first=1)
    assert np.allclose(np.tril(R, -1), 0.0) and np.all(np.diag(R) > 0)
    fact = oracle.factorization_error(W, Q, R)
    ortho = oracle.sketched_orthogonality(Q, kind, k, seed)[0]
    return Q, R, ref, fact, ortho, st


QR_CASES = [
    # n, m, mb, kind, k
    (3000, 32, 8, "gauss", 160),
    (777, 12, 3, "rademacher", 60),
    (5000, 64, 64, "gauss", 128),
    (4096, 16, 1, "srht", 64),
    (3000, 40, 10, "srht", 200),
    (20000, 48, 16, "srht", 300),
    (1000, 6, 2, "gauss", 6),
]


@pytest.mark.parametrize("n,m,mb,kind,k", QR_CASES)
@pytest.mark.parametrize("reorth", [False, True])
def test_rbgs_fp64_matches_oracle(rb, n, m, mb, kind, k, reorth):
    cond = 1e4
    W = synth.svd_matrix(n, m, cond, n + m)
    Q, R, ref, fact, ortho, st = _check_qr_against_oracle(rb, W, mb, kind, k, 99, 3, reorth, cond)
    tol = 1e-13 * cond
    assert np.abs(R - ref["R"]).max() <= tol * np.abs(ref["R"]).max()
    assert np.abs(Q - ref["Q"]).max() <= tol * np.abs(ref["Q"]).max()
    assert fact < 1e-14
    assert abs(st.delta - ref["delta"]) <= 1e-10 + 1e-3 * ref["delta"]
    assert st.passes2 == (m // mb - 1 if reorth else 0)


@pytest.mark.parametrize("reorth", [False, True])
def test_fp64_second_cholesky_round_only_where_needed(rb, reorth):
    """FP64 sketch space: Alg. 5's Cholesky QR takes its second round only where
    the first round's R has ||R||_F ||R^{-1}||_F > 4 m_p.  Columns u_j sigma_j
    make every block as ill-conditioned as its sigmas (about 10^2.9), so each
    first pass that settles a block needs the second round, while the second
    projection pass (a nearly orthonormal block) does not; the factors match
    the oracle's either way."""
    n, m, mb, k = 4000, 32, 16, 200
    rng = np.random.Generator(np.random.PCG64(11))
    U, _ = np.linalg.qr(rng.standard_normal((n, m)))
    cond = 1e6
    W = np.asfortranarray(U * synth.sigmas(m, cond))
    Q, R, ref, fact, ortho, st = _check_qr_against_oracle(rb, W, mb, "gauss", k, 99, 3, reorth, cond)
    tol = 1e-13 * cond
    assert np.abs(R - ref["R"]).max() <= tol * np.abs(ref["R"]).max()
    assert np.abs(Q - ref["Q"]).max() <= tol * np.abs(ref["Q"]).max()
    assert fact < 1e-14
    assert st.chol_rounds2 == (1 if reorth else m // mb)


def test_fp64_single_cholesky_round_when_well_conditioned(rb):
    """A well-conditioned W (cond 2) needs no second Cholesky QR round in FP64;
    the FP32 sketch space, whose first round is shifted, always takes it."""
    n, m, mb, k = 3000, 40, 10, 200
    W = synth.svd_matrix(n, m, 2.0, 21)
    _, _, ref, fact, ortho, st = _check_qr_against_oracle(rb, W, mb, "srht", k, 3, 1, False, 2.0)
    assert st.chol_rounds2 == 0 and fact < 1e-14 and ortho < 1e-13
    _, _, st32 = rb.rbgs_qr(dev(W, torch.float32), mb, "srht", k, 3, prec="fp32", ls_iters=1, reorth=0)
    assert st32.chol_rounds2 == m // mb


@pytest.mark.parametrize("prec", ["fp64", "f16x3", "tf32x3", "fp32"])
@pytest.mark.parametrize("interblock", [1, 3])
@pytest.mark.parametrize("reorth", [0, 1])
def test_rbgs_column_by_column_interblock_matches_oracle(rb, prec, interblock, reorth):
    """Steps 4-5 one column at a time after the projection: single-vector RGS
    (1, explicit sketches) or vRCholeskyQR (3, Alg. 3, implicit sketches),
    against the oracle's; a ragged last block included."""
    n, m, mb, kind, k = 3000, 44, 16, "srht", 200
    cond = 1e4 if prec == "fp64" else 1e3
    W = synth.svd_matrix(n, m, cond, 78)
    if prec != "fp64":
        W = W.astype(np.float32).astype(np.float64)
    td = torch.float64 if prec == "fp64" else torch.float32
    Qd, Rd, st = rb.rbgs_qr(dev(W, td), mb, kind, k, 5, prec=prec, ls_iters=3, reorth=reorth, interblock=interblock,
                            fine=prec != "fp64")
    Q, R = host(Qd), host(Rd)
    ref = oracle.rbgs(W, mb, kind, k, 5, variant=interblock, ls="richardson", ls_iters=3, reorth=bool(reorth),
                      ls_iters_first=1)
    assert np.allclose(np.tril(R, -1), 0.0) and np.all(np.diag(R) > 0)
    fact = oracle.factorization_error(W, Q, R)
    ortho = oracle.sketched_orthogonality(Q, kind, k, 5)[0]
    if prec == "fp64":
        tol = 1e-12 * cond
        assert np.abs(R - ref["R"]).max() <= tol * np.abs(ref["R"]).max()
        assert np.abs(Q - ref["Q"]).max() <= tol * np.abs(ref["Q"]).max()
        assert fact < 1e-14 and ortho < 1e-12
    else:
        assert fact < 2e-6 and ortho < (1e-4 if reorth else 1e-3)
        assert_factor_parity(Q, R, ref["Q"], ref["R"], U32, label=f"interblock {interblock} {prec} reorth {reorth}")


@pytest.mark.parametrize("prec", ["fp64", "f16x3", "tf32x3"])
@pytest.mark.parametrize("reorth", [0, 1])
def test_rbgs_alg4_matches_oracle(rb, prec, reorth):
    """Steps 4-5 by Alg. 4 (RCholeskyQR on the explicit sketch Theta Q'_i:
    projection, sketch, Cholesky QR, in-place scaling by R_ii^{-1}) against
    the oracle's Alg. 4."""
    n, m, mb, kind, k = 3000, 48, 16, "srht", 200
    cond = 1e4 if prec == "fp64" else 1e3
    W = synth.svd_matrix(n, m, cond, 77)
    if prec != "fp64":
        W = W.astype(np.float32).astype(np.float64)
    td = torch.float64 if prec == "fp64" else torch.float32
    Qd, Rd, st = rb.rbgs_qr(dev(W, td), mb, kind, k, 5, prec=prec, ls_iters=3, reorth=reorth, interblock=4,
                            certify=True, fine=prec != "fp64")
    Q, R = host(Qd), host(Rd)
    ref = oracle.rbgs(W, mb, kind, k, 5, variant=4, ls="richardson", ls_iters=3, reorth=bool(reorth),
                      ls_iters_first=1)
    assert np.allclose(np.tril(R, -1), 0.0) and np.all(np.diag(R) > 0)
    fact = oracle.factorization_error(W, Q, R)
    ortho = oracle.sketched_orthogonality(Q, kind, k, 5)[0]
    if prec == "fp64":
        tol = 1e-13 * cond
        assert np.abs(R - ref["R"]).max() <= tol * np.abs(ref["R"]).max()
        assert np.abs(Q - ref["Q"]).max() <= tol * np.abs(ref["Q"]).max()
        assert fact < 1e-14 and ortho < 1e-12
    else:
        assert fact < 2e-6 and ortho < (1e-4 if reorth else 1e-3)
        assert_factor_parity(Q, R, ref["Q"], ref["R"], U32, label=f"alg4 {prec} reorth {reorth}")
    if reorth:
        assert st.passes2 == m // mb - 1


@pytest.mark.parametrize("prec", ["fp64", "f16x3", "tf32x3", "fp32"])
@pytest.mark.parametrize("reorth", [0, 1])
def test_rbgs_alg4_triangular_solve_matches_oracle(rb, prec, reorth):
    """Alg. 4 with Q_i = Q'_i R_ii^{-1} by a row-wise triangular solve
    (opts.trsm) instead of the explicit inverse: the same factorization as the
    oracle's Alg. 4, ragged last block included."""
    n, m, mb, kind, k = 3000, 45, 16, "srht", 200
    cond = 1e4 if prec == "fp64" else 1e3
    W = synth.svd_matrix(n, m, cond, 71)
    if prec != "fp64":
        W = W.astype(np.float32).astype(np.float64)
    td = torch.float64 if prec == "fp64" else torch.float32
    ld = (n + 3) // 4 * 4
    Qd, Rd, st = rb.rbgs_qr(dev_ld(W, td, ld), mb, kind, k, 5, prec=prec, ls_iters=3, reorth=reorth, interblock=4,
                            trsm=True, Q=dev_ld(np.zeros((n, m)), td, ld), fine=prec != "fp64")
    Q, R = host(Qd), host(Rd)
    ref = oracle.rbgs(W, mb, kind, k, 5, variant=4, ls="richardson", ls_iters=3, reorth=bool(reorth),
                      ls_iters_first=1)
    assert np.allclose(np.tril(R, -1), 0.0) and np.all(np.diag(R) > 0)
    fact = oracle.factorization_error(W, Q, R)
    if prec == "fp64":
        assert_factor_parity(Q, R, ref["Q"], ref["R"], U64, label=f"alg4 trsm {prec} reorth {reorth}")
        assert fact < 1e-15
    else:
        assert fact < 2e-7
        assert_factor_parity(Q, R, ref["Q"], ref["R"], U32, label=f"alg4 trsm {prec} reorth {reorth}")


@pytest.mark.parametrize("prec,fine", [("f16x3", 1), ("f16x3", 2), ("fp64", 0)])
def test_triangular_solve_keeps_near_duplicate_columns_well_conditioned(rb, prec, fine):
    """Columns that nearly repeat earlier ones at the FP32 rounding level (the
    many-small-problems workload) make a block's R_ii about as ill-conditioned
    as 1/u_32.  With the explicit inverse the mixed path loses W = QR and
    cond(Q); with the row-wise triangular solve, Alg. 4's explicit sketch and
    the second pass it keeps ||W - QR|| / ||W|| at the FP32 level and
    cond(Q) = O(1) (the regime of the paper's first experiment).  FP64 gains
    the FP64 level of W = QR."""
    n, m, mb = 20000, 128, 16
    td = torch.float32 if prec == "f16x3" else torch.float64
    W = synth.near_duplicate_matrix_torch(n, m, 11, device="cuda", dtype=td)
    Wh = host(W)
    out = {}
    for trsm in (True, False):
        Q, R, st = rb.rbgs_qr(W, mb, "gauss", 2 * m, 7, prec=prec, ls_iters=1, reorth=1, interblock=4, trsm=trsm,
                              fine=fine)
        Qh, Rh = host(Q), host(R)
        sv = np.linalg.svd(Qh, compute_uv=False)
        out[trsm] = (oracle.factorization_error(Wh, Qh, Rh), sv[0] / sv[-1])
    print(f"[near-duplicates] {prec}: trsm {out[True]}, explicit inverse {out[False]}")
    if prec == "f16x3":
        assert out[True][0] < 1e-6 and out[True][1] < 10.0
        assert out[False][1] > 1e3  # the explicit inverse's failure, for contrast
    else:
        assert out[True][0] < 1e-14 and out[True][1] < 10.0


@pytest.mark.parametrize("prec", ["fp64", "f16x3", "fp32"])
@pytest.mark.parametrize("reorth,m", [(0, 48), (1, 48), (2, 48), (1, 45)])
def test_rbgs_alg6_matches_oracle(rb, prec, reorth, m):
    """Steps 4-5 by Alg. 6 (an l2 QR of Q'_i by Cholesky QR twice, then Alg. 4
    on its orthonormal factor, R_ii = R'' R') against the oracle's Alg. 6
    (Householder l2 QR with a positive diagonal: the same thin QR), ragged
    last block included."""
    n, mb, kind, k = 3000, 16, "srht", 200
    cond = 1e4 if prec == "fp64" else 1e3
    W = synth.svd_matrix(n, m, cond, 78)
    if prec != "fp64":
        W = W.astype(np.float32).astype(np.float64)
    td = torch.float64 if prec == "fp64" else torch.float32
    Qd, Rd, st = rb.rbgs_qr(dev(W, td), mb, kind, k, 5, prec=prec, ls_iters=3, reorth=reorth, interblock=6,
                            certify=True, fine=prec != "fp64")
    Q, R = host(Qd), host(Rd)
    ref = oracle.rbgs(W, mb, kind, k, 5, variant=6, ls="richardson", ls_iters=3, reorth=bool(reorth),
                      ls_iters_first=1 if reorth == 1 else 0)
    assert np.allclose(np.tril(R, -1), 0.0) and np.all(np.diag(R) > 0)
    fact = oracle.factorization_error(W, Q, R)
    ortho = oracle.sketched_orthogonality(Q, kind, k, 5)[0]
    if prec == "fp64":
        if reorth != 2:
            tol = 1e-13 * cond
            assert np.abs(R - ref["R"]).max() <= tol * np.abs(ref["R"]).max()
            assert np.abs(Q - ref["Q"]).max() <= tol * np.abs(ref["Q"]).max()
        # the adaptive second pass is skipped where the block's coefficients on
        # the basis are below reorth_tol (1e-8), which then bounds the defect
        assert fact < 1e-14 and ortho < (1e-8 if reorth == 2 else 1e-12)
        assert 0 <= st.passes2 <= (m + mb - 1) // mb - 1
    else:
        assert fact < 2e-6 and ortho < (1e-4 if reorth else 1e-3)
        if reorth != 2:
            assert_factor_parity(Q, R, ref["Q"], ref["R"], U32, label=f"alg6 {prec} reorth {reorth} m {m}")
    if reorth == 1:
        assert st.passes2 == (m + mb - 1) // mb - 1


@pytest.mark.parametrize("prec", ["fp64", "fp32", "f16x3", "tf32x3"])
@pytest.mark.parametrize("interblock", [5, 4])
@pytest.mark.parametrize("m,mb,reorth", [(50, 16, 0), (60, 50, 1), (9, 4, 1)])
def test_rbgs_ragged_last_block_matches_oracle(rb, prec, interblock, m, mb, reorth):
    """m not a multiple of m_p: the last block takes the remaining columns
    (a narrower tall update, sketch and Cholesky QR) on every precision path."""
    n, kind, k = 2048, "srht", 4 * m
    cond = 1e4 if prec == "fp64" else 1e3
    W = synth.svd_matrix(n, m, cond, 90 + m)
    if prec != "fp64":
        W = W.astype(np.float32).astype(np.float64)
    td = torch.float64 if prec == "fp64" else torch.float32
    Qd, Rd, st = rb.rbgs_qr(dev(W, td), mb, kind, k, 7, prec=prec, ls_iters=3, reorth=reorth,
                            interblock=interblock, fine=prec != "fp64")
    Q, R = host(Qd), host(Rd)
    ref = oracle.rbgs(W, mb, kind, k, 7, variant=interblock, ls="richardson", ls_iters=3, reorth=bool(reorth),
                      ls_iters_first=1)
    assert np.allclose(np.tril(R, -1), 0.0) and np.all(np.diag(R) > 0)
    fact = oracle.factorization_error(W, Q, R)
    ortho = oracle.sketched_orthogonality(Q, kind, k, 7)[0]
    if prec == "fp64":
        tol = 1e-13 * cond
        assert np.abs(R - ref["R"]).max() <= tol * np.abs(ref["R"]).max()
        assert np.abs(Q - ref["Q"]).max() <= tol * np.abs(ref["Q"]).max()
        assert fact < 1e-14 and ortho < 1e-12
    else:
        assert fact < 2e-6 and ortho < (1e-4 if reorth else 1e-3)
        assert_factor_parity(Q, R, ref["Q"], ref["R"], U32,
                             label=f"ragged {prec} interblock {interblock} m {m} mb {mb} reorth {reorth}")
    if reorth:
        assert st.passes2 == (m + mb - 1) // mb - 1


def test_c1_config_fp64(rb):
    """n = 1e4, m = 100, m_p = 10, Gaussian k = 200, cond(W) = 1e8:
    ||W - QR||/||W|| <= 1e-13 and sketched orthogonality <= 1e-12 with the
    second pass; the single pass (Alg. 2 as written) loses ~u cond(W)."""
    n, m, mb, k = 10_000, 100, 10, 200
    W = synth.svd_matrix(n, m, 1e8, 7)
    Q, R, ref, fact, ortho, st = _check_qr_against_oracle(rb, W, mb, "gauss", k, 1, 3, True, 1e8)
    assert fact <= 1e-13
    assert ortho <= 1e-12
    assert np.linalg.norm(R - ref["R"]) <= 1e-7 * np.linalg.norm(ref["R"])
    Q1, R1, ref1, fact1, ortho1, _ = _check_qr_against_oracle(rb, W, mb, "gauss", k, 1, 3, False, 1e8)
    assert fact1 <= 1e-13
    assert 1e-12 < ortho1 < 1e-5
    # the single-pass loss is rounding noise of size ~u cond(W): same order as the oracle's
    assert 0.1 < ortho1 / ref1["delta"] < 10


@pytest.mark.parametrize("kind", ["gauss", "srht"])
def test_rbgs_fp32_path(rb, kind):
    """FP32 storage, SIMT FP32 tall product: errors at u_fp32 * cond level."""
    n, m, mb, k = 6000, 48, 8, 240
    cond = 1e3
    W = synth.svd_matrix(n, m, cond, 3)
    Q, R, ref, fact, ortho, st = _check_qr_against_oracle(rb, W, mb, kind, k, 5, 3, True, cond, prec="fp32")
    assert fact < 1e-6
    assert ortho < 1e-4
    assert_factor_parity(Q, R, ref["Q"], ref["R"], U32, label=f"fp32 simt {kind}")


def test_breakdown_reported(rb):
    """A zero block makes R_ii singular: the call reports RBGS_EBREAKDOWN
    through its return code (no device fault)."""
    W = synth.gaussian(500, 8, 1)
    W[:, 4:] = 0.0
    with pytest.raises(rb.RbgsError) as e:
        rb.rbgs_qr(dev(W), 4, "gauss", 32, 0, prec="fp64")
    assert e.value.code == 4


def test_invalid_arguments(rb):
    W = dev(synth.gaussian(100, 8, 1))
    with pytest.raises(rb.RbgsError):
        rb.rbgs_qr(W, 65, "gauss", 16, 0, prec="fp64")    # mb > 64
    with pytest.raises(rb.RbgsError):                       # the column-by-column variants need reorth 0 or 1
        rb.rbgs_qr(W, 4, "gauss", 16, 0, prec="fp64", reorth=2, interblock=3)
    with pytest.raises(rb.RbgsError):
        rb.rbgs_qr(W, 4, "gauss", 101, 0, prec="fp64")    # k > n
    with pytest.raises(rb.RbgsError):
        rb.rbgs_qr(W, 4, "srht", 129, 0, prec="fp64")     # k > n'


# -------------------------------------------------- tensor-core (tcgen05) ---

def dev_ld(A, dtype, ld):
    """numpy (n x m) -> column-major CUDA tensor with leading dimension ld."""
    A = np.asarray(A)
    n, m = A.shape
    buf = torch.zeros((m, ld), dtype=dtype, device="cuda")
    buf[:, :n] = torch.from_numpy(np.ascontiguousarray(A.T)).to("cuda", dtype)
    return buf.t()[:n]


@pytest.mark.parametrize("n,c,mb", [(1, 0, 1), (128, 0, 50), (129, 5, 3), (1000, 64, 16), (4097, 200, 50),
                                    (300, 0, 64), (2000, 950, 50), (513, 33, 64)])
@pytest.mark.parametrize("inplace", [False, True])
def test_tall_update_tc_matches_numpy(rb, n, c, mb, inplace):
    """3xTF32 tcgen05 product: Qout = [Qprev | X] G with FP32-level accuracy."""
    rng = np.random.default_rng(7 * n + c + mb)
    ld = (n + 3) // 4 * 4 + 4
    Qp = rng.standard_normal((n, c)).astype(np.float32).astype(np.float64)
    X = rng.standard_normal((n, mb)).astype(np.float32).astype(np.float64)
    G = rng.standard_normal((c + mb, mb))
    Qd = dev_ld(Qp, torch.float32, ld) if c > 0 else None
    Xd = dev_ld(X, torch.float32, ld)
    out = Xd if inplace else dev_ld(np.zeros((n, mb)), torch.float32, ld)
    res = host(rb.tall_update(Qd, Xd, torch.from_numpy(G), prec="tf32x3", out=out))
    ref = np.hstack([Qp, X]) @ G
    scale = np.abs(np.hstack([Qp, X])).sum(axis=1, keepdims=True) * np.abs(G).max() + 1e-300
    assert (np.abs(res - ref) / scale).max() <= 2e-6


@pytest.mark.parametrize("kind", ["gauss", "srht"])
@pytest.mark.parametrize("reorth", [False, True])
@pytest.mark.parametrize("fine", [False, True])
def test_rbgs_tf32x3_matches_oracle(rb, kind, reorth, fine):
    """fine=True keeps the sketch-space steps in FP64 (the paper's u_fine)."""
    n, m, mb, k = 6000, 48, 8, 240
    cond = 1e3
    W = synth.svd_matrix(n, m, cond, 3).astype(np.float32).astype(np.float64)
    Wd = dev_ld(W, torch.float32, n + 4)
    Qd = dev_ld(np.zeros((n, m)), torch.float32, n + 4)
    _, Rd, st = rb.rbgs_qr(Wd, mb, kind, k, 5, prec="tf32x3", ls_iters=3, reorth=int(reorth), Q=Qd, certify=True,
                           fine=fine)
    Q, R = host(Qd), host(Rd)
    ref = oracle.rbgs(W, mb, kind, k, 5, variant=5, ls="richardson", ls_iters=3, reorth=reorth, ls_iters_first=1)
    assert np.allclose(np.tril(R, -1), 0.0) and np.all(np.diag(R) > 0)
    assert oracle.factorization_error(W, Q, R) < 2e-6
    ortho = oracle.sketched_orthogonality(Q, kind, k, 5)[0]
    assert ortho < (1e-4 if reorth else 1e-3)
    assert_factor_parity(Q, R, ref["Q"], ref["R"], U32, label=f"tf32x3 {kind} reorth {reorth} fine {fine}")
    assert st.passes2 == (m // mb - 1 if reorth else 0)


# ------------------------------------------- FP16 hi/lo split tensor path --

@pytest.mark.parametrize("n,c,mb", [(1, 0, 1), (128, 0, 50), (129, 5, 3), (1000, 64, 16), (4097, 200, 50),
                                    (300, 0, 64), (2000, 950, 50), (513, 33, 64), (700, 130, 7)])
@pytest.mark.parametrize("inplace", [False, True])
def test_tall_update_f16x3_matches_numpy(rb, n, c, mb, inplace):
    """FP16 hi/lo split tcgen05 product (power-of-two column scales):
    Qout = [Qprev | X] G with FP32-level accuracy."""
    rng = np.random.default_rng(11 * n + c + mb)
    ld = (n + 3) // 4 * 4 + 4
    Qp = rng.standard_normal((n, c)).astype(np.float32).astype(np.float64)
    X = (rng.standard_normal((n, mb)) * np.logspace(0, -6, mb)).astype(np.float32).astype(np.float64)
    G = rng.standard_normal((c + mb, mb)) * np.logspace(0, 5, mb)
    Qd = dev_ld(Qp, torch.float32, ld) if c > 0 else None
    Xd = dev_ld(X, torch.float32, ld)
    out = Xd if inplace else dev_ld(np.zeros((n, mb)), torch.float32, ld)
    res = host(rb.tall_update(Qd, Xd, torch.from_numpy(G), prec="f16x3", out=out))
    ref = np.hstack([Qp, X]) @ G
    scale = np.abs(np.hstack([Qp, X])) @ np.abs(G) + 1e-300
    assert (np.abs(res - ref) / scale).max() <= 2e-6


F16_QR_CASES = [
    # n, m, mb, kind, k
    (6000, 48, 8, "gauss", 240),
    (3000, 150, 50, "srht", 400),
    (5000, 128, 64, "srht", 300),
    (2049, 39, 13, "rademacher", 120),
]


@pytest.mark.parametrize("n,m,mb,kind,k", F16_QR_CASES)
@pytest.mark.parametrize("reorth", [0, 1, 2])
@pytest.mark.parametrize("fine", [False, True])
def test_rbgs_f16x3_matches_oracle(rb, n, m, mb, kind, k, reorth, fine):
    """RBGS with the pre-split basis: block boundaries that do not fall on the
    64-column chunks, all second-pass modes, FP32 or FP64 sketch space."""
    cond = 1e3
    W = synth.svd_matrix(n, m, cond, 5 + m).astype(np.float32).astype(np.float64)
    ld = (n + 3) // 4 * 4 + 4  # the tensor-core paths need ld % 4 == 0
    Wd = dev_ld(W, torch.float32, ld)
    Qd = dev_ld(np.zeros((n, m)), torch.float32, ld)
    _, Rd, st = rb.rbgs_qr(Wd, mb, kind, k, 5, prec="f16x3", ls_iters=3, reorth=reorth, reorth_tol=1e-6, Q=Qd,
                           certify=True, fine=fine)
    Q, R = host(Qd), host(Rd)
    ref = oracle.rbgs(W, mb, kind, k, 5, variant=5, ls="richardson", ls_iters=3, reorth=bool(reorth),
                      ls_iters_first=1)
    assert np.allclose(np.tril(R, -1), 0.0) and np.all(np.diag(R) > 0)
    assert oracle.factorization_error(W, Q, R) < 2e-6
    ortho = oracle.sketched_orthogonality(Q, kind, k, 5)[0]
    assert ortho < (1e-4 if reorth else 1e-3)
    # the adaptive pass (reorth 2) may skip a block whose coefficients on the
    # basis are below reorth_tol, which the oracle (second pass always) takes
    assert_factor_parity(Q, R, ref["Q"], ref["R"], U32, extra=1e-6 if reorth == 2 else 0.0,
                         label=f"f16x3 n {n} m {m} mb {mb} {kind} reorth {reorth} fine {fine}")
    if reorth == 1:
        assert st.passes2 == m // mb - 1


# ------------------------------------- several 128-row tiles per CTA --

@pytest.mark.parametrize("prec", ["f16x3", "tf32x3"])
@pytest.mark.parametrize("fine", [True, False, 2])
@pytest.mark.parametrize("reorth", [0, 1])
def test_rbgs_tensor_core_tile_walk_matches_oracle(rb, prec, fine, reorth):
    """n = 65,536 rows: 512 tiles of 128 rows over 152 persistent CTAs, so every
    CTA walks three or four tiles and its copy/MMA rings wrap across tiles;
    m = 300 with m_p = 50 gives up to four 64-column basis chunks per tile
    (and block starts that do not fall on chunk boundaries).  Element-wise
    parity of Q and R with the oracle's Alg. 2 / Alg. 5 in FP64.  fine = 2
    takes the FP64 sketch space's products in double-FP32 arithmetic."""
    n, m, mb, kind, k = 65536, 300, 50, "srht", 600
    cond = 1e3
    oracle.set_threads(os.cpu_count() or 1)
    W = synth.svd_matrix(n, m, cond, 17).astype(np.float32).astype(np.float64)
    Wd = dev_ld(W, torch.float32, n)
    Qd = dev_ld(np.zeros((n, m)), torch.float32, n)
    _, Rd, st = rb.rbgs_qr(Wd, mb, kind, k, 5, prec=prec, ls_iters=1, reorth=reorth, Q=Qd, fine=fine)
    Q, R = host(Qd), host(Rd)
    ref = oracle.rbgs(W, mb, kind, k, 5, variant=5, ls="richardson", ls_iters=1, reorth=bool(reorth),
                      ls_iters_first=1)
    assert np.allclose(np.tril(R, -1), 0.0) and np.all(np.diag(R) > 0)
    assert oracle.factorization_error(W, Q, R) < 2e-6
    assert_factor_parity(Q, R, ref["Q"], ref["R"], U32, label=f"tile walk {prec} fine {fine} reorth {reorth}")
    assert st.passes2 == (m // mb - 1 if reorth else 0)


# ------------------------------------------------ full-size mixed workload --

C2_GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rbgs_c2_fp64.json")


@pytest.fixture(scope="module")
def c2_golden():
    import json

    with open(C2_GOLDEN) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def c2_matrix(rb, c2_golden):
    """The full-size workload on the device (FP32), built bit for bit as the
    oracle's input was: its bit checksum must equal the stored one."""
    g = c2_golden
    W = synth.hadamard_svd_matrix_torch(g["n"], g["m"], g["cond"], g["seed_w"], device="cuda", dtype=torch.float32)
    chk = int(W.contiguous().view(torch.int32).to(torch.int64).sum()) if W.is_contiguous() else \
        int(W.t().contiguous().view(torch.int32).to(torch.int64).sum())
    assert chk == g["w_bit_checksum"], "the device built a different W than the oracle factored"
    return W


def _compare_c2(Q, R, g, u, label):
    """Sampled outputs of a full-size factorization against the stored oracle
    values, with the per-column bound of assert_factor_parity (kappa_j stored
    for the sampled columns): R's diagonal, sixteen whole columns of R and
    four whole rows of Q."""
    m = g["m"]
    Rd = R.diagonal().double().cpu().numpy()
    worst = 0.0
    kap_all = {int(j): c["kappa"] for j, c in g["R_cols"].items()}
    for j, c in g["R_cols"].items():
        j = int(j)
        ref = np.array(c["R"])
        got = R[: j + 1, j].double().cpu().numpy()
        unit = u * np.sqrt(m) * c["kappa"]
        er = np.abs(got - ref).max() / np.linalg.norm(ref)
        assert er <= PARITY_C * unit, f"{label} R column {j}: {er:.3e} > {PARITY_C * unit:.3e}"
        worst = max(worst, er / unit)
        # the diagonal entry of a sampled column: same bound
        assert abs(Rd[j] - g["R_diag"][j]) <= PARITY_C * unit * np.linalg.norm(ref)
    # rows of Q: entry j carries column j's bound; kappa_j of the unsampled
    # columns is bounded by that of the next sampled column (kappa_j grows with j)
    cols = sorted(kap_all)
    kap = np.array([kap_all[min(c for c in cols if c >= j)] for j in range(m)])
    qscale = np.abs(np.array([g["Q_rows"][r] for r in g["Q_rows"]])).max(axis=0)
    for r, ref in g["Q_rows"].items():
        got = Q[int(r)].double().cpu().numpy()
        unit = u * np.sqrt(m) * kap
        err = np.abs(got - np.array(ref)) / qscale
        bad = np.nonzero(err > PARITY_C * unit)[0]
        assert bad.size == 0, f"{label} Q row {r} column {bad[0]}: {err[bad[0]]:.3e}"
        worst = max(worst, float((err / unit).max()))
    print(f"[parity] {label} max err/(u sqrt(m) kappa_j) over the samples: {worst:.3f}")


def _c2_quality(W, Q, R, g):
    n, m = g["n"], g["m"]
    num = den = 0.0
    R64 = R.double()
    for r0 in range(0, n, 100_000):
        Wc = W[r0:r0 + 100_000].double()
        E = Wc - Q[r0:r0 + 100_000].double() @ R64
        num += float((E * E).sum())
        den += float((Wc * Wc).sum())
    oracle.set_threads(os.cpu_count() or 1)
    S = oracle.theta_apply(g["sketch"], g["k"], g["seed_theta"], host(Q))
    E = np.eye(m) - S.T @ S
    return np.sqrt(num / den), np.linalg.norm(E), np.linalg.norm(E, 2)


def test_c2_full_size_fp64_matches_oracle(rb, c2_golden, c2_matrix):
    """The plain FP64 GPU path at the full size (n = 1e6, m = 1000, m_p = 50,
    SRHT k = 2000, second pass on every block, one Richardson iteration)
    against the oracle's FP64 run of the same options on the same matrix
    (stored by tests/golden/make_rbgs_c2_fp64.py): sampled columns of R and
    rows of Q within C u_64 sqrt(m) kappa_j, and the quality targets
    ||W - QR||/||W|| <= 1e-13 and sketched orthogonality <= 1e-12."""
    g = c2_golden
    W64 = c2_matrix.double()
    Q, R, st = rb.rbgs_qr(W64, g["mb"], g["sketch"], g["k"], g["seed_theta"], prec="fp64", ls_iters=1, reorth=1)
    assert st.passes2 == g["passes2"]
    Rh = R.cpu().numpy()
    assert np.allclose(np.tril(Rh, -1), 0.0) and np.all(np.diag(Rh) > 0)
    _compare_c2(Q, R, g, U64, "c2 fp64")
    fact, d_fro, d_two = _c2_quality(W64, Q, R, g)
    assert fact <= 1e-13 and d_fro <= 1e-12
    del W64, Q, R
    torch.cuda.empty_cache()


@pytest.mark.parametrize("fine", [1, 2])
def test_c2_full_size_mixed_matches_oracle(rb, c2_golden, c2_matrix, fine):
    """The mixed path at the full size in the launch configuration bench.py
    times (F16X3 tall products, FP64 sketch space, one Richardson iteration,
    second pass on every block) against the same stored oracle run: sampled
    columns of R and rows of Q within C u_32 sqrt(m) kappa_j (binding for the
    leading columns, where kappa_j is small), W = QR to 1e-6, and sketched
    orthogonality (the oracle's own Theta) <= 1e-6 in the 2-norm; the
    Frobenius norm, floored by the FP32 storage of Q, is held to 2e-5."""
    g = c2_golden
    W = c2_matrix
    Q, R, st = rb.rbgs_qr(W, g["mb"], g["sketch"], g["k"], g["seed_theta"], prec="f16x3", ls_iters=1, reorth=1,
                          fine=fine)
    assert st.passes2 == g["m"] // g["mb"] - 1
    Rh = R.cpu().numpy()
    assert np.allclose(np.tril(Rh, -1), 0.0) and np.all(np.diag(Rh) > 0)
    _compare_c2(Q, R, g, U32, f"c2 f16x3 fine {fine}")
    fact, d_fro, d_two = _c2_quality(W, Q, R, g)
    print(f"[quality] c2 f16x3 fine {fine}: ||W-QR||/||W|| {fact:.3e}, Delta_F {d_fro:.3e}, Delta_2 {d_two:.3e}")
    assert fact <= 1e-6
    assert d_two <= 1e-6
    assert d_fro <= 2e-5


# ------------------------------------------- the a posteriori Phi check --

@pytest.mark.parametrize("prec,kind", [("fp64", "gauss"), ("fp64", "srht"), ("f16x3", "srht"), ("fp32", "gauss")])
def test_embedding_check_matches_oracle(rb, prec, kind):
    """||I - (Theta Q_phi)^T Theta Q_phi||_F with Q_phi the RBGS factor of Z
    under an independent sketch Phi, against the oracle; Phi = Theta gives the
    sketched orthogonality of RBGS itself."""
    n, m, mb, k = 3000, 32, 8, 128
    td = torch.float64 if prec == "fp64" else torch.float32
    Z = synth.svd_matrix(n, m, 1e2, 74)
    if prec != "fp64":
        Z = Z.astype(np.float32).astype(np.float64)
    Zd = dev(Z, td)
    got = rb.embedding_check(Zd, mb, kind, k, 5, 9, prec=prec, ls_iters=3, fine=prec != "fp64")
    want = oracle.embedding_check(Z, mb, kind, k, 5, 9, ls="richardson", ls_iters=3)
    tol = 1e-9 * want if prec == "fp64" else 1e-4
    assert abs(got - want) <= tol and 0.05 < want < 10.0
    same = rb.embedding_check(Zd, mb, kind, k, 5, 5, prec=prec, ls_iters=3, fine=prec != "fp64")
    assert same < (1e-12 if prec == "fp64" else 1e-4)


# ------------------------------------------------ Cholesky QR post-processing --

@pytest.mark.parametrize("prec", ["fp64", "f16x3", "tf32x3", "fp32"])
@pytest.mark.parametrize("pmb", [64, 16, 48])
def test_cholqr_postprocess_matches_oracle(rb, prec, pmb):
    """The post-processing of an RBGS factorization on the GPU against the
    oracle's on the same Q, R: an l2-orthonormal Q, W = QR kept, and for FP64
    the thin Householder QR of W."""
    n, m, mb, k = 5000, 100, 20, 240
    cond = 1e4 if prec == "fp64" else 1e2
    td = torch.float64 if prec == "fp64" else torch.float32
    W = synth.svd_matrix(n, m, cond, 83)
    if prec != "fp64":
        W = W.astype(np.float32).astype(np.float64)
    Qd, Rd, _ = rb.rbgs_qr(dev(W, td), mb, "srht", k, 4, prec=prec, ls_iters=2, reorth=1, fine=prec != "fp64")
    Q0, R0 = host(Qd), host(Rd)
    rb.cholqr_postprocess(Qd, Rd, mb=pmb, prec=prec)
    Q, R = host(Qd), host(Rd)
    Qo, Ro = oracle.cholqr_postprocess(Q0, R0)
    assert np.allclose(np.tril(R, -1), 0.0) and np.all(np.diag(R) > 0)
    orth = np.abs(Q.T @ Q - np.eye(m)).max()
    fact = oracle.factorization_error(W, Q, R)
    if prec == "fp64":
        assert orth < 1e-13 and fact < 1e-14
        np.testing.assert_allclose(R, Ro, atol=1e-12 * np.abs(Ro).max())
        np.testing.assert_allclose(Q, Qo, atol=1e-10)
        Rn = np.linalg.qr(W)[1]
        np.testing.assert_allclose(R, np.sign(np.diag(Rn))[:, None] * Rn, atol=1e-10 * np.abs(Rn).max())
    else:
        assert orth < 2e-5 and fact < 5e-6
        np.testing.assert_allclose(R, Ro, atol=1e-5 * np.abs(Ro).max())


# ------------------------------------------------ step 2 by conjugate gradients --

@pytest.mark.parametrize("prec,fine", [("fp64", False), ("f16x3", True), ("fp32", False)])
@pytest.mark.parametrize("interblock", [5, 4, 6])
@pytest.mark.parametrize("reorth,m", [(0, 48), (1, 48), (1, 45)])
def test_rbgs_householder_step2_matches_oracle(rb, prec, fine, interblock, reorth, m):
    """Step 2 by Householder least squares (the textbook solver of Sec. 3.1):
    the blocked Householder QR of S in compact WY form, one panel per block,
    against the oracle's column-by-column Householder solver.  Both give the
    exact least-squares solution up to rounding; fp32 with fine=False runs the
    factorization in FP32."""
    n, mb, kind, k = 3000, 16, "gauss", 200
    cond = 1e4 if prec == "fp64" else 1e3
    W = synth.svd_matrix(n, m, cond, 80)
    if prec != "fp64":
        W = W.astype(np.float32).astype(np.float64)
    td = torch.float64 if prec == "fp64" else torch.float32
    Qd, Rd, st = rb.rbgs_qr(dev(W, td), mb, kind, k, 5, prec=prec, reorth=reorth, interblock=interblock,
                            ls="householder", fine=fine)
    Q, R = host(Qd), host(Rd)
    ref = oracle.rbgs(W, mb, kind, k, 5, variant=interblock, ls="householder", reorth=bool(reorth))
    assert np.allclose(np.tril(R, -1), 0.0) and np.all(np.diag(R) > 0)
    fact = oracle.factorization_error(W, Q, R)
    ortho = oracle.sketched_orthogonality(Q, kind, k, 5)[0]
    if prec == "fp64":
        tol = 1e-13 * cond
        assert np.abs(R - ref["R"]).max() <= tol * np.abs(ref["R"]).max()
        assert np.abs(Q - ref["Q"]).max() <= tol * np.abs(ref["Q"]).max()
        assert fact < 1e-14 and ortho < 10 * ref["delta"] + 1e-13
    else:
        assert fact < 2e-6 and ortho < (1e-4 if reorth else 1e-3)
        assert_factor_parity(Q, R, ref["Q"], ref["R"], U32,
                             label=f"householder step 2 {prec} interblock {interblock} reorth {reorth} m {m}")
    if reorth:
        assert st.passes2 == (m + mb - 1) // mb - 1


def test_rbgs_householder_step2_column_by_column(rb):
    """The column-by-column inter-block variant runs its inner factorization
    with the same solver."""
    n, m, mb, kind, k = 2000, 24, 8, "gauss", 96
    W = synth.svd_matrix(n, m, 1e3, 81)
    Qd, Rd, _ = rb.rbgs_qr(dev(W), mb, kind, k, 5, prec="fp64", reorth=1, interblock=3, ls="householder")
    ref = oracle.rbgs(W, mb, kind, k, 5, variant=3, ls="householder", reorth=True)
    R = host(Rd)
    assert np.abs(R - ref["R"]).max() <= 1e-10 * np.abs(ref["R"]).max()
    assert oracle.factorization_error(W, host(Qd), R) < 1e-14


@pytest.mark.parametrize("prec", ["fp64", "f16x3"])
@pytest.mark.parametrize("interblock", [5, 4])
@pytest.mark.parametrize("reorth", [0, 1])
def test_rbgs_cg_step2_matches_oracle(rb, prec, interblock, reorth):
    """Step 2 by l conjugate-gradient steps on the normal equations, column
    by column (20 steps, the paper's first experiment), against the oracle."""
    n, m, mb, kind, k = 3000, 48, 16, "gauss", 200
    cond = 1e4 if prec == "fp64" else 1e3
    W = synth.svd_matrix(n, m, cond, 79)
    if prec != "fp64":
        W = W.astype(np.float32).astype(np.float64)
    td = torch.float64 if prec == "fp64" else torch.float32
    Qd, Rd, st = rb.rbgs_qr(dev(W, td), mb, kind, k, 5, prec=prec, ls_iters=20, reorth=reorth, interblock=interblock,
                            ls="cg", fine=prec != "fp64")
    Q, R = host(Qd), host(Rd)
    ref = oracle.rbgs(W, mb, kind, k, 5, variant=interblock, ls="cg", ls_iters=20, reorth=bool(reorth),
                      ls_iters_first=1)
    assert np.allclose(np.tril(R, -1), 0.0) and np.all(np.diag(R) > 0)
    fact = oracle.factorization_error(W, Q, R)
    ortho = oracle.sketched_orthogonality(Q, kind, k, 5)[0]
    if prec == "fp64":
        tol = 1e-12 * cond
        assert np.abs(R - ref["R"]).max() <= tol * np.abs(ref["R"]).max()
        assert np.abs(Q - ref["Q"]).max() <= tol * np.abs(ref["Q"]).max()
        assert fact < 1e-14 and ortho < 10 * ref["delta"] + 1e-13  # single pass: about u cond(W), like the oracle
    else:
        assert fact < 2e-6 and ortho < (1e-4 if reorth else 1e-3)
        assert_factor_parity(Q, R, ref["Q"], ref["R"], U32, label=f"cg step 2 {prec} interblock {interblock} reorth {reorth}")
