"""GPU parity for the sparse-sign sketch (the block construction of the sparse
JL transform: z = min(8, k) row segments, one nonzero +-1/sqrt(z) per segment
and column): the CUDA sketch and the factorization built on it against the CPU
oracle on the same seeded inputs."""
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
    A = np.asarray(A)
    return torch.from_numpy(np.ascontiguousarray(A.T)).to("cuda", dtype).t()


def host(T):
    return T.detach().double().cpu().numpy()


# (n, columns, k): one entry; ragged row and column tiles; more than 64 columns
# (two launches); k <= 8 (a dense sign matrix); several 64-row tiles of Theta
CASES = [(1, 1, 1), (100, 3, 40), (3001, 9, 200), (777, 70, 129), (5000, 5, 7), (20000, 16, 1000)]


@pytest.mark.parametrize("n,c,k", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sparse_sketch_matches_oracle(rb, n, c, k, prec):
    seed = 4321 + n
    X = synth.gaussian(n, c, seed=n + 2 * c)
    if prec == "fp32":
        X = X.astype(np.float32).astype(np.float64)
    Y = host(rb.sketch_apply(dev(X, torch.float64 if prec == "fp64" else torch.float32), "sparse", k, seed,
                             prec=prec))
    Yr = oracle.theta_apply("sparse", k, seed, X)
    scale = np.linalg.norm(X, axis=0)[None, :] + 1e-300
    err = np.abs(Y - Yr) / scale
    assert err.max() <= (1e-14 if prec == "fp64" else 3e-6), f"max rel err {err.max():.3e}"


@pytest.mark.parametrize("n,m,mb,k", [(3000, 32, 8, 160), (4001, 45, 16, 200)])
@pytest.mark.parametrize("reorth", [0, 1])
def test_rbgs_fp64_with_sparse_sketch_matches_oracle(rb, n, m, mb, k, reorth):
    cond = 1e4
    W = synth.svd_matrix(n, m, cond, n + m)
    Qd, Rd, st = rb.rbgs_qr(dev(W), mb, "sparse", k, 17, prec="fp64", ls_iters=3, reorth=reorth)
    Q, R = host(Qd), host(Rd)
    ref = oracle.rbgs(W, mb, "sparse", k, 17, variant=5, ls="richardson", ls_iters=3, reorth=bool(reorth),
                      ls_iters_first=1)
    assert np.allclose(np.tril(R, -1), 0.0) and np.all(np.diag(R) > 0)
    tol = 1e-13 * cond
    assert np.abs(R - ref["R"]).max() <= tol * np.abs(ref["R"]).max()
    assert np.abs(Q - ref["Q"]).max() <= tol * np.abs(ref["Q"]).max()
    assert oracle.factorization_error(W, Q, R) < 1e-14
    assert oracle.sketched_orthogonality(Q, "sparse", k, 17)[0] < (1e-12 if reorth else 10 * ref["delta"] + 1e-13)


def test_rbgs_mixed_with_sparse_sketch(rb):
    """FP32 storage, F16X3 tall products, FP64 sketch space, second pass."""
    n, m, mb, k = 50000, 96, 32, 384
    W = synth.svd_matrix(n, m, 1e3, 5).astype(np.float32).astype(np.float64)
    Qd, Rd, st = rb.rbgs_qr(dev(W, torch.float32), mb, "sparse", k, 2, prec="f16x3", ls_iters=1, reorth=1, fine=True)
    Q, R = host(Qd), host(Rd)
    assert st.passes2 == m // mb - 1
    assert np.allclose(np.tril(R, -1), 0.0) and np.all(np.diag(R) > 0)
    assert oracle.factorization_error(W, Q, R) < 2e-6
    S = oracle.theta_apply("sparse", k, 2, Q)
    assert np.linalg.norm(np.eye(m) - S.T @ S, 2) < 1e-5
