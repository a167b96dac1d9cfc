"""GPU parity of the randomized block Krylov methods (Sec. 5) against the CPU
oracle: the 5-point convection-diffusion operator, RBGS-Arnoldi (Alg. 7),
restarted randomized block GMRES / FOM (Sec. 5.2, 5.3), and the restarted
randomized Rayleigh-Ritz method (Alg. 8, Sec. 5.4)."""
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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nx,ny,bx,by", [(37, 29, 100.0, 50.0), (1, 5, 0.0, 3.0), (64, 64, 7.0, -2.0)])
def test_op_apply_matches_oracle(rb, prec, nx, ny, bx, by):
    X = synth.gaussian(nx * ny, 3, nx + ny)
    td = torch.float64 if prec == "fp64" else torch.float32
    if prec == "fp32":
        X = X.astype(np.float32).astype(np.float64)
    Y = host(rb.op_apply(rb.stencil_op(nx, ny, bx, by), dev(X, td), prec=prec))
    ref = oracle.stencil5_apply(nx, ny, bx, by, X)
    tol = 1e-14 if prec == "fp64" else 2e-6
    assert np.abs(Y - ref).max() <= tol * np.abs(ref).max()


def _arnoldi_checks(Q, R, A, mp, p, kind, k, seed, tol):
    AQ = A @ Q[:, : (p - 1) * mp]
    assert np.abs(AQ - Q @ R[:, mp:]).max() <= tol * np.abs(AQ).max()
    S = oracle.theta_apply(kind, k, seed, Q)
    return np.abs(S.T @ S - np.eye(p * mp)).max()


@pytest.mark.parametrize("kind,k", [("gauss", 60), ("srht", 64)])
@pytest.mark.parametrize("reorth", [0, 1])
def test_arnoldi_fp64_matches_oracle(rb, kind, k, reorth):
    nx, ny, mp, p = 24, 20, 4, 6
    n = nx * ny
    B = synth.gaussian(n, mp, 17)
    Qd, Rd = rb.block_arnoldi(rb.stencil_op(nx, ny, 30.0, 10.0), dev(B), p, kind, k, 3, prec="fp64", ls_iters=3,
                              reorth=reorth)
    Q, R = host(Qd), host(Rd)
    ref = oracle.rbgs_arnoldi(nx, ny, 30.0, 10.0, B, p, kind, k, 3, variant=5, ls="richardson", ls_iters=3,
                              reorth=bool(reorth), ls_iters_first=1)
    A = oracle.stencil5_dense(nx, ny, 30.0, 10.0)
    ortho = _arnoldi_checks(Q, R, A, mp, p, kind, k, 3, 1e-12)
    assert ortho < 1e-10
    assert np.abs(R - ref["R"]).max() <= 1e-9 * np.abs(ref["R"]).max()
    assert np.abs(Q - ref["Q"]).max() <= 1e-9 * np.abs(ref["Q"]).max()


@pytest.mark.parametrize("prec", ["f16x3", "tf32x3", "fp32"])
def test_arnoldi_mixed_identity(rb, prec):
    nx, ny, mp, p, k = 40, 32, 8, 6, 96
    n = nx * ny
    B = synth.gaussian(n, mp, 18).astype(np.float32).astype(np.float64)
    Qd, Rd = rb.block_arnoldi(rb.stencil_op(nx, ny, 100.0, 50.0), dev(B, torch.float32), p, "srht", k, 5, prec=prec,
                              ls_iters=1, reorth=1, fine=True)
    Q, R = host(Qd), host(Rd)
    A = oracle.stencil5_dense(nx, ny, 100.0, 50.0)
    ortho = _arnoldi_checks(Q, R, A, mp, p, "srht", k, 5, 1e-5)
    assert ortho < 1e-5


@pytest.mark.parametrize("method", ["gmres", "fom"])
def test_block_solver_fp64_matches_oracle_and_direct(rb, method):
    nx, ny, mp, p, k = 16, 12, 2, 8, 64
    n = nx * ny
    B = synth.gaussian(n, mp, 31)
    op = rb.stencil_op(nx, ny, 12.0, 6.0)
    solve = rb.block_gmres if method == "gmres" else rb.block_fom
    Xd, cyc, rel = solve(op, dev(B), p=p, rtol=1e-11, max_cycles=300, sketch="gauss", k=k, seed=8, prec="fp64",
                         ls_iters=3)
    X = host(Xd)
    assert max(rel) <= 1e-11
    Xs = np.linalg.solve(oracle.stencil5_dense(nx, ny, 12.0, 6.0), B)
    assert np.abs(X - Xs).max() <= 1e-8 * np.abs(Xs).max()
    Xo, cyc_o, rel_o = oracle.block_krylov(method, nx, ny, 12.0, 6.0, B, np.zeros((n, mp)), p, "gauss", k, 8, 1e-11,
                                           300, ls="richardson", ls_iters=3)
    assert abs(cyc - cyc_o) <= max(1, cyc_o // 5)


@pytest.mark.parametrize("prec", ["f16x3", "fp32"])
def test_gmres_mixed_precision_refinement(rb, prec):
    """FP32 Krylov basis (tensor-core or SIMT products), FP64 residuals and
    solution: the restarts act as iterative refinement down to 1e-9."""
    nx, ny, mp, p, k = 32, 32, 4, 10, 160
    n = nx * ny
    B = synth.gaussian(n, mp, 41)
    op = rb.stencil_op(nx, ny, 100.0, 50.0)
    Xd, cyc, rel = rb.block_gmres(op, dev(B), p=p, rtol=1e-9, max_cycles=400, sketch="srht", k=k, seed=2, prec=prec,
                                  ls_iters=1, reorth=1, fine=True)
    assert max(rel) <= 1e-9
    Xs = np.linalg.solve(oracle.stencil5_dense(nx, ny, 100.0, 50.0), B)
    assert np.abs(host(Xd) - Xs).max() <= 1e-6 * np.abs(Xs).max()


def test_krylov_invalid_arguments(rb):
    op = rb.stencil_op(8, 8, 1.0, 1.0)
    B = dev(synth.gaussian(64, 2, 1))
    with pytest.raises(rb.RbgsError):
        rb.block_gmres(op, B, p=1, sketch="gauss", k=16)          # p < 2
    with pytest.raises(rb.RbgsError):
        rb.block_gmres(op, B, p=8, sketch="gauss", k=8)           # k < m
    with pytest.raises(rb.RbgsError):
        rb.block_arnoldi(rb.stencil_op(0, 8, 1.0, 1.0), B, 4, "gauss", 16)  # empty grid


# ------------------------------------------------ Alg. 8: Rayleigh-Ritz --

def _closed_form_eigs(nx, ny, bx, by):
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    px, py = bx * hx / 2, by * hy / 2
    ex = (2.0 - 2.0 * np.sqrt(1 - px ** 2) * np.cos(np.arange(1, nx + 1) * np.pi * hx)) / hx ** 2
    ey = (2.0 - 2.0 * np.sqrt(1 - py ** 2) * np.cos(np.arange(1, ny + 1) * np.pi * hy)) / hy ** 2
    return np.sort((ex[:, None] + ey[None, :]).ravel())


@pytest.mark.parametrize("which", ["LR", "SR"])
@pytest.mark.parametrize("kind,k,n_iter", [("gauss", 80, 1), ("srht", 96, 4), ("gauss", 80, 7)])
def test_rayleigh_ritz_fp64_matches_oracle(rb, which, kind, k, n_iter):
    """FP64 basis: Ritz values, residual estimates and the returned vectors
    agree with the oracle's Alg. 8 (numpy's eig for the small problem)."""
    nx, ny, bx, by, mp, p = 12, 10, 12.0, 6.0, 3, 6
    n = nx * ny
    B = synth.gaussian(n, mp, 51)
    vals, Xd, res = rb.rayleigh_ritz(rb.stencil_op(nx, ny, bx, by), dev(B), p=p, n_iter=n_iter, which=which,
                                     sketch=kind, k=k, seed=9, prec="fp64", ls_iters=3)
    ref = oracle.rayleigh_ritz(nx, ny, bx, by, B, p, n_iter, which, kind, k, 9, ls="richardson", ls_iters=3,
                               ls_iters_first=1)
    scale = _closed_form_eigs(nx, ny, bx, by)[-1]
    np.testing.assert_allclose(np.array(vals), ref["values"], rtol=0, atol=1e-8 * scale)
    np.testing.assert_allclose(np.array(res), ref["resid"], rtol=0, atol=1e-8 * scale)
    X = host(Xd)
    np.testing.assert_allclose(np.linalg.norm(X, axis=0), 1.0, atol=1e-13)
    assert np.abs(X - ref["X"]).max() <= 1e-7


def test_rayleigh_ritz_complex_pairs_match_oracle(rb):
    """Cell Peclet numbers above 1 give a complex spectrum: conjugate Ritz
    pairs take the columns Re y, Im y with the same scaling on both sides."""
    nx, ny, bx, by, mp, p, k = 10, 9, 90.0, 60.0, 4, 7, 90
    n = nx * ny
    B = synth.gaussian(n, mp, 53)
    vals, Xd, res = rb.rayleigh_ritz(rb.stencil_op(nx, ny, bx, by), dev(B), p=p, n_iter=2, which="LR",
                                     sketch="gauss", k=k, seed=4, prec="fp64", ls_iters=3)
    ref = oracle.rayleigh_ritz(nx, ny, bx, by, B, p, 2, "LR", "gauss", k, 4, ls="richardson", ls_iters=3,
                               ls_iters_first=1)
    assert any(abs(v.imag) > 0 for v in ref["values"])
    scale = abs(np.linalg.eigvals(oracle.stencil5_dense(nx, ny, bx, by))).max()
    np.testing.assert_allclose(np.array(vals), ref["values"], rtol=0, atol=1e-8 * scale)
    np.testing.assert_allclose(np.array(res), ref["resid"], rtol=0, atol=1e-8 * scale)
    assert np.abs(host(Xd) - ref["X"]).max() <= 1e-7


@pytest.mark.parametrize("which", ["LR", "SR"])
def test_rayleigh_ritz_converges_to_closed_form(rb, which):
    """Restarts drive the leading Ritz value to the extreme eigenvalue of the
    closed form and its residual estimate to zero; its vector is an
    eigenvector of the operator (checked through the GPU operator)."""
    nx, ny, bx, by, mp, p, k = 10, 8, 12.0, 6.0, 3, 6, 60
    n = nx * ny
    ev = _closed_form_eigs(nx, ny, bx, by)
    op = rb.stencil_op(nx, ny, bx, by)
    vals, Xd, res = rb.rayleigh_ritz(op, dev(synth.gaussian(n, mp, 31)), p=p, n_iter=60, which=which,
                                     sketch="gauss", k=k, seed=4, prec="fp64", ls_iters=3)
    target = ev[-1] if which == "LR" else ev[0]
    assert vals[0].imag == 0.0 and abs(vals[0].real - target) <= 1e-10 * ev[-1]
    assert res[0] <= 1e-8 * ev[-1]
    x = Xd[:, :1].contiguous()
    r = host(rb.op_apply(op, x, prec="fp64"))[:, 0] - vals[0].real * host(x)[:, 0]
    assert np.linalg.norm(r) <= 1e-7 * ev[-1]


@pytest.mark.parametrize("prec", ["f16x3", "fp32"])
def test_rayleigh_ritz_mixed_basis(rb, prec):
    """FP32 basis (F16X3 tensor-core or SIMT products), FP64 sketch space and
    small problem: Ritz values within the FP32 level of the oracle's."""
    nx, ny, bx, by, mp, p, k = 32, 24, 40.0, 20.0, 4, 8, 128
    n = nx * ny
    B = synth.gaussian(n, mp, 57)
    vals, Xd, res = rb.rayleigh_ritz(rb.stencil_op(nx, ny, bx, by), dev(B), p=p, n_iter=2, which="LR",
                                     sketch="srht", k=k, seed=6, prec=prec, ls_iters=1, reorth=1, fine=True)
    ref = oracle.rayleigh_ritz(nx, ny, bx, by, B.astype(np.float32).astype(np.float64), p, 2, "LR", "srht", k, 6,
                               ls="richardson", ls_iters=1, reorth=True, ls_iters_first=1)
    scale = _closed_form_eigs(nx, ny, bx, by)[-1]
    np.testing.assert_allclose(np.array(vals), ref["values"], rtol=0, atol=1e-4 * scale)
    np.testing.assert_allclose(np.array(res), ref["resid"], rtol=0, atol=1e-4 * scale)


def test_rayleigh_ritz_full_size_properties(rb):
    """The 1024^2 convection-diffusion operator, 8 vectors, 40 blocks, SRHT
    k = 1280, F16X3 basis: a real Ritz value's sketched residual estimate
    matches the l2 residual of its returned unit vector (cond(Q) = 1 + O(eps)).
    The sketched Galerkin projection is not an l2 Rayleigh quotient, so the
    Ritz values may leave the spectrum's range by O(eps) ||A||; they are only
    checked to lie near it."""
    nx = ny = 1024
    mp, p, k = 8, 40, 1280
    n = nx * ny
    op = rb.stencil_op(nx, ny, 100.0, 50.0)
    B = torch.randn((mp, n), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(3)).t()
    vals, Xd, res = rb.rayleigh_ritz(op, B, p=p, n_iter=2, which="LR", sketch="srht", k=k, seed=1, prec="f16x3",
                                     ls_iters=1, reorth=1, fine=True)
    ev = _closed_form_eigs(nx, ny, 100.0, 50.0)
    X = Xd
    AX = rb.op_apply(op, X, prec="fp64")
    for j, v in enumerate(vals):
        assert 0.5 * ev[0] <= v.real <= ev[-1] * (1 + 1e-2)
        if v.imag == 0.0:
            r = float(torch.linalg.norm(AX[:, j] - v.real * X[:, j]))
            assert 0.5 * res[j] <= r <= 2.0 * res[j] + 1e-6 * ev[-1]
