"""Pins of the oracle for the learned preconditioner and randomized block
flexible GMRES (oracle/learned.py), each against something the mathematics
or an independent implementation fixes."""
import numpy as np
import pytest

import oracle
import synth
from oracle import learned as L

# --------------------------------------------------------------- the inputs --


def test_random_field_has_the_stated_covariance():
    """Zero mean, variance 1, squared-exponential correlation exp(-r^2 / (2 l^2))
    with l = 0.05 (averaged over 40 fields; loose statistical bounds)."""
    N = 63
    h = 1.0 / (N + 1)
    gs = np.array([synth.gaussian_random_field(N, s) for s in range(40)])
    assert gs.shape == (40, N + 2, N + 2)
    assert abs(gs.mean()) < 0.1 and abs(gs.var() - 1.0) < 0.1
    for lag in (1, 3):
        c = np.mean(gs[:, :, :-lag] * gs[:, :, lag:]) / gs.var()
        assert abs(c - np.exp(-(lag * h) ** 2 / (2 * 0.05 ** 2))) < 0.05


# ------------------------------------------------------------ the operator --


def test_unit_coefficient_is_the_five_point_laplacian():
    """a = 1 gives -Laplace, the C oracle's stencil with zero convection;
    a = alpha scales it by alpha (harmonic means of equal values)."""
    N = 11
    X = np.random.default_rng(0).standard_normal((N * N, 3))
    ref = oracle.stencil5_apply(N, N, 0.0, 0.0, X)
    np.testing.assert_allclose(L.diffusion_apply(np.ones((N + 2, N + 2)), X), ref, rtol=1e-13, atol=1e-9)
    np.testing.assert_allclose(L.diffusion_apply(np.full((N + 2, N + 2), 2.5), X), 2.5 * ref, rtol=1e-13, atol=1e-9)


def test_operator_is_symmetric_positive_definite_and_matches_its_matrix():
    N = 9
    a = np.exp(synth.gaussian_random_field(N, 3))
    A = L.diffusion_matrix(a).toarray()
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-9 * np.abs(A).max())
    assert np.linalg.eigvalsh(A).min() > 0
    X = np.random.default_rng(1).standard_normal((N * N, 4))
    np.testing.assert_allclose(L.diffusion_apply(a, X), A @ X, rtol=1e-12, atol=1e-9 * np.abs(A).max())


def test_operator_is_second_order_on_a_manufactured_solution():
    """u = sin(pi x) sin(pi y), a = 1 + x y: -div(a grad u) = 2 pi^2 a u -
    pi (y cos(pi x) sin(pi y) + x sin(pi x) cos(pi y)).  The scheme's
    error at the nodes falls by about 4 when h halves."""
    errs = []
    for N in (15, 31, 63):
        h = 1.0 / (N + 1)
        x = np.arange(N + 2) * h
        Xn, Yn = np.meshgrid(x, x, indexing="ij")
        a = 1.0 + Xn * Yn
        u = np.sin(np.pi * Xn) * np.sin(np.pi * Yn)
        f = (2 * np.pi ** 2 * a * u
             - np.pi * (Yn * np.cos(np.pi * Xn) * np.sin(np.pi * Yn) + Xn * np.sin(np.pi * Xn) * np.cos(np.pi * Yn)))
        Au = L.diffusion_apply(a, u[1:-1, 1:-1].reshape(-1, order="F"))
        errs.append(np.abs(Au - f[1:-1, 1:-1].reshape(-1, order="F")).max())
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


# ---------------------------------------------------------- flexible GMRES --


def test_fgmres_with_identity_is_the_c_oracles_block_gmres():
    """M = I turns the flexible method into randomized block GMRES (Sec. 5.2):
    two cycles agree with the independent C implementation."""
    nx, ny, bx, by, mp, p, k = 12, 10, 3.0, 1.5, 3, 6, 72
    n = nx * ny
    B = synth.gaussian(n, mp, 5)
    X0 = np.zeros((n, mp))
    Xc, cyc_c, _ = oracle.block_krylov("gmres", nx, ny, bx, by, B, X0, p, "gauss", k, 9, 0.0, 2, variant=5,
                                       ls="householder")
    Xf, cyc_f, hist = L.block_fgmres(lambda X: oracle.stencil5_apply(nx, ny, bx, by, X), None, B, X0, p, "gauss", k,
                                     9, 0.0, 2)
    assert cyc_c == cyc_f == 2
    np.testing.assert_allclose(Xf, Xc, rtol=0, atol=1e-10 * np.abs(Xc).max())
    assert hist[2] < hist[1] < hist[0]


def test_fgmres_with_the_exact_inverse_converges_in_one_step():
    """M = A^{-1}: A Z_1 = Q_1, so r - A Z_1 z = 0 for z = R_11 after one
    Arnoldi expansion."""
    N, mp = 10, 2
    a = np.exp(synth.gaussian_random_field(N, 4))
    A = L.diffusion_matrix(a).toarray()
    B = synth.gaussian(N * N, mp, 6)
    X, cyc, hist = L.block_fgmres(lambda X: A @ X, lambda Q: np.linalg.solve(A, Q), B, np.zeros_like(B), 2,
                                  "gauss", 40, 3, 1e-12, 3)
    assert cyc == 1 and hist[-1] < 1e-12


def test_fgmres_minimises_the_sketched_residual():
    """One cycle's z equals the brute-force minimiser of ||Theta (r - A Z z)||
    over the explicit matrices (Z from a fixed nonlinear preconditioner)."""
    N, mp, p, k = 8, 2, 4, 48
    n = N * N
    a = np.exp(synth.gaussian_random_field(N, 5))
    params = synth.unet_params(2, 7)
    B = synth.gaussian(n, mp, 8)
    A = lambda X: L.diffusion_apply(a, X)  # noqa: E731
    Zs = []

    def M(Q):
        Z = L.precondition(params, Q)
        Zs.append(Z)
        return Z

    X, cyc, _ = L.block_fgmres(A, M, B, np.zeros_like(B), p, "rademacher", k, 2, 0.0, 1)
    Z = np.hstack(Zs)
    TR = oracle.theta_apply("rademacher", k, 2, B)
    TAZ = oracle.theta_apply("rademacher", k, 2, A(Z))
    zref = np.linalg.lstsq(TAZ, TR, rcond=None)[0]
    np.testing.assert_allclose(X, Z @ zref, rtol=0, atol=1e-9 * np.abs(X).max())


# ---------------------------------------------------------------- the U-Net --


def test_conv_is_the_cross_correlation_of_scipy():
    from scipy.signal import correlate2d

    rng = np.random.default_rng(2)
    x = rng.standard_normal((3, 7, 6))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = L.conv3x3(x, w, b)
    for o in range(4):
        ref = b[o] + sum(correlate2d(x[c], w[o, c], mode="same", boundary="fill") for c in range(3))
        np.testing.assert_allclose(y[o], ref, rtol=1e-13, atol=1e-13)


def test_pool_and_upsample_backward_are_the_adjoints():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 6, 8))
    g = rng.standard_normal((2, 3, 4))
    assert abs(np.sum(L.avgpool2(x) * g) - np.sum(x * L.avgpool2_backward(g))) < 1e-12
    assert abs(np.sum(L.upsample2(g) * x) - np.sum(g * L.upsample2_backward(x))) < 1e-12


def test_unet_gradients_match_finite_differences():
    """Central differences of sum(gy * y) against the backward pass, for
    sampled entries of every parameter and of the input."""
    rng = np.random.default_rng(4)
    params = synth.unet_params(3, 11)
    for name in params:
        if name.endswith(".b"):
            params[name] = 0.1 * rng.standard_normal(params[name].shape)
    x = rng.standard_normal((1, 8, 8))
    y, cache = L.unet_forward(params, x)
    gy = rng.standard_normal(y.shape)
    grads, gx = L.unet_backward(params, cache, gy)

    def f(P, xx):
        return float(np.sum(gy * L.unet_forward(P, xx)[0]))

    eps = 1e-6
    for name in params:
        flat = params[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(5, flat.size), replace=False):
            Pp = {k2: v.copy() for k2, v in params.items()}
            Pm = {k2: v.copy() for k2, v in params.items()}
            Pp[name].reshape(-1)[idx] += eps
            Pm[name].reshape(-1)[idx] -= eps
            fd = (f(Pp, x) - f(Pm, x)) / (2 * eps)
            an = grads[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, idx, fd, an)
    for idx in rng.choice(x.size, size=8, replace=False):
        xp, xm = x.copy(), x.copy()
        xp.reshape(-1)[idx] += eps
        xm.reshape(-1)[idx] -= eps
        fd = (f(params, xp) - f(params, xm)) / (2 * eps)
        assert abs(fd - gx.reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_preconditioner_is_positively_homogeneous():
    params = synth.unet_params(2, 12)
    R = synth.gaussian(64, 2, 13)
    np.testing.assert_allclose(L.precondition(params, 3.5 * R), 3.5 * L.precondition(params, R), rtol=1e-12,
                               atol=1e-14)
    assert np.all(L.precondition(params, np.zeros((64, 1))) == 0.0)


def test_adam_first_step_moves_by_the_learning_rate():
    """With m_0 = v_0 = 0 the bias-corrected first step is
    -lr g / (|g| + eps): every nonzero-gradient entry moves by lr."""
    rng = np.random.default_rng(5)
    P = {"w": rng.standard_normal(10)}
    g = {"w": rng.standard_normal(10) * 10.0 ** rng.integers(-3, 3, size=10)}
    st = {}
    w0 = P["w"].copy()
    L.adam_step(P, g, st, lr=1e-2, eps=0.0)
    np.testing.assert_allclose(P["w"] - w0, -1e-2 * np.sign(g["w"]), rtol=1e-12, atol=0)


@pytest.mark.parametrize("loss", ["residual", "correction"])
def test_pair_loss_gradients_match_finite_differences(loss):
    """Both pair losses; the residual-norm one differentiates through the operator."""
    N = 8
    a = np.exp(synth.gaussian_random_field(N, 31))
    params = synth.unet_params(2, 32)
    r = synth.gaussian(N * N, 1, 33)[:, 0]
    e = L.correction_targets(a, r)[:, 0]
    val, g = L.pair_loss_and_grad(params, a, r, e, loss=loss)
    rng = np.random.default_rng(6)
    eps = 1e-6
    for name in ("e1.w", "m2.w", "o1.b", "o2.w"):
        for idx in rng.choice(params[name].size, size=min(3, params[name].size), replace=False):
            Pp = {k2: v.copy() for k2, v in params.items()}
            Pm = {k2: v.copy() for k2, v in params.items()}
            Pp[name].reshape(-1)[idx] += eps
            Pm[name].reshape(-1)[idx] -= eps
            fd = (L.pair_loss_and_grad(Pp, a, r, e, loss=loss)[0] - L.pair_loss_and_grad(Pm, a, r, e, loss=loss)[0]) \
                / (2 * eps)
            an = g[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * val), (name, idx, fd, an)


# ----------------------------------------------------- training, end to end --


@pytest.mark.timeout(600)
def test_trained_network_beats_plain_block_gmres_on_an_unseen_field():
    """Training inputs are the Arnoldi blocks of plain block GMRES (three
    cycles on each of six random fields), the loss the residual-norm pair
    loss.  Adam lowers it; on an unseen field flexible GMRES with the network
    (plain GMRES as the fallback, accept 0.9) reaches 1e-8 in fewer cycles
    than plain block GMRES, which is still above 1e-8 by then."""
    N, mp, p, k = 16, 2, 6, 48
    n = N * N
    data = []
    for s in range(6):
        a = np.exp(synth.gaussian_random_field(N, 100 + s))
        B = synth.gaussian(n, mp, 200 + s)
        _, _, _, rec = L.block_fgmres(lambda X, a=a: L.diffusion_apply(a, X), None, B, np.zeros_like(B), p, "gauss",
                                      k, 1, 0.0, 3, record=True)
        data += [(a, Q[:, j]) for Q in rec["bases"] for j in range(Q.shape[1])]
    params = synth.unet_params(8, 21)
    state = {}

    def mean_loss(P):
        return np.mean([L.pair_loss_and_grad(P, a, r)[0] for a, r in data[::5]])

    loss0 = mean_loss(params)
    rng = np.random.default_rng(0)
    for _ in range(2000):
        a, r = data[rng.integers(len(data))]
        _, g = L.pair_loss_and_grad(params, a, r)
        L.adam_step(params, g, state, lr=1e-3)
    assert mean_loss(params) < 0.25 * loss0
    a = np.exp(synth.gaussian_random_field(N, 998))
    B = synth.gaussian(n, mp, 1005)
    A = lambda X: L.diffusion_apply(a, X)  # noqa: E731
    _, cyc_net, hist_net, rec = L.block_fgmres(A, lambda Q: L.precondition(params, Q), B, np.zeros_like(B), p,
                                               "gauss", k, 1, 1e-8, 80, record=True, accept=0.9)
    _, cyc_plain, hist_plain = L.block_fgmres(A, None, B, np.zeros_like(B), p, "gauss", k, 1, 1e-8, 80)
    assert hist_net[-1] <= 1e-8
    assert cyc_net < cyc_plain and hist_plain[cyc_net] > 1e-8
    assert rec["fallbacks"] < cyc_net
