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


# ----------------------------------------------------- the L-level U-Net --


def test_two_level_network_is_the_l_level_network_with_two_levels():
    """unet_forward_levels with widths (c, 2c) is the two-level network of the
    pins above, layer for layer (enc0a = e1, enc0b = e2, enc1a = m1,
    enc1b = m2, dec0 = o1, out = o2), forward and backward."""
    c, N = 3, 8
    p2 = synth.unet_params(c, 5)
    names = {"e1": "enc0a", "e2": "enc0b", "m1": "enc1a", "m2": "enc1b", "o1": "dec0", "o2": "out"}
    pl = {names[k.split(".")[0]] + "." + k.split(".")[1]: v for k, v in p2.items()}
    x = np.random.default_rng(1).standard_normal((1, N, N))
    y2, c2 = L.unet_forward(p2, x)
    yl, cl = L.unet_forward_levels(pl, x, (c, 2 * c))
    np.testing.assert_allclose(yl, y2, rtol=1e-13, atol=1e-13)
    gy = np.random.default_rng(2).standard_normal(y2.shape)
    g2, gx2 = L.unet_backward(p2, c2, gy)
    gl, gxl = L.unet_backward_levels(pl, cl, gy, (c, 2 * c))
    np.testing.assert_allclose(gxl, gx2, rtol=1e-12, atol=1e-12)
    for k, v in g2.items():
        np.testing.assert_allclose(gl[names[k.split(".")[0]] + "." + k.split(".")[1]], v, rtol=1e-12, atol=1e-12)


def test_layer_list_of_the_four_level_network():
    """Widths (16, 32, 64, 64): twelve convolutions, concatenations of the
    upsampled level and the skip, a linear single-channel output."""
    lay = L.unet_layers((16, 32, 64, 64))
    assert [x[0] for x in lay] == ["enc0a", "enc0b", "enc1a", "enc1b", "enc2a", "enc2b", "enc3a", "enc3b", "dec2",
                                   "dec1", "dec0", "out"]
    assert [(x[1], x[2]) for x in lay] == [(1, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (64, 64),
                                           (64, 64), (128, 64), (96, 32), (48, 16), (16, 1)]
    assert [x[3] for x in lay] == [True] * 11 + [False]
    P = synth.unet_params_levels((16, 32, 64, 64), 3)
    assert set(P) == {f"{n}.{t}" for n, _, _, _ in lay for t in "wb"}
    for n, ci, co, _ in lay:
        assert P[n + ".w"].shape == (co, ci, 3, 3) and P[n + ".b"].shape == (co,)


def test_l_level_gradients_match_finite_differences():
    """Four levels on a 16 x 16 image (levels 16, 8, 4, 2): the backward pass
    equals central differences of sum(gy * y) for sampled weights, biases and
    inputs."""
    widths = (4, 6, 8, 8)
    N = 16
    P = synth.unet_params_levels(widths, 9)
    rng = np.random.default_rng(4)
    for k in P:
        if k.endswith(".b"):
            P[k] = 0.1 * rng.standard_normal(P[k].shape)
    x = rng.standard_normal((1, N, N))
    y, cache = L.unet_forward_levels(P, x, widths)
    gy = rng.standard_normal(y.shape)
    g, gx = L.unet_backward_levels(P, cache, gy, widths)

    def f(PP, xx):
        return float(np.sum(gy * L.unet_forward_levels(PP, xx, widths)[0]))

    eps = 1e-5
    for name in ("enc0a.w", "enc2b.w", "enc3a.b", "dec1.w", "dec0.b", "out.w"):
        for _ in range(2):
            idx = tuple(rng.integers(0, s) for s in P[name].shape)
            Pp = {k: v.copy() for k, v in P.items()}
            Pm = {k: v.copy() for k, v in P.items()}
            Pp[name][idx] += eps
            Pm[name][idx] -= eps
            fd = (f(Pp, x) - f(Pm, x)) / (2 * eps)
            assert abs(fd - g[name][idx]) <= 1e-5 * (abs(fd) + abs(g[name][idx])) + 1e-6, name
    for _ in range(3):
        idx = (0,) + tuple(rng.integers(0, N, size=2))
        xp, xm = x.copy(), x.copy()
        xp[idx] += eps
        xm[idx] -= eps
        fd = (f(P, xp) - f(P, xm)) / (2 * eps)
        assert abs(fd - gx[idx]) <= 1e-5 * (abs(fd) + 1e-3)


def test_bf16_gradients_stay_within_their_rounding_of_the_fp64_gradients():
    """With bf16 the backward products take rounded operands.  The gradients of
    a randomly initialised ReLU network are sensitive: perturbing the weights
    by 2^-9 relative noise alone moves some layers' gradients by 5-16%, and
    the bf16 roundings move them by up to about 30%.  The check is that they
    stay of that size (an error in a rounding point or a dropped term gives
    O(1))."""
    widths = (4, 6, 8, 8)
    N = 16
    P = synth.unet_params_levels(widths, 9)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((1, N, N))
    gy = rng.standard_normal((1, N, N))
    g64, gx64 = L.unet_backward_levels(P, L.unet_forward_levels(P, x, widths)[1], gy, widths)
    g16, gx16 = L.unet_backward_levels(P, L.unet_forward_levels(P, x, widths, bf16=True)[1], gy, widths, bf16=True)
    for k in g64:
        rel = np.linalg.norm(g16[k] - g64[k]) / (np.linalg.norm(g64[k]) + 1e-30)
        assert rel < 0.5, (k, rel)
    assert 1e-4 < np.linalg.norm(gx16 - gx64) / np.linalg.norm(gx64) < 0.5


def test_bfloat16_rounding_is_round_to_nearest_even():
    """round_bf16 against torch's float32 -> bfloat16 conversion (round to
    nearest, ties to even) on random values and on the ties themselves."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-6, 6, 10000),
                        1.0 + np.array([2 ** -8, 3 * 2 ** -8, 2 ** -9, 3 * 2 ** -9, -2 ** -8])])
    want = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(L.round_bf16(x), want)
    assert L.round_bf16(1.0 + 2 ** -8) == 1.0 and L.round_bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6


def test_bf16_network_stays_within_its_rounding_of_the_fp64_network():
    """The bf16 forward differs from the FP64 one by the operand roundings:
    a few 2^-8 relative, far above the FP64 level and far below O(1)."""
    widths = (8, 16, 16)
    N = 16
    P = synth.unet_params_levels(widths, 2)
    x = np.random.default_rng(6).standard_normal((1, N, N))
    y64 = L.unet_forward_levels(P, x, widths)[0]
    y16 = L.unet_forward_levels(P, x, widths, bf16=True)[0]
    rel = np.linalg.norm(y16 - y64) / np.linalg.norm(y64)
    assert 1e-4 < rel < 0.05
