"""GPU parity of the learned right preconditioner (the U-Net and randomized
block flexible GMRES) against the CPU oracle (oracle/learned.py).

The network stores activations in bfloat16 and multiplies bfloat16 operands
with FP32 accumulation; the oracle's bf16 mode rounds at the same points and
sums in FP64.  What is left between the two is FP32 accumulation order and,
where an FP32 value lies within that error of a bfloat16 rounding boundary,
a one-ulp (2^-8) difference in a stored activation, which the following
layers carry on.  An image without such a flip agrees to FP32 level (about
1e-7); with flips the forward output of the four-level network moves by up
to a few 1e-3.  The tolerances below are norm-wise, of that size, and the
tests also check that the GPU is closer to the oracle's bf16 network than to
its FP64 one by at least a factor 2 (a kernel that kept FP32 activations
would match the FP64 network instead).  The gradients of a randomly initialised ReLU network amplify such
flips (the oracle pins show 2^-9 weight noise moving some layers' gradients
by 5-16%), so the gradient check is per layer with a correspondingly looser
bound, and again against the FP64 network for contrast."""
import numpy as np
import pytest

import oracle
import synth
from oracle import learned as L

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

WIDTHS = (16, 32, 64, 64)


@pytest.fixture(scope="module")
def rb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2111_14641_gb300 as rb
    from paper_2111_14641_gb300 import build

    build.build()
    rb.load()
    return rb


def cols(A, dtype=torch.float64):
    """numpy (n x c) -> column-major CUDA tensor."""
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A).T)).to("cuda", dtype).t()


def field_coef(rb, N, seed):
    """Node values a = exp(g) (oracle layout a[i, j], i along x) and the
    device face coefficients."""
    a = np.exp(synth.gaussian_random_field(N, seed))
    fc = rb.diffusion_faces(torch.from_numpy(np.ascontiguousarray(a.T)).cuda())
    return a, fc


def relnorm(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


# ----------------------------------------------------------- the operator --

@pytest.mark.parametrize("N", [1, 7, 37])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_diffusion_operator_matches_oracle(rb, N, prec):
    """-div(a grad u) with harmonic-mean face coefficients against the oracle."""
    a, fc = field_coef(rb, N, 3 + N)
    X = np.random.default_rng(N).standard_normal((N * N, 3))
    if prec == "fp32":
        X = X.astype(np.float32).astype(np.float64)
    op = rb.diffusion_op(N, N, fc)
    Y = rb.op_apply(op, cols(X, torch.float64 if prec == "fp64" else torch.float32)).double().cpu().numpy()
    ref = L.diffusion_apply(a, X)
    tol = 1e-14 if prec == "fp64" else 2e-6
    assert np.abs(Y - ref).max() <= tol * np.abs(ref).max()


def test_plain_block_gmres_on_the_diffusion_operator_matches_oracle(rb):
    """Block GMRES (Sec. 5.2) with the diffusion operator: two cycles against
    the oracle's flexible GMRES with M = I (FP64 basis, Gaussian sketch)."""
    N, mp, p, k = 24, 3, 8, 96
    a, fc = field_coef(rb, N, 5)
    B = synth.gaussian(N * N, mp, 9)
    op = rb.diffusion_op(N, N, fc)
    X, cyc, rel = rb.block_gmres(op, cols(B), None, p=p, rtol=0.0, max_cycles=2, sketch="gauss", k=k, seed=4,
                                 prec="fp64", ls_iters=6)
    Xo, cyco, hist = L.block_fgmres(lambda V: L.diffusion_apply(a, V), None, B, np.zeros_like(B), p, "gauss", k, 4,
                                    0.0, 2)
    assert cyc == cyco == 2
    np.testing.assert_allclose(X.cpu().numpy(), Xo, rtol=0, atol=1e-9 * np.abs(Xo).max())
    assert abs(max(rel) - hist[-1]) <= 1e-8 * hist[-1]


# ------------------------------------------------------------ the network --

def _net_case(N, batch, seed):
    P = synth.unet_params_levels(WIDTHS, seed)
    rng = np.random.default_rng(seed)
    for k in P:
        if k.endswith(".b"):
            P[k] = 0.05 * rng.standard_normal(P[k].shape)
    flat = synth.unet_flat_params(P, WIDTHS)
    # the oracle sees the FP32 parameters the device holds
    P32 = synth.unet_dict_params(flat, WIDTHS)
    X = rng.standard_normal((N * N, batch)).astype(np.float32).astype(np.float64)
    return P32, flat, X


def _img(v, N):
    return v.reshape(1, N, N, order="F")


@pytest.mark.parametrize("N,batch", [(32, 2), (48, 1), (128, 1)])
def test_unet_forward_matches_oracle(rb, N, batch):
    """Four levels, widths 16-32-64-64: the forward pass against the oracle's
    bf16 network (N = 48: levels 48, 24, 12, 6, tiles that do not divide the
    image; N = 128: several 8 x 64 tiles per image at every level)."""
    P, flat, X = _net_case(N, batch, 7)
    Y = rb.unet_forward(WIDTHS, torch.from_numpy(flat).cuda(), N, cols(X, torch.float32)).double().cpu().numpy()
    for b in range(batch):
        ref16 = L.unet_forward_levels(P, _img(X[:, b], N), WIDTHS, bf16=True)[0].reshape(-1, order="F")
        ref64 = L.unet_forward_levels(P, _img(X[:, b], N), WIDTHS)[0].reshape(-1, order="F")
        e16, e64 = relnorm(Y[:, b], ref16), relnorm(Y[:, b], ref64)
        print(f"[unet fwd] N {N} image {b}: vs bf16 oracle {e16:.2e}, vs fp64 oracle {e64:.2e}")
        assert e16 <= 1e-2
        assert e16 <= 0.5 * e64


def test_unet_backward_matches_oracle(rb):
    """Parameter gradients of sum(gy * y) against the oracle's bf16 backward,
    per layer, for two images of 32 x 32."""
    N, batch = 32, 2
    P, flat, X = _net_case(N, batch, 8)
    gy = np.random.default_rng(3).standard_normal((N * N, batch)).astype(np.float32)
    pd = torch.from_numpy(flat).cuda()
    xd = cols(X, torch.float32)
    rb.unet_forward(WIDTHS, pd, N, xd, save=True)
    G = rb.unet_backward(WIDTHS, pd, N, xd, cols(gy, torch.float32)).cpu().numpy()
    Gd = synth.unet_dict_params(G, WIDTHS)
    g16 = {k: 0.0 for k in P}
    g64 = {k: 0.0 for k in P}
    for b in range(batch):
        x = _img(X[:, b], N)
        gyb = _img(gy[:, b].astype(np.float64), N)
        r16, _ = L.unet_backward_levels(P, L.unet_forward_levels(P, x, WIDTHS, bf16=True)[1], gyb, WIDTHS, bf16=True)
        r64, _ = L.unet_backward_levels(P, L.unet_forward_levels(P, x, WIDTHS)[1], gyb, WIDTHS)
        for k in P:
            g16[k] = g16[k] + r16[k]
            g64[k] = g64[k] + r64[k]
    worst16, worst64 = 0.0, 0.0
    for k in P:
        e16, e64 = relnorm(Gd[k], g16[k]), relnorm(Gd[k], g64[k])
        worst16, worst64 = max(worst16, e16), max(worst64, e64)
        assert e16 <= 0.05, (k, e16)
    print(f"[unet bwd] worst layer vs bf16 oracle {worst16:.2e}, vs fp64 oracle {worst64:.2e}")
    assert worst16 <= 0.5 * worst64


@pytest.mark.parametrize("N,batch", [(128, 2), (256, 1)])
def test_tensor_core_forward_matches_simt_and_oracle(rb, N, batch):
    """At N >= 128 the levels with 128-pixel rows run their convolutions on the
    tcgen05 tensor cores (bfloat16 operands, FP32 accumulators in tensor
    memory): against the SIMT kernels (the same roundings, another summation
    order) and, at N = 128, against the oracle's bf16 network."""
    P, flat, X = _net_case(N, batch, 12)
    pd = torch.from_numpy(flat).cuda()
    xd = cols(X, torch.float32)
    Ytc = rb.unet_forward(WIDTHS, pd, N, xd).double().cpu().numpy()
    Ysi = rb.unet_forward(WIDTHS, pd, N, xd, simt=True).double().cpu().numpy()
    for b in range(batch):
        e = relnorm(Ytc[:, b], Ysi[:, b])
        print(f"[unet tc fwd] N {N} image {b}: tensor cores vs SIMT {e:.2e}")
        assert e <= 1e-2
    if N == 128:
        ref16 = L.unet_forward_levels(P, _img(X[:, 0], N), WIDTHS, bf16=True)[0].reshape(-1, order="F")
        ref64 = L.unet_forward_levels(P, _img(X[:, 0], N), WIDTHS)[0].reshape(-1, order="F")
        e16, e64 = relnorm(Ytc[:, 0], ref16), relnorm(Ytc[:, 0], ref64)
        print(f"[unet tc fwd] N {N}: vs bf16 oracle {e16:.2e}, vs fp64 oracle {e64:.2e}")
        assert e16 <= 1e-2 and e16 <= 0.5 * e64


def test_tensor_core_backward_matches_simt_and_oracle(rb):
    """Parameter gradients with the tensor-core forward and backward
    convolutions (levels of 128 and more pixels per row) against the SIMT
    path, and against the oracle's bf16 backward, per layer."""
    N, batch = 128, 1
    P, flat, X = _net_case(N, batch, 13)
    gy = np.random.default_rng(4).standard_normal((N * N, batch)).astype(np.float32)
    pd = torch.from_numpy(flat).cuda()
    xd, gyd = cols(X, torch.float32), cols(gy, torch.float32)
    rb.unet_forward(WIDTHS, pd, N, xd, save=True)
    Gtc = synth.unet_dict_params(rb.unet_backward(WIDTHS, pd, N, xd, gyd).cpu().numpy(), WIDTHS)
    rb.unet_forward(WIDTHS, pd, N, xd, save=True, simt=True)
    Gsi = synth.unet_dict_params(rb.unet_backward(WIDTHS, pd, N, xd, gyd, simt=True).cpu().numpy(), WIDTHS)
    x = _img(X[:, 0], N)
    g16, _ = L.unet_backward_levels(P, L.unet_forward_levels(P, x, WIDTHS, bf16=True)[1],
                                    _img(gy[:, 0].astype(np.float64), N), WIDTHS, bf16=True)
    worst_si = worst_or = 0.0
    for k in P:
        es, eo = relnorm(Gtc[k], Gsi[k]), relnorm(Gtc[k], g16[k])
        worst_si, worst_or = max(worst_si, es), max(worst_or, eo)
        assert es <= 0.05 and eo <= 0.05, (k, es, eo)
    print(f"[unet tc bwd] worst layer: vs SIMT {worst_si:.2e}, vs bf16 oracle {worst_or:.2e}")


def test_backward_needs_a_saved_forward(rb):
    N = 16
    flat = synth.unet_flat_params(synth.unet_params_levels(WIDTHS, 1), WIDTHS)
    rb.release_workspace()
    x = torch.zeros((1, N * N), dtype=torch.float32, device="cuda").t()
    with pytest.raises(rb.RbgsError):
        rb.unet_backward(WIDTHS, torch.from_numpy(flat).cuda(), N, x, x)


def test_residual_loss_and_gradient_match_oracle(rb):
    """L = 1/2 mean (B_f y - x)^2 over a batch of images of two fields, and
    dL/dy = B_f (B_f y - x) / total, against the oracle's definition in FP64
    on the same x and y."""
    N = 20
    n = N * N
    fields = [field_coef(rb, N, s) for s in (11, 12)]
    coef = torch.stack([f[1] for f in fields])
    which = np.array([1, 0, 1], dtype=np.int32)
    rng = np.random.default_rng(0)
    X = rng.standard_normal((n, 3)).astype(np.float32).astype(np.float64)
    Y = rng.standard_normal((n, 3)).astype(np.float32).astype(np.float64)
    loss, gy = rb.unet_residual_loss(N, coef, torch.from_numpy(which).cuda(), cols(X, torch.float32),
                                     cols(Y, torch.float32))
    hh8 = (1.0 / (N + 1)) ** 2 / 8.0
    res = np.column_stack([hh8 * L.diffusion_apply(fields[f][0], Y[:, j]) - X[:, j] for j, f in enumerate(which)])
    want = 0.5 * np.mean(res ** 2)
    gwant = np.column_stack([hh8 * L.diffusion_apply(fields[f][0], res[:, j]) for j, f in enumerate(which)]) / res.size
    assert abs(float(loss.item()) - want) <= 1e-5 * want
    assert relnorm(gy.double().cpu().numpy(), gwant) <= 1e-5


def test_adam_step_matches_oracle(rb):
    rng = np.random.default_rng(1)
    p = rng.standard_normal(1000).astype(np.float32)
    g = rng.standard_normal(1000).astype(np.float32)
    pd, gd = torch.from_numpy(p.copy()).cuda(), torch.from_numpy(g).cuda()
    m, v = torch.zeros_like(pd), torch.zeros_like(pd)
    params = {"w": p.astype(np.float64)}
    state = {}
    for t in (1, 2, 3):
        rb.adam_step(pd, gd, m, v, t, lr=1e-2)
        L.adam_step(params, {"w": g.astype(np.float64)}, state, lr=1e-2)
    np.testing.assert_allclose(pd.cpu().numpy(), params["w"], rtol=0, atol=1e-6)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_precondition_matches_oracle(rb, prec):
    """Z = M(Q): per-column scaling around the network, against the oracle
    (bf16 network); a zero column gives zero and M is positively homogeneous."""
    N = 32
    P, flat, _ = _net_case(N, 1, 9)
    Q = np.random.default_rng(2).standard_normal((N * N, 3)) * np.array([1e-3, 1.0, 0.0])
    td = torch.float64 if prec == "fp64" else torch.float32
    if prec == "fp32":
        Q = Q.astype(np.float32).astype(np.float64)
    pd = torch.from_numpy(flat).cuda()
    Z = rb.unet_precondition(WIDTHS, pd, N, cols(Q, td)).double().cpu().numpy()
    ref = L.precondition_levels(P, Q, WIDTHS, bf16=True)
    assert relnorm(Z[:, :2], ref[:, :2]) <= 2e-3
    assert np.all(Z[:, 2] == 0.0)
    Z2 = rb.unet_precondition(WIDTHS, pd, N, cols(3.0 * Q, td)).double().cpu().numpy()
    assert relnorm(Z2[:, :2], 3.0 * Z[:, :2]) <= 1e-5


def test_fgmres_with_an_untrained_network_matches_oracle_and_falls_back(rb):
    """Flexible block GMRES with the (untrained) U-Net: the GPU's relative
    residual history follows the oracle's flexible GMRES with the same bf16
    network, fallbacks included, and the fallback keeps it converging."""
    N, mp, p, k = 32, 2, 6, 48
    a, fc = field_coef(rb, N, 21)
    P, flat, _ = _net_case(N, 1, 10)
    B = synth.gaussian(N * N, mp, 4)
    op = rb.diffusion_op(N, N, fc)
    pd = torch.from_numpy(flat).cuda()
    hist = []
    X = None
    fb_total = 0
    for _ in range(3):
        X, cyc, rel, fb = rb.block_fgmres(op, WIDTHS, pd, cols(B), X, p=p, rtol=0.0, max_cycles=1, accept=0.9,
                                          sketch="gauss", k=k, seed=6, prec="fp64", ls_iters=6)
        hist.append(max(rel))
        fb_total += fb
    Xo, cyco, ho, rec = L.block_fgmres(lambda V: L.diffusion_apply(a, V),
                                       lambda V: L.precondition_levels(P, V, WIDTHS, bf16=True), B, np.zeros_like(B),
                                       p, "gauss", k, 6, 0.0, 3, record=True, accept=0.9)
    print(f"[fgmres] gpu {hist} fallbacks {fb_total}; oracle {ho[1:]} fallbacks {rec['fallbacks']}")
    assert fb_total == rec["fallbacks"]
    for g, o in zip(hist, ho[1:]):
        assert abs(g - o) <= 1e-2 * o
    assert hist[-1] < hist[0]


def test_plain_and_flexible_agree_without_a_network(rb):
    """net = NULL runs plain block GMRES: identical to rbgs_block_gmres."""
    N, mp, p, k = 16, 2, 5, 40
    a, fc = field_coef(rb, N, 2)
    B = synth.gaussian(N * N, mp, 1)
    op = rb.diffusion_op(N, N, fc)
    X1, c1, r1, fb = rb.block_fgmres(op, None, None, cols(B), None, p=p, rtol=0.0, max_cycles=2, sketch="gauss", k=k,
                                     seed=3, prec="fp64", ls_iters=3)
    X2, c2, r2 = rb.block_gmres(op, cols(B), None, p=p, rtol=0.0, max_cycles=2, sketch="gauss", k=k, seed=3,
                                prec="fp64", ls_iters=3)
    assert c1 == c2 == 2 and fb == 0
    assert torch.equal(X1, X2)


# ------------------------------------------------------- training on the GPU --

def _training_pairs(rb, N, mp, p, k, fields):
    """The inputs M sees inside flexible GMRES: the Arnoldi bases of three
    plain block GMRES cycles per field (as the oracle's training test), scaled
    to unit root mean square by the library; returns (X, field index per
    column, stacked face coefficients)."""
    n = N * N
    xs, fid, coefs = [], [], []
    for f, s in enumerate(fields):
        a, fc = field_coef(rb, N, s)
        coefs.append(fc)
        op = rb.diffusion_op(N, N, fc)
        B = cols(synth.gaussian(n, mp, 100 + s))
        X = torch.zeros((mp, n), dtype=torch.float64, device="cuda").t()
        for _ in range(3):
            R = B - rb.op_apply(op, X)
            Q, _ = rb.block_arnoldi(op, rb.colmajor(R), p=p, sketch="gauss", k=k, seed=1, prec="fp64", ls_iters=6)
            xs.append(rb.unet_scale_inputs(Q))
            fid += [f] * Q.shape[1]
            X, _, _ = rb.block_gmres(op, B, X, p=p, rtol=0.0, max_cycles=1, sketch="gauss", k=k, seed=1, prec="fp64",
                                     ls_iters=6)
    Xall = torch.cat([x.t() for x in xs], dim=0).t()  # column-major n x pairs
    return Xall, torch.tensor(fid, dtype=torch.int32, device="cuda"), torch.stack(coefs)


def _mean_loss(rb, widths, params, N, X, fid, coef):
    y = rb.unet_forward(widths, params, N, X)
    loss, _ = rb.unet_residual_loss(N, coef, fid, X, y)
    return float(loss.item())


def test_gpu_training_lowers_the_loss_and_beats_plain_gmres_on_an_unseen_field(rb):
    """The oracle's training recipe on the GPU, by the library's own forward,
    backward, residual-loss and Adam kernels: the two-level network of widths
    (8, 16) (the oracle's c = 8 network), trained on the Arnoldi bases of
    three plain block GMRES cycles on each of six random fields (216 pairs),
    2000 Adam steps of four random pairs at learning rate 1e-3.  The loss
    falls below a quarter of its start, and on an unseen field flexible GMRES
    with the network reaches 1e-8 in fewer cycles than plain block GMRES, which
    is still above 1e-8 by then."""
    N, mp, p, k = 16, 2, 6, 48
    n = N * N
    widths = (8, 16)
    X, fid, coef = _training_pairs(rb, N, mp, p, k, [100 + s for s in range(6)])
    assert X.shape[1] == 216
    params = torch.from_numpy(synth.unet_flat_params(synth.unet_params_levels(widths, 21), widths)).cuda()
    m, v = torch.zeros_like(params), torch.zeros_like(params)
    grads = torch.empty_like(params)
    loss0 = _mean_loss(rb, widths, params, N, X, fid, coef)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(0)
    bs = 4
    for step in range(1, 2001):
        idx = torch.randint(0, X.shape[1], (bs,), device="cuda", generator=gen)
        xb = X[:, idx].t().contiguous().t()
        fb = fid[idx].contiguous()
        y = rb.unet_forward(widths, params, N, xb, save=True, sync=False)
        _, gy = rb.unet_residual_loss(N, coef, fb, xb, y, sync=False)
        rb.unet_backward(widths, params, N, xb, gy, grads=grads, sync=False)
        rb.adam_step(params, grads, m, v, step, lr=1e-3, sync=False)
    loss1 = _mean_loss(rb, widths, params, N, X, fid, coef)
    print(f"[train] mean loss {loss0:.3f} -> {loss1:.3f}")
    assert loss1 < 0.25 * loss0
    # an unseen field
    a, fc = field_coef(rb, N, 998)
    op = rb.diffusion_op(N, N, fc)
    B = cols(synth.gaussian(n, mp, 1005))
    _, cyc_l, rel_l, fbk = rb.block_fgmres(op, widths, params, B, None, p=p, rtol=1e-8, max_cycles=80, accept=0.9,
                                           sketch="gauss", k=k, seed=1, prec="fp64", ls_iters=6)
    _, cyc_p, rel_p, _ = rb.block_fgmres(op, None, None, B, None, p=p, rtol=1e-8, max_cycles=cyc_l, sketch="gauss",
                                         k=k, seed=1, prec="fp64", ls_iters=6)
    print(f"[train] unseen field: learned {cyc_l} cycles ({fbk} fallbacks, {max(rel_l):.1e}); "
          f"plain after {cyc_p} cycles {max(rel_p):.1e}")
    assert max(rel_l) <= 1e-8
    assert max(rel_p) > 1e-8
    assert fbk < cyc_l
