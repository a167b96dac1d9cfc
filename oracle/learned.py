"""CPU oracle for the learned right preconditioner: randomized block flexible
GMRES on random-coefficient diffusion problems, with a small U-Net as the
preconditioner.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this module:
only tests/ use it.  Plain FP64 numpy, written step by step; a library
primitive (a QR, a least-squares solve, a sparse direct solve) serves as a
step where one is named.

None of this is in the paper, which preconditions its block GMRES with
ILU(0) (Sec. 5, second experiment).  What it builds on is the paper's:

* the Krylov layer: RBGS-Arnoldi (Alg. 7) with steps 4-5 by Alg. 5 and step 2
  by Householder least squares, and block GMRES by the sketched minimal
  residual (Sec. 5.2);
* the flexible variant of GMRES (Saad, SIAM J. Sci. Comput. 14, 1993): the
  j-th Arnoldi block is expanded through Z_j = M(Q_j) with a preconditioner
  M that may change (here: a nonlinear network), the solution is corrected
  by Z z instead of Q z, and the small problem is unchanged.

The problem: -div(a grad u) = f on the unit square, N x N interior nodes,
h = 1/(N+1), zero Dirichlet boundary, a > 0 given at all (N+2)^2 nodes; the
cell-centred five-point scheme with harmonic-mean face coefficients.  The
unknown at node (ix, iy) (1-based interior) is entry (ix-1) + N (iy-1).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sps
import scipy.sparse.linalg as spsl

from . import householder_qr, ls_solve, theta_apply

# ----------------------------------------------------------- the operator --


def face_coefficients(a):
    """Harmonic means of a on the faces between neighbouring nodes:
    ax[i, j] between nodes (i, j) and (i+1, j), shape (N+1, N+2);
    ay[i, j] between nodes (i, j) and (i, j+1), shape (N+2, N+1)."""
    a = np.asarray(a, dtype=np.float64)
    ax = 2.0 * a[:-1, :] * a[1:, :] / (a[:-1, :] + a[1:, :])
    ay = 2.0 * a[:, :-1] * a[:, 1:] / (a[:, :-1] + a[:, 1:])
    return ax, ay


def diffusion_apply(a, X) -> np.ndarray:
    """Y = A X, (A u)_node = sum over the four faces of a_face (u_node -
    u_neighbour) / h^2, boundary values zero."""
    a = np.asarray(a, dtype=np.float64)
    N = a.shape[0] - 2
    h = 1.0 / (N + 1)
    ax, ay = face_coefficients(a)
    X = np.asarray(X, dtype=np.float64)
    one = X.ndim == 1
    X = X.reshape(N * N, -1, order="F")
    Y = np.zeros_like(X)
    for c in range(X.shape[1]):
        P = np.zeros((N + 2, N + 2))
        P[1:-1, 1:-1] = X[:, c].reshape(N, N, order="F")
        u = P[1:-1, 1:-1]
        y = (ax[1:, 1:-1] * (u - P[2:, 1:-1]) + ax[:-1, 1:-1] * (u - P[:-2, 1:-1])
             + ay[1:-1, 1:] * (u - P[1:-1, 2:]) + ay[1:-1, :-1] * (u - P[1:-1, :-2])) / h ** 2
        Y[:, c] = y.reshape(-1, order="F")
    return Y[:, 0] if one else Y


def diffusion_matrix(a) -> sps.csr_matrix:
    """The same operator assembled entry by entry (for direct solves)."""
    a = np.asarray(a, dtype=np.float64)
    N = a.shape[0] - 2
    h2 = (1.0 / (N + 1)) ** 2
    ax, ay = face_coefficients(a)
    rows, cols, vals = [], [], []

    def idx(i, j):  # 1-based interior node -> unknown
        return (i - 1) + N * (j - 1)

    for j in range(1, N + 1):
        for i in range(1, N + 1):
            faces = [(ax[i, j], i + 1, j), (ax[i - 1, j], i - 1, j), (ay[i, j], i, j + 1), (ay[i, j - 1], i, j - 1)]
            diag = 0.0
            for coef, ii, jj in faces:
                diag += coef
                if 1 <= ii <= N and 1 <= jj <= N:
                    rows.append(idx(i, j))
                    cols.append(idx(ii, jj))
                    vals.append(-coef / h2)
            rows.append(idx(i, j))
            cols.append(idx(i, j))
            vals.append(diag / h2)
    return sps.csr_matrix((vals, (rows, cols)), shape=(N * N, N * N))


# -------------------------------------------- the Krylov layer (Alg. 7) --


class SketchedBasis:
    """Q (n x c), S = Theta Q (k x c) and R (c x c), grown one block at a time
    by Alg. 2: step 1 P = Theta W; step 2 X = argmin ||S X - P|| (Householder);
    step 3 Q' = W - Q X; steps 4-5 by Alg. 5: R_ii = R of qr(P - S X) with a
    positive diagonal, Q_i = Q' R_ii^{-1}, S_i = Theta Q_i."""

    def __init__(self, n: int, kind: str, k: int, seed: int):
        self.n, self.kind, self.k, self.seed = n, kind, k, seed
        self.Q = np.zeros((n, 0))
        self.S = np.zeros((k, 0))
        self.R = np.zeros((0, 0))

    def add(self, W) -> np.ndarray:
        W = np.asarray(W, dtype=np.float64).reshape(self.n, -1)
        mb = W.shape[1]
        c = self.Q.shape[1]
        P = theta_apply(self.kind, self.k, self.seed, W)
        X = ls_solve(self.S, P, "householder") if c else np.zeros((0, mb))
        Qp = W - self.Q @ X
        Sp = P - self.S @ X
        _, Rii, rc = householder_qr(Sp)
        if rc:
            raise np.linalg.LinAlgError("breakdown: rank-deficient sketched block")
        Qi = np.linalg.solve(Rii.T, Qp.T).T
        Si = theta_apply(self.kind, self.k, self.seed, Qi)
        R = np.zeros((c + mb, c + mb))
        R[:c, :c] = self.R
        R[:c, c:] = X
        R[c:, c:] = Rii
        self.Q = np.hstack([self.Q, Qi])
        self.S = np.hstack([self.S, Si])
        self.R = R
        return R[:, c:]


def _fgmres_cycle(apply_A, precond, r, p: int, kind: str, k: int, seed: int):
    """One cycle on the residual block r: (the correction Z_{1:p-1} z, Q_{1:p})."""
    n, mp = r.shape
    basis = SketchedBasis(n, kind, k, seed)
    basis.add(r)
    Z = []
    for j in range(p - 1):
        Qj = basis.Q[:, j * mp:(j + 1) * mp]
        Zj = Qj if precond is None else precond(Qj)
        Z.append(Zj)
        basis.add(apply_A(Zj))
    H = basis.R[:, mp:]
    F = basis.R[:, :mp]
    z = np.linalg.lstsq(H, F, rcond=None)[0]
    return np.hstack(Z) @ z, basis.Q


def block_fgmres(apply_A, precond, B, X0, p: int, kind: str, k: int, seed: int, rtol: float, max_cycles: int,
                 record: bool = False, accept: float | None = None):
    """Restarted randomized block flexible GMRES.  Each cycle runs the
    Arnoldi process on r = B - A X: Q_1 R_11 = r, then for j = 1..p-1
    Z_j = precond(Q_j) and W_{j+1} = A Z_j, so that A Z_{1:p-1} = Q_{1:p} H
    with H = R_{(1:p,2:p)}; z = argmin ||H z - R_{(1:p,1)}|| (the sketched
    residual, Theta Q being orthonormal) and X <- X + Z_{1:p-1} z.
    precond=None is M = I (plain block GMRES).

    With accept = a (0 < a <= 1) plain block GMRES is the fallback and the
    true residual decides: a preconditioned cycle is kept only when it
    brings max_j ||r_j|| / ||b_j|| down to at most a times its value before
    the cycle; otherwise the cycle is run again from the same X with M = I.

    Stops when max_j ||r_j|| / ||b_j|| <= rtol or after max_cycles cycles.
    Returns (X, cycles, history of that ratio), plus with record=True a dict
    with the residual blocks seen at the start of each cycle ("residuals"),
    the Arnoldi bases Q_{1:p} of the kept cycles ("bases") and the number of
    cycles that fell back to M = I ("fallbacks")."""
    B = np.asarray(B, dtype=np.float64)
    n, mp = B.shape
    X = np.array(X0, dtype=np.float64, copy=True).reshape(n, mp)
    bn = np.linalg.norm(B, axis=0)

    def ratio(XX):
        rr = B - apply_A(XX)
        return rr, float(np.max(np.linalg.norm(rr, axis=0) / bn))

    hist = []
    rec = dict(residuals=[], bases=[], fallbacks=0)
    cyc = 0
    r, rel = ratio(X)
    while True:
        hist.append(rel)
        if record:
            rec["residuals"].append(r.copy())
        if rel <= rtol or cyc >= max_cycles:
            break
        dX, Qb = _fgmres_cycle(apply_A, precond, r, p, kind, k, seed)
        rn, reln = ratio(X + dX)
        if accept is not None and precond is not None and reln > accept * rel:
            rec["fallbacks"] += 1
            dX, Qb = _fgmres_cycle(apply_A, None, r, p, kind, k, seed)
            rn, reln = ratio(X + dX)
        if record:
            rec["bases"].append(Qb)
        X, r, rel = X + dX, rn, reln
        cyc += 1
    return (X, cyc, hist, rec) if record else (X, cyc, hist)


# --------------------------------------------------------------- the U-Net --
# Layers (3 x 3 convolutions, zero padding, stride 1):
#   a1 = relu(conv_e1(x))  1 -> c        a2 = relu(conv_e2(a1))  c -> c
#   d  = avgpool2(a2)                    (half resolution)
#   b1 = relu(conv_m1(d))  c -> 2c       b2 = relu(conv_m2(b1))  2c -> 2c
#   u  = upsample2(b2)                   (nearest neighbour)
#   o  = relu(conv_o1([u; a2]))  3c -> c   y = conv_o2(o)  c -> 1 (linear)
# x and y are single-channel N x N images (N even); see precondition() for
# the scaling around the network.


def conv3x3(x, w, b):
    """y[o, i, j] = b[o] + sum_{c, s, t} w[o, c, s, t] x[c, i + s - 1, j + t - 1]
    (x zero outside the image): cross-correlation, as in CNN libraries."""
    C, H, W = x.shape
    xp = np.zeros((C, H + 2, W + 2))
    xp[:, 1:-1, 1:-1] = x
    y = np.broadcast_to(b[:, None, None], (w.shape[0], H, W)).copy()
    for s in range(3):
        for t in range(3):
            y += np.einsum("oc,chw->ohw", w[:, :, s, t], xp[:, s:s + H, t:t + W])
    return y


def conv3x3_backward(x, w, gy):
    """Gradients of sum(gy * conv3x3(x, w, b)) with respect to x, w and b."""
    C, H, W = x.shape
    xp = np.zeros((C, H + 2, W + 2))
    xp[:, 1:-1, 1:-1] = x
    dw = np.zeros_like(w)
    dxp = np.zeros_like(xp)
    for s in range(3):
        for t in range(3):
            dw[:, :, s, t] = np.einsum("ohw,chw->oc", gy, xp[:, s:s + H, t:t + W])
            dxp[:, s:s + H, t:t + W] += np.einsum("oc,ohw->chw", w[:, :, s, t], gy)
    return dxp[:, 1:-1, 1:-1], dw, gy.sum(axis=(1, 2))


def avgpool2(x):
    C, H, W = x.shape
    return x.reshape(C, H // 2, 2, W // 2, 2).mean(axis=(2, 4))


def avgpool2_backward(gy):
    return np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2) / 4.0


def upsample2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample2_backward(gy):
    C, H, W = gy.shape
    return gy.reshape(C, H // 2, 2, W // 2, 2).sum(axis=(2, 4))


def unet_forward(params: dict, x):
    """y = U-Net(x) for x (1, N, N); returns (y, cache for the backward pass)."""
    P = params
    z1 = conv3x3(x, P["e1.w"], P["e1.b"])
    a1 = np.maximum(z1, 0.0)
    z2 = conv3x3(a1, P["e2.w"], P["e2.b"])
    a2 = np.maximum(z2, 0.0)
    d = avgpool2(a2)
    z3 = conv3x3(d, P["m1.w"], P["m1.b"])
    b1 = np.maximum(z3, 0.0)
    z4 = conv3x3(b1, P["m2.w"], P["m2.b"])
    b2 = np.maximum(z4, 0.0)
    u = upsample2(b2)
    cat = np.concatenate([u, a2], axis=0)
    z5 = conv3x3(cat, P["o1.w"], P["o1.b"])
    o = np.maximum(z5, 0.0)
    y = conv3x3(o, P["o2.w"], P["o2.b"])
    cache = dict(x=x, z1=z1, a1=a1, z2=z2, a2=a2, d=d, z3=z3, b1=b1, z4=z4, b2=b2, cat=cat, z5=z5, o=o)
    return y, cache


def unet_backward(params: dict, cache: dict, gy):
    """Gradients of sum(gy * y) with respect to every parameter and to x."""
    P, C = params, cache
    g = {}
    go, g["o2.w"], g["o2.b"] = conv3x3_backward(C["o"], P["o2.w"], gy)
    gz5 = go * (C["z5"] > 0)
    gcat, g["o1.w"], g["o1.b"] = conv3x3_backward(C["cat"], P["o1.w"], gz5)
    c2 = C["b2"].shape[0]
    gu, ga2 = gcat[:c2], gcat[c2:].copy()
    gb2 = upsample2_backward(gu)
    gz4 = gb2 * (C["z4"] > 0)
    gb1, g["m2.w"], g["m2.b"] = conv3x3_backward(C["b1"], P["m2.w"], gz4)
    gz3 = gb1 * (C["z3"] > 0)
    gd, g["m1.w"], g["m1.b"] = conv3x3_backward(C["d"], P["m1.w"], gz3)
    ga2 += avgpool2_backward(gd)
    gz2 = ga2 * (C["z2"] > 0)
    ga1, g["e2.w"], g["e2.b"] = conv3x3_backward(C["a1"], P["e2.w"], gz2)
    gz1 = ga1 * (C["z1"] > 0)
    gx, g["e1.w"], g["e1.b"] = conv3x3_backward(C["x"], P["e1.w"], gz1)
    return g, gx


# ------------------------------------------------- the L-level U-Net --
# The same network with L levels of widths c_0 .. c_{L-1} (level l at 1/2^l of
# the resolution; N divisible by 2^(L-1)):
#   encoder, l = 0 .. L-1:  a = relu(conv_enc{l}a(x_l)), s_l = relu(conv_enc{l}b(a)),
#                           x_0 = the input (1 channel), x_{l+1} = avgpool2(s_l)
#   decoder, l = L-2 .. 0:  d_l = relu(conv_dec{l}([upsample2(d_{l+1}); s_l])),
#                           d_{L-1} = s_{L-1}
#   output:                 y = conv_out(d_0)  (c_0 -> 1, linear)
# With L = 2 and widths (c, 2c) it is the two-level network above
# (enc0a = e1, enc0b = e2, enc1a = m1, enc1b = m2, dec0 = o1, out = o2).
# bf16=True rounds every convolution's operands (its input activations or
# gradients, and its weights) to bfloat16 after rounding them to FP32, the
# points where a network that stores activations in bfloat16 and computes in
# FP32 rounds; the sums stay in FP64.


def unet_layers(widths) -> list:
    """[(name, C_in, C_out, relu)] of the L-level network, in evaluation order."""
    L = len(widths)
    out = []
    for l in range(L):
        out.append((f"enc{l}a", 1 if l == 0 else widths[l - 1], widths[l], True))
        out.append((f"enc{l}b", widths[l], widths[l], True))
    for l in range(L - 2, -1, -1):
        out.append((f"dec{l}", widths[l + 1] + widths[l], widths[l], True))
    out.append(("out", widths[0], 1, False))
    return out


def round_bf16(x) -> np.ndarray:
    """x rounded to FP32, then to bfloat16 (round to nearest, ties to even),
    returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(f.shape)


def _conv_fwd(x, w, b, bf16):
    if bf16:
        return conv3x3(round_bf16(x), round_bf16(w), b)
    return conv3x3(x, w, b)


def _conv_bwd(x, w, gz, bf16):
    """conv3x3_backward with the operands of the two backward products
    rounded as the forward ones: x and gz for the weights, w and gz for x."""
    if bf16:
        gx, gw, _ = conv3x3_backward(round_bf16(x), round_bf16(w), round_bf16(gz))
        return gx, gw, gz.sum(axis=(1, 2))
    return conv3x3_backward(x, w, gz)


def unet_forward_levels(params: dict, x, widths, bf16: bool = False):
    """y = U-Net(x) of the L-level network, x (1, N, N); returns (y, cache)."""
    L = len(widths)
    P = params
    cache = {"x": x}
    skips = []
    h = x
    for l in range(L):
        if l > 0:
            h = avgpool2(skips[-1])
            cache[f"pool{l}"] = h
        cache[f"in_enc{l}a"] = h
        z = _conv_fwd(h, P[f"enc{l}a.w"], P[f"enc{l}a.b"], bf16)
        a = np.maximum(z, 0.0)
        if bf16:
            a = round_bf16(a)
        cache[f"z_enc{l}a"], cache[f"in_enc{l}b"] = z, a
        z = _conv_fwd(a, P[f"enc{l}b.w"], P[f"enc{l}b.b"], bf16)
        s_l = np.maximum(z, 0.0)
        if bf16:
            s_l = round_bf16(s_l)
        cache[f"z_enc{l}b"] = z
        skips.append(s_l)
    d = skips[L - 1]
    for l in range(L - 2, -1, -1):
        cat = np.concatenate([upsample2(d), skips[l]], axis=0)
        cache[f"in_dec{l}"] = cat
        z = _conv_fwd(cat, P[f"dec{l}.w"], P[f"dec{l}.b"], bf16)
        d = np.maximum(z, 0.0)
        if bf16:
            d = round_bf16(d)
        cache[f"z_dec{l}"] = z
    cache["in_out"] = d
    y = _conv_fwd(d, P["out.w"], P["out.b"], bf16)
    return y, cache


def unet_backward_levels(params: dict, cache: dict, gy, widths, bf16: bool = False):
    """Gradients of sum(gy * y) of the L-level network with respect to every
    parameter and to x."""
    L = len(widths)
    P, C = params, cache
    g = {}
    gd, g["out.w"], g["out.b"] = _conv_bwd(C["in_out"], P["out.w"], gy, bf16)
    gskip = [None] * L
    for l in range(0, L - 1):
        gz = gd * (C[f"z_dec{l}"] > 0)
        gcat, g[f"dec{l}.w"], g[f"dec{l}.b"] = _conv_bwd(C[f"in_dec{l}"], P[f"dec{l}.w"], gz, bf16)
        cu = widths[l + 1]
        gskip[l] = gcat[cu:].copy()
        gd = upsample2_backward(gcat[:cu])
    gs = gd  # gradient of s_{L-1}
    gx = None
    for l in range(L - 1, -1, -1):
        if l < L - 1:
            gs = gskip[l] + gs_from_pool
        gz = gs * (C[f"z_enc{l}b"] > 0)
        ga, g[f"enc{l}b.w"], g[f"enc{l}b.b"] = _conv_bwd(C[f"in_enc{l}b"], P[f"enc{l}b.w"], gz, bf16)
        gz = ga * (C[f"z_enc{l}a"] > 0)
        gh, g[f"enc{l}a.w"], g[f"enc{l}a.b"] = _conv_bwd(C[f"in_enc{l}a"], P[f"enc{l}a.w"], gz, bf16)
        if l > 0:
            gs_from_pool = avgpool2_backward(gh)
        else:
            gx = gh
    return g, gx


def precondition_levels(params: dict, R, widths, bf16: bool = False) -> np.ndarray:
    """precondition() with the L-level network: z = s (h^2 / 8) U-Net(r / s)
    per column, s = ||r|| / sqrt(n) (zero columns give zero).  With bf16 the
    scaled input r / s is rounded to FP32 first, as a network with FP32 inputs
    receives it."""
    R = np.asarray(R, dtype=np.float64)
    one = R.ndim == 1
    R = R.reshape(R.shape[0], -1)
    n = R.shape[0]
    N = int(round(np.sqrt(n)))
    hh8 = (1.0 / (N + 1)) ** 2 / 8.0
    Z = np.zeros_like(R)
    for j in range(R.shape[1]):
        s = np.linalg.norm(R[:, j]) / np.sqrt(n)
        if s == 0.0:
            continue
        x = (R[:, j] / s).reshape(1, N, N, order="F")
        if bf16:
            x = x.astype(np.float32).astype(np.float64)
        y, _ = unet_forward_levels(params, x, widths, bf16=bf16)
        Z[:, j] = s * hh8 * y[0].reshape(-1, order="F")
    return Z[:, 0] if one else Z


def precondition(params: dict, R) -> np.ndarray:
    """Z = M(R), column by column: s = ||r|| / sqrt(n) (zero columns give zero),
    z = s (h^2 / 8) vec(U-Net(r / s as an N x N image)), an approximation of
    A^{-1} r once the network approximates the inverse of A h^2 / 8 (see
    pair_loss_and_grad).  M(alpha r) = alpha M(r) for alpha > 0."""
    R = np.asarray(R, dtype=np.float64)
    one = R.ndim == 1
    R = R.reshape(R.shape[0], -1)
    n = R.shape[0]
    N = int(round(np.sqrt(n)))
    hh8 = (1.0 / (N + 1)) ** 2 / 8.0
    Z = np.zeros_like(R)
    for j in range(R.shape[1]):
        s = np.linalg.norm(R[:, j]) / np.sqrt(n)
        if s == 0.0:
            continue
        y, _ = unet_forward(params, (R[:, j] / s).reshape(1, N, N, order="F"))
        Z[:, j] = s * hh8 * y[0].reshape(-1, order="F")
    return Z[:, 0] if one else Z


def correction_targets(a, R) -> np.ndarray:
    """E = A^{-1} R by a sparse direct solve: the exact corrections the
    network learns (residual r -> error e with A e = r)."""
    A = diffusion_matrix(a).tocsc()
    lu = spsl.splu(A)
    R = np.asarray(R, dtype=np.float64).reshape(A.shape[0], -1)
    return np.column_stack([lu.solve(R[:, j]) for j in range(R.shape[1])])


def pair_loss_and_grad(params: dict, a, r, e=None, loss: str = "residual"):
    """Loss of one (residual, correction) pair r, e = A^{-1} r and its gradients.
    With s = ||r|| / sqrt(n), x = r / s, y = U-Net(x) and B = A h^2 / 8 (its
    spectrum inside (0, 1]), the network's target is B^{-1} x = (8 / h^2) e / s:
      "residual":   L = 1/2 mean((B y - x)^2), the target error measured in the
                    residual norm ||B (y - B^{-1} x)||, which is what flexible
                    GMRES needs of M (A M(q) close to q); e is not used;
      "correction": L = 1/2 mean((y - t)^2), t = e / ||e|| * sqrt(n), the
                    direction of the correction in the plain 2-norm.
    Returns (L, gradients)."""
    n = r.size
    N = int(round(np.sqrt(n)))
    hh8 = (1.0 / (N + 1)) ** 2 / 8.0
    s = np.linalg.norm(r) / np.sqrt(n)
    x = (r / s).reshape(1, N, N, order="F")
    y, cache = unet_forward(params, x)
    if loss == "residual":
        res = hh8 * diffusion_apply(a, y[0].reshape(-1, order="F")) - x.reshape(-1, order="F")
        val = 0.5 * float(np.mean(res ** 2))
        gy = hh8 * diffusion_apply(a, res / res.size)  # B is symmetric: the gradient is B^T res / n
        g, _ = unet_backward(params, cache, gy.reshape(1, N, N, order="F"))
        return val, g
    t = (e / (np.linalg.norm(e) / np.sqrt(n))).reshape(1, N, N, order="F")
    diff = y - t
    g, _ = unet_backward(params, cache, diff / diff.size)
    return 0.5 * float(np.mean(diff ** 2)), g


def adam_step(params: dict, grads: dict, state: dict, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8) -> None:
    """One Adam update (Kingma and Ba, ICLR 2015), in place: first and second
    moment estimates with bias correction; state holds t, m, v."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for name, g in grads.items():
        m = state.setdefault("m." + name, np.zeros_like(g))
        v = state.setdefault("v." + name, np.zeros_like(g))
        m *= beta1
        m += (1.0 - beta1) * g
        v *= beta2
        v += (1.0 - beta2) * g * g
        mhat = m / (1.0 - beta1 ** t)
        vhat = v / (1.0 - beta2 ** t)
        params[name] = params[name] - lr * mhat / (np.sqrt(vhat) + eps)
