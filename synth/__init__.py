"""Seeded synthetic inputs shared by the tests, the oracle runs and bench.py.

This module holds none of the method's arithmetic: it only draws matrices with
prescribed structure.  Recipes:

* ``svd_matrix``: W = U diag(sigma) V^T with U (n x m) and V (m x m) the
  orthonormal factors of seeded N(0,1) matrices and sigma log-spaced from 1
  down to 1/cond (the test matrices of the QR workloads).
* ``ex1_matrix``: the parametric test matrix of the paper's first experiment,
  W_ij = sin(10(mu_j + x_i)) / (cos(100(mu_j - x_i)) + 1.1) on equispaced grids
  x_i = i/(n-1), mu_j = j/(m-1) (0-based), numerically rank-deficient.
* ``gaussian``: seeded N(0,1) blocks.
* ``batch_specs`` / ``near_duplicate_matrix_torch``: the many-small-problems
  workload.  Per problem n ~ U[2e4, 2e5] and m in {64, 128, 192, 256}, m_p in
  {16, 32}, drawn from numpy's Philox generator with seed 3; the columns are
  N(0,1), and every 8th column j (j = 8, 16, ...) is replaced by column
  j - 1 - (r mod j), r a seeded integer, plus Gaussian noise of relative size
  1e-7 (a numerically rank-deficient matrix in FP32).
* ``gaussian_random_field``: the log-coefficient g of the random diffusion
  problems, a ~ exp(g): a stationary Gaussian field on the (N+2) x (N+2) grid
  nodes of the unit square (spacing h = 1/(N+1)), zero mean, variance ``var``,
  squared-exponential covariance var * exp(-|x - y|^2 / (2 corr^2)), drawn by
  the spectral method on a periodic grid of twice the size (so the wrap-around
  does not correlate opposite sides) from numpy's PCG64 with the given seed.
* ``unet_params``: He-normal initial weights and zero biases of the small
  U-Net preconditioner (3 x 3 kernels; the layer widths c, c, 2c, 2c, c, 1).

CPU draws use numpy's PCG64; device draws (large sizes) use torch's generator
on the given device, so the two do not produce the same numbers: a test that
needs both sides on the same input copies one array to the other side.
"""
from __future__ import annotations

import numpy as np


def sigmas(m: int, cond: float) -> np.ndarray:
    """m singular values log-spaced from 1 down to 1/cond."""
    if m == 1:
        return np.ones(1)
    return np.logspace(0.0, -np.log10(cond), m)


def svd_matrix(n: int, m: int, cond: float, seed: int, dtype=np.float64) -> np.ndarray:
    """W = U diag(sigma) V^T (n x m, Fortran order) built on the CPU in FP64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    G = rng.standard_normal((n, m))
    U, _ = np.linalg.qr(G)
    H = rng.standard_normal((m, m))
    V, _ = np.linalg.qr(H)
    W = (U * sigmas(m, cond)) @ V.T
    return np.asfortranarray(W.astype(dtype))


def _orthonormal_cols_torch(G):
    """Orthonormal basis of the columns of the FP64 device matrix G (n x m,
    well conditioned): two Cholesky-QR rounds, Gram products on the device and
    the m x m Cholesky factor on the host, which in exact arithmetic is the Q
    factor of G with positive-diagonal R (the Householder-QR factor)."""
    import torch

    for _ in range(2):
        C = (G.t() @ G).cpu().numpy()
        L = np.linalg.cholesky(C)
        Rinv = np.linalg.inv(L.T)
        G = G @ torch.from_numpy(Rinv).to(G.device)
    return G


def svd_matrix_torch(n: int, m: int, cond: float, seed: int, device="cuda", dtype=None):
    """Same recipe drawn with torch on ``device`` (for sizes too large for the
    host).  Returns a column-major (n x m) tensor: shape (n, m), strides (1, n)."""
    import torch

    dtype = dtype or torch.float32
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    G = torch.randn((m, n), generator=g, device=device, dtype=torch.float64).t()  # column-major n x m
    U = _orthonormal_cols_torch(G)
    del G
    H = torch.randn((m, m), generator=g, device=device, dtype=torch.float64)
    V = torch.from_numpy(np.linalg.qr(H.cpu().numpy())[0]).to(device)
    s = torch.as_tensor(sigmas(m, cond), device=device, dtype=torch.float64)
    Wt = (V * s) @ U.t()  # (m x n) row-major == W column-major
    del U
    out = Wt.to(dtype).contiguous()
    del Wt
    return out.t()


def ex1_matrix(n: int, m: int, dtype=np.float64) -> np.ndarray:
    x = np.linspace(0.0, 1.0, n)[:, None]
    mu = np.linspace(0.0, 1.0, m)[None, :]
    W = np.sin(10.0 * (mu + x)) / (np.cos(100.0 * (mu - x)) + 1.1)
    return np.asfortranarray(W.astype(dtype))


def gaussian(n: int, m: int, seed: int, dtype=np.float64) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.asfortranarray(rng.standard_normal((n, m)).astype(dtype))


def batch_specs(count: int, seed: int = 3) -> list:
    """(n, m, m_p) of each problem of the many-small-problems workload."""
    rng = np.random.Generator(np.random.Philox(seed))
    out = []
    for _ in range(count):
        n = int(rng.integers(20000, 200001))
        m = int(rng.choice([64, 128, 192, 256]))
        mp = int(rng.choice([16, 32]))
        out.append((n, m, mp))
    return out


def near_duplicate_matrix_torch(n: int, m: int, seed: int, device="cuda", dtype=None):
    """n x m column-major device matrix (leading dimension a multiple of 4):
    N(0,1) columns, every 8th column j a copy of column j - 1 - (r mod j) plus
    noise of relative size 1e-7."""
    import torch

    dtype = dtype or torch.float32
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    rng = np.random.Generator(np.random.Philox(seed))
    ld = (n + 3) // 4 * 4
    W = torch.randn((m, ld), device=device, generator=g, dtype=dtype).t()[:n]
    for j in range(8, m, 8):
        src = j - 1 - int(rng.integers(0, 1 << 30)) % j
        scale = float(torch.linalg.norm(W[:, src])) / n ** 0.5
        W[:, j] = W[:, src] + 1e-7 * scale * torch.randn(n, device=device, generator=g, dtype=dtype)
    return W


def gaussian_random_field(N: int, seed: int, corr: float = 0.05, var: float = 1.0) -> np.ndarray:
    """(N+2) x (N+2) node values of a zero-mean stationary Gaussian field with
    covariance var * exp(-r^2 / (2 corr^2)) on the unit square."""
    h = 1.0 / (N + 1)
    M = 2 * (N + 2)
    f = np.fft.fftfreq(M, d=h)  # cycles per unit length
    kx, ky = np.meshgrid(f, f, indexing="ij")
    # spectral density of the squared-exponential covariance (2-D Fourier transform)
    dens = var * 2.0 * np.pi * corr ** 2 * np.exp(-2.0 * np.pi ** 2 * corr ** 2 * (kx ** 2 + ky ** 2))
    rng = np.random.Generator(np.random.PCG64(seed))
    xi = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    L = M * h  # period of the embedding grid
    g = np.fft.ifft2(xi * np.sqrt(dens / L ** 2)) * M * M
    return np.ascontiguousarray(g.real[: N + 2, : N + 2])


def unet_params(c: int, seed: int) -> dict:
    """Initial weights of the U-Net preconditioner: w (C_out, C_in, 3, 3) He
    normal (std sqrt(2 / (9 C_in))), b zero.  Layers: e1 1->c, e2 c->c, m1
    c->2c, m2 2c->2c, o1 3c->c, o2 c->1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shapes = {"e1": (c, 1), "e2": (c, c), "m1": (2 * c, c), "m2": (2 * c, 2 * c), "o1": (c, 3 * c), "o2": (1, c)}
    out = {}
    for name, (co, ci) in shapes.items():
        out[name + ".w"] = rng.standard_normal((co, ci, 3, 3)) * np.sqrt(2.0 / (9 * ci))
        out[name + ".b"] = np.zeros(co)
    return out

