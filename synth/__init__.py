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
  U-Net preconditioner (3 x 3 kernels; the layer widths c, c, 2c, 2c, c, 1);
  ``unet_params_levels`` the same for the L-level network of widths
  c_0 .. c_{L-1}.

* ``hadamard_svd_matrix`` / ``hadamard_svd_matrix_torch``: the full-size
  mixed-precision workload, W = 2^-s (Omega diag(sigma) H_L)[:, :m] with
  Omega (n x L) random signs, sigma L FP32 values log-spaced from 1 to
  1/cond, H_L the Sylvester-Hadamard matrix of order L = 2^ceil(log2 m) and
  2^-s a power of two that brings the largest singular value near 1.  Omega
  / sqrt(n) is orthonormal up to sqrt(L/n) and H_L / sqrt(L) is orthogonal,
  so this is the U diag(sigma) V^T recipe with cond(W) about cond.  Every
  partial sum of the product is an integer multiple of the smallest sigma's
  ulp below 2^53, so the FP64 product is exact in any summation order: the
  CPU and the device build the same W bit for bit, and the oracle can be
  run on exactly the matrix the device factors.

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


def gaussian_random_field_torch(N: int, seed: int, corr: float = 0.05, var: float = 1.0, device="cuda"):
    """gaussian_random_field drawn with torch on ``device`` (same spectral
    recipe, torch's generator: not the same numbers as the CPU version).
    Returns an (N+2) x (N+2) float64 tensor indexed [i, j], i along x."""
    import torch

    h = 1.0 / (N + 1)
    M = 2 * (N + 2)
    f = torch.fft.fftfreq(M, d=h, dtype=torch.float64, device=device)
    kx, ky = torch.meshgrid(f, f, indexing="ij")
    dens = var * 2.0 * np.pi * corr ** 2 * torch.exp(-2.0 * np.pi ** 2 * corr ** 2 * (kx ** 2 + ky ** 2))
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    xi = torch.complex(torch.randn((M, M), generator=g, device=device, dtype=torch.float64),
                       torch.randn((M, M), generator=g, device=device, dtype=torch.float64))
    L = M * h
    out = torch.fft.ifft2(xi * torch.sqrt(dens / L ** 2)) * M * M
    return out.real[: N + 2, : N + 2].contiguous()


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


def unet_params_levels(widths, seed: int) -> dict:
    """Initial weights of the L-level U-Net (layer list of
    oracle.learned.unet_layers, written out here): w (C_out, C_in, 3, 3) He
    normal, std sqrt(2 / (9 C_in)), b zero."""
    L = len(widths)
    shapes = []
    for l in range(L):
        shapes.append((f"enc{l}a", widths[l], 1 if l == 0 else widths[l - 1]))
        shapes.append((f"enc{l}b", widths[l], widths[l]))
    for l in range(L - 2, -1, -1):
        shapes.append((f"dec{l}", widths[l], widths[l + 1] + widths[l]))
    shapes.append(("out", 1, widths[0]))
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {}
    for name, co, ci in shapes:
        out[name + ".w"] = rng.standard_normal((co, ci, 3, 3)) * np.sqrt(2.0 / (9 * ci))
        out[name + ".b"] = np.zeros(co)
    return out


def unet_flat_params(params: dict, widths) -> np.ndarray:
    """The dict of unet_params_levels in the library's parameter layout: layer
    after layer (enc0a, enc0b, ..., enc{L-1}b, dec{L-2}, ..., dec0, out),
    w[o, c, s, t] stored as w[3 s + t][c][o], then b[o]; float32."""
    L = len(widths)
    names = [f"enc{l}{h}" for l in range(L) for h in "ab"] + [f"dec{l}" for l in range(L - 2, -1, -1)] + ["out"]
    parts = []
    for nm in names:
        w = params[nm + ".w"]
        co, ci = w.shape[:2]
        parts.append(np.transpose(w, (2, 3, 1, 0)).reshape(9 * ci * co))
        parts.append(params[nm + ".b"])
    return np.concatenate(parts).astype(np.float32)


def unet_dict_params(flat, widths) -> dict:
    """The inverse of unet_flat_params (float64 arrays)."""
    flat = np.asarray(flat, dtype=np.float64)
    L = len(widths)
    shapes = []
    for l in range(L):
        shapes.append((f"enc{l}a", widths[l], 1 if l == 0 else widths[l - 1]))
        shapes.append((f"enc{l}b", widths[l], widths[l]))
    for l in range(L - 2, -1, -1):
        shapes.append((f"dec{l}", widths[l], widths[l + 1] + widths[l]))
    shapes.append(("out", 1, widths[0]))
    out, off = {}, 0
    for nm, co, ci in shapes:
        w = flat[off:off + 9 * ci * co].reshape(3, 3, ci, co)
        out[nm + ".w"] = np.ascontiguousarray(np.transpose(w, (3, 2, 0, 1)))
        off += 9 * ci * co
        out[nm + ".b"] = flat[off:off + co].copy()
        off += co
    assert off == flat.size
    return out


def _hadamard_cols(L: int, m: int) -> np.ndarray:
    """The first m columns of the unnormalised Sylvester-Hadamard matrix of
    order L (entries (-1)^popcount(l & j))."""
    l = np.arange(L)[:, None]
    j = np.arange(m)[None, :]
    v = l & j
    par = np.zeros_like(v)
    while np.any(v):
        par ^= v & 1
        v >>= 1
    return 1.0 - 2.0 * par


def _hadamard_plan(n: int, m: int, cond: float):
    L = 1 << max(0, (m - 1).bit_length())
    sig = np.logspace(0.0, -np.log10(cond), L).astype(np.float32).astype(np.float64)
    # exactness: all sigma are multiples of the smallest one's FP32 ulp, and
    # sum(sigma) / ulp must stay below 2^53 (then every partial sum is exact)
    ulp = 2.0 ** (np.floor(np.log2(sig.min())) - 23)
    assert sig.sum() / ulp < 2.0 ** 53, "the product would not be exact in FP64"
    s = int(np.ceil(np.log2(np.sqrt(float(n) * L))))
    return L, sig, 2.0 ** (-s)


def _sign_words(n: int, L: int, seed: int) -> np.ndarray:
    """n L sign bits from numpy's Philox generator (platform independent),
    64 per word: bit (i L + l) gives Omega[i, l] = -1 where set."""
    bg = np.random.Philox(seed)
    return bg.random_raw((n * L + 63) // 64).astype(np.uint64)


def _signs_rows(words: np.ndarray, r0: int, r1: int, L: int) -> np.ndarray:
    """Omega[r0:r1] as a float64 array of +-1 (L a multiple of 64 or the rows
    packed contiguously)."""
    b0, b1 = r0 * L, r1 * L
    w0, w1 = b0 // 64, (b1 + 63) // 64
    bits = np.unpackbits(words[w0:w1].view(np.uint8), bitorder="little")[b0 - 64 * w0: b1 - 64 * w0]
    return 1.0 - 2.0 * bits.reshape(r1 - r0, L).astype(np.float64)


def hadamard_svd_matrix(n: int, m: int, cond: float, seed: int, chunk: int = 65536) -> np.ndarray:
    """n x m FP32 matrix (Fortran order) of the exact recipe, on the CPU."""
    L, sig, scale = _hadamard_plan(n, m, cond)
    Hs = _hadamard_cols(L, m) * (sig * scale)[:, None]  # diag(sigma) H 2^-s: exact (powers of two, +-1)
    words = _sign_words(n, L, seed)
    W = np.empty((n, m), dtype=np.float32, order="F")
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        W[r0:r1] = (_signs_rows(words, r0, r1, L) @ Hs).astype(np.float32)
    return W


def hadamard_svd_matrix_torch(n: int, m: int, cond: float, seed: int, device="cuda", dtype=None,
                              chunk: int = 131072):
    """The same matrix built on ``device`` (the signs are unpacked on the CPU,
    the exact FP64 product runs on the device); column-major (n x m) with a
    leading dimension of n.  dtype float32 (default) or float64 (the FP32
    values widened)."""
    import torch

    dtype = dtype or torch.float32
    L, sig, scale = _hadamard_plan(n, m, cond)
    Hs = torch.from_numpy(_hadamard_cols(L, m) * (sig * scale)[:, None]).to(device)
    words = _sign_words(n, L, seed)
    Wt = torch.empty((m, n), dtype=dtype, device=device)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        Om = torch.from_numpy(_signs_rows(words, r0, r1, L)).to(device)
        Wt[:, r0:r1] = (Om @ Hs).to(torch.float32).to(dtype).t()
        del Om
    return Wt.t()


def bit_checksum(W32) -> int:
    """Sum of the FP32 bit patterns of W as signed 32-bit integers (an exact
    fingerprint that the CPU and the device compute alike)."""
    a = np.asarray(W32, dtype=np.float32)
    return int(a.view(np.int32).astype(np.int64).sum())

