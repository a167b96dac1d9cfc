"""Plain FP64 CPU oracle for randomized block Gram-Schmidt (RBGS).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never links or calls it, and the two share no code:
the C source here is compiled on its own with gcc.

What each function follows (Balabanov & Grigori, arXiv 2111.14641):

* ``theta_*`` / ``srht_samples`` / ``philox``: the sketching matrices of
  Sec. 2.3 (Rademacher, SRHT with zero padding) plus the Gaussian N(0, 1/k)
  sketch, drawn from a Philox4x32-10 counter generator whose bit-level
  layout is a project convention (the paper asks only for a seeded
  generator).  Each side implements that convention separately.
* ``rbgs``: Alg. 2 with steps 4-5 from Alg. 4, 5 or 6 and step-2 solvers
  from Sec. 3.1 and its supplement (Householder, Richardson, CG).
* ``cholqr_postprocess``: the Cholesky QR post-processing of the remark
  after Alg. 2 (an l2-orthonormal Q).
* ``embedding_check``: the a posteriori check of Theta with an independent
  sketch Phi (Sec. 4, the epsilon-embedding subsection).
* ``rcholqr``: the closed form that RBGS reaches in exact arithmetic
  (R = R factor of Theta W with a positive diagonal, Q = W R^{-1}).
* ``householder_qr``: textbook Householder QR with a positive diagonal.
* ``rbgs_arnoldi`` / ``block_krylov`` / ``rayleigh_ritz``: Alg. 7, the
  restarted randomized block GMRES and FOM of Sec. 5.2-5.3, and Alg. 8
  (Sec. 5.4) on the 5-point convection-diffusion stencil.

Every array is float64, column-major (Fortran order).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "rbgs_oracle.c"
_BUILD = _HERE / "_build"
_LIB = _BUILD / "liborbgs.so"

THETA = {"gauss": 0, "rademacher": 1, "srht": 2, "identity": 3, "sparse": 4}
LS = {"householder": 0, "richardson": 1, "cg": 2}

_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (plain C99, -ffp-contract=off so the x86 and
    Arm builds round identically)."""
    _BUILD.mkdir(exist_ok=True)
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB.with_suffix(f".{os.getpid()}.tmp")
        cmd = ["gcc", "-O2", "-std=gnu99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-pthread", "-o", str(tmp), str(_SRC), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(str(_LIB))
        i64, u64, dp = ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
        lib.or_philox4x32_10.argtypes = [dp, dp, dp]
        lib.or_theta_dense.argtypes = [ctypes.c_int, i64, i64, u64, dp]
        lib.or_theta_dense.restype = ctypes.c_int
        lib.or_theta_apply.argtypes = [ctypes.c_int, i64, i64, u64, dp, i64, i64, dp, i64]
        lib.or_theta_apply.restype = ctypes.c_int
        lib.or_theta_gauss_entry.argtypes = [u64, i64, i64, i64]
        lib.or_theta_gauss_entry.restype = ctypes.c_double
        lib.or_srht_samples.argtypes = [u64, i64, i64, dp]
        lib.or_srht_samples.restype = ctypes.c_int
        lib.or_srht_sign.argtypes = [u64, i64]
        lib.or_srht_sign.restype = ctypes.c_double
        lib.or_srht_padded.argtypes = [i64]
        lib.or_srht_padded.restype = i64
        lib.or_fwht.argtypes = [dp, i64]
        lib.or_sparse_column.argtypes = [u64, i64, i64, dp, dp]
        lib.or_sparse_column.restype = ctypes.c_int
        lib.or_householder_qr.argtypes = [i64, i64, dp, i64, dp]
        lib.or_qr_r.argtypes = [i64, i64, dp, i64, dp, i64]
        lib.or_qr_r.restype = ctypes.c_int
        lib.or_qr_full.argtypes = [i64, i64, dp, i64, dp, i64, dp, i64]
        lib.or_qr_full.restype = ctypes.c_int
        lib.or_rbgs.argtypes = [dp, i64, i64, i64, i64, ctypes.c_int, i64, u64, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, i64, dp, i64, dp, dp, dp]
        lib.or_rbgs.restype = ctypes.c_int
        lib.or_rcholqr.argtypes = [dp, i64, i64, i64, ctypes.c_int, i64, u64, dp, i64, dp, i64]
        lib.or_rcholqr.restype = ctypes.c_int
        lib.or_ls_solve.argtypes = [ctypes.c_int, ctypes.c_int, i64, i64, dp, i64, dp, i64, i64, dp, i64]
        lib.or_ls_solve.restype = ctypes.c_int
        dd = ctypes.c_double
        lib.or_stencil5_apply.argtypes = [ctypes.c_void_p, dp, i64, i64, dp, i64]
        lib.or_stencil5_apply.restype = None
        lib.or_rbgs_arnoldi.argtypes = [i64, i64, dd, dd, dp, i64, i64, i64, ctypes.c_int, i64, ctypes.c_uint64,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, i64,
                                        dp, i64, dp]
        lib.or_rbgs_arnoldi.restype = ctypes.c_int
        lib.or_block_krylov.argtypes = [ctypes.c_int, i64, i64, dd, dd, dp, i64, dp, i64, i64, i64, ctypes.c_int, i64,
                                        ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, dd, i64, dp]
        lib.or_block_krylov.restype = ctypes.c_int
        lib.or_set_threads.argtypes = [ctypes.c_int]
        lib.or_get_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> None:
    """Worker threads for the tall loops (rows of step 3, columns of Theta X)."""
    _load().or_set_threads(int(n))


def get_threads() -> int:
    return int(_load().or_get_threads())


def philox(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block: four uint32 counter words, two key words."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.zeros(4, dtype=np.uint32)
    _load().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def srht_padded(n: int) -> int:
    return int(_load().or_srht_padded(int(n)))


def srht_samples(seed: int, n: int, k: int) -> np.ndarray:
    """Sorted sampled rows s_0 < ... < s_{k-1} of the n' x n' Hadamard matrix."""
    out = np.zeros(k, dtype=np.int64)
    if _load().or_srht_samples(int(seed), srht_padded(n), int(k), _ptr(out)):
        raise ValueError("k exceeds the padded dimension")
    return out


def srht_signs(seed: int, n: int) -> np.ndarray:
    lib = _load()
    return np.array([lib.or_srht_sign(int(seed), j) for j in range(int(n))])


def sparse_columns(seed: int, k: int, j0: int, count: int):
    """Rows (count x z, int64) and signs (count x z, +-1.0) of the nonzeros of
    columns j0 .. j0 + count - 1 of the sparse-sign Theta, z = min(8, k)."""
    lib = _load()
    z = min(8, int(k))
    rows = np.zeros((count, z), dtype=np.int64)
    signs = np.zeros((count, z), dtype=np.float64)
    r8 = np.zeros(8, dtype=np.int64)
    s8 = np.zeros(8, dtype=np.float64)
    for t in range(count):
        lib.or_sparse_column(int(seed), int(k), int(j0) + t, _ptr(r8), _ptr(s8))
        rows[t], signs[t] = r8[:z], s8[:z]
    return rows, signs


def theta_dense(kind: str, k: int, n: int, seed: int) -> np.ndarray:
    """Theta (k x n) from the entry definitions, for small cases."""
    T = np.zeros((k, n), dtype=np.float64, order="F")
    if _load().or_theta_dense(THETA[kind], int(k), int(n), int(seed), _ptr(T)):
        raise ValueError("bad sketch arguments")
    return T


def theta_gauss_entries(k: int, seed: int, r, j) -> np.ndarray:
    """Entries Theta(r[t], j[t]) of the Gaussian Theta, one C call each (for
    columns beyond what theta_dense can hold)."""
    lib = _load()
    r = np.asarray(r, dtype=np.int64).ravel()
    j = np.asarray(j, dtype=np.int64).ravel()
    return np.array([lib.or_theta_gauss_entry(int(seed), int(k), int(a), int(b)) for a, b in zip(r, j)])


def theta_apply(kind: str, k: int, seed: int, X) -> np.ndarray:
    """Theta X for X (n x c); SRHT goes through the Hadamard transform."""
    X = _f64(X)
    if X.ndim == 1:
        X = X.reshape(-1, 1, order="F")
    n, c = X.shape
    Y = np.zeros((k, c), dtype=np.float64, order="F")
    if _load().or_theta_apply(THETA[kind], int(k), int(n), int(seed), _ptr(X), max(n, 1), int(c), _ptr(Y), max(k, 1)):
        raise ValueError("bad sketch arguments")
    return Y


def fwht(x) -> np.ndarray:
    """Sylvester-ordered Walsh-Hadamard transform (unnormalised) of a vector of length 2^q."""
    y = np.ascontiguousarray(np.asarray(x, dtype=np.float64).copy())
    _load().or_fwht(_ptr(y), y.size)
    return y


def householder_qr(A):
    """Thin Householder QR with a positive diagonal: returns (Q, R)."""
    A = _f64(A)
    m, n = A.shape
    Q = np.zeros((m, n), order="F")
    R = np.zeros((n, n), order="F")
    rc = _load().or_qr_full(m, n, _ptr(A), m, _ptr(Q), m, _ptr(R), n)
    return Q, R, rc


def rbgs(W, mp: int, kind: str, k: int, seed: int, variant: int = 5, ls: str = "householder",
         ls_iters: int = 5, reorth: bool = False, ls_iters_first: int = 0):
    """Alg. 2.  Returns dict(Q, R, S, P, delta, delta_tilde, passes2, rc).
    With reorth, ls_iters_first > 0 sets the iterations of the first pass."""
    W = _f64(W)
    n, m = W.shape
    Q = np.zeros((n, m), order="F")
    R = np.zeros((m, m), order="F")
    S = np.zeros((k, m), order="F")
    P = np.zeros((k, m), order="F")
    st = np.zeros(3)
    rc = _load().or_rbgs(_ptr(W), n, m, n, int(mp), THETA[kind], int(k), int(seed), int(variant), LS[ls],
                         int(ls_iters), int(ls_iters_first), int(bool(reorth)), _ptr(Q), n, _ptr(R), m, _ptr(S),
                         _ptr(P), _ptr(st))
    if rc == -1:
        raise ValueError("bad RBGS arguments")
    return dict(Q=Q, R=R, S=S, P=P, delta=st[0], delta_tilde=st[1], passes2=int(st[2]), rc=rc)


def ls_solve(S, P, method: str = "householder", iters: int = 5) -> np.ndarray:
    """Step-2 solution X = argmin ||S X - P||_F by the chosen method."""
    S = _f64(S)
    P = _f64(P)
    k, c = S.shape
    mp = P.shape[1]
    X = np.zeros((c, mp), order="F")
    rc = _load().or_ls_solve(LS[method], int(iters), k, c, _ptr(S), k, _ptr(P), k, mp, _ptr(X), c)
    if rc:
        raise np.linalg.LinAlgError("singular least-squares matrix")
    return X


def rcholqr(W, kind: str, k: int, seed: int):
    """Closed form: R = R(Theta W), Q = W R^{-1}.  Returns (Q, R, rc)."""
    W = _f64(W)
    n, m = W.shape
    Q = np.zeros((n, m), order="F")
    R = np.zeros((m, m), order="F")
    rc = _load().or_rcholqr(_ptr(W), n, m, n, THETA[kind], int(k), int(seed), _ptr(Q), n, _ptr(R), m)
    if rc == -1:
        raise ValueError("bad arguments")
    return Q, R, rc


# ---- Sec. 5: the stencil operator, Alg. 7 (RBGS-Arnoldi), block GMRES / FOM ----

class _Stencil(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("bx", ctypes.c_double), ("by", ctypes.c_double)]


def stencil5_apply(nx: int, ny: int, bx: float, by: float, X) -> np.ndarray:
    """Y = A X for the 5-point convection-diffusion operator (-Laplace + b . grad,
    nx x ny interior points of the unit square, zero Dirichlet boundary)."""
    X = _f64(X)
    if X.ndim == 1:
        X = X.reshape(-1, 1, order="F")
    n, c = X.shape
    Y = np.zeros((n, c), order="F")
    op = _Stencil(nx, ny, bx, by)
    _load().or_stencil5_apply(ctypes.byref(op), _ptr(X), n, c, _ptr(Y), n)
    return Y


def rbgs_arnoldi(nx: int, ny: int, bx: float, by: float, B, p: int, kind: str, k: int, seed: int, variant: int = 5,
                 ls: str = "householder", ls_iters: int = 5, reorth: bool = False, ls_iters_first: int = 0):
    """Alg. 7: Q (n x p mp), R (p mp x p mp); H = R[:, mp:].  Returns dict(Q, R, delta, delta_tilde, rc)."""
    B = _f64(B)
    n, mp = B.shape
    m = p * mp
    Q = np.zeros((n, m), order="F")
    R = np.zeros((m, m), order="F")
    st = np.zeros(3)
    rc = _load().or_rbgs_arnoldi(nx, ny, bx, by, _ptr(B), n, mp, p, THETA[kind], int(k), int(seed), int(variant),
                                 LS[ls], int(ls_iters), int(ls_iters_first), int(bool(reorth)), _ptr(Q), n, _ptr(R),
                                 m, _ptr(st))
    if rc == -1:
        raise ValueError("bad Arnoldi arguments")
    return dict(Q=Q, R=R, delta=st[0], delta_tilde=st[1], rc=rc)


def block_krylov(method: str, nx: int, ny: int, bx: float, by: float, B, X0, p: int, kind: str, k: int, seed: int,
                 rtol: float, max_cycles: int, variant: int = 5, ls: str = "householder", ls_iters: int = 5,
                 reorth: bool = False, ls_iters_first: int = 0):
    """Restarted randomized block GMRES (method "gmres") or FOM ("fom") with p
    Arnoldi blocks per cycle.  Returns (X, cycles, relres)."""
    B = _f64(B)
    X = np.array(_f64(X0), order="F", copy=True)
    n, mp = B.shape
    relres = np.zeros(mp)
    cyc = _load().or_block_krylov({"gmres": 0, "fom": 1}[method], nx, ny, bx, by, _ptr(B), n, _ptr(X), n, mp, p,
                                  THETA[kind], int(k), int(seed), int(variant), LS[ls], int(ls_iters),
                                  int(ls_iters_first), int(bool(reorth)), float(rtol), int(max_cycles), _ptr(relres))
    if cyc < 0:
        raise np.linalg.LinAlgError(f"block Krylov solver failed ({cyc})")
    return X, int(cyc), relres


def cholqr_postprocess(Q, R):
    """The Cholesky QR post-processing of the remark after Alg. 2: R' the
    upper Cholesky factor of Q^T Q, Q <- Q R'^{-1}, R <- R' R (numpy's
    Cholesky and triangular solve as the library steps).  Returns (Q, R)."""
    Q = _f64(Q)
    R = _f64(R)
    Rp = np.linalg.cholesky(Q.T @ Q).T
    Qn = np.linalg.solve(Rp.T, Q.T).T
    return np.asfortranarray(Qn), np.asfortranarray(Rp @ R)


def embedding_check(Z, mp: int, kind: str, k: int, seed_theta: int, seed_phi: int, variant: int = 5,
                    ls: str = "householder", ls_iters: int = 5, reorth: bool = False, ls_iters_first: int = 0):
    """The a posteriori check of the epsilon-embedding property (Sec. 4, the
    epsilon-embedding subsection): with an independent sketch Phi, Y = the
    inverse of the R factor of Phi Z, and (Theta Z) Y should have orthonormal
    columns when Theta embeds range(Z) well.  Y is obtained from RBGS with the
    sketch Phi (Q_phi = Z R_phi^{-1}, R_phi the R factor of Phi Z), so that
    (Theta Z) Y = Theta Q_phi.  Returns ||I - (Theta Q_phi)^T (Theta Q_phi)||_F."""
    out = rbgs(Z, mp, kind, k, seed_phi, variant=variant, ls=ls, ls_iters=ls_iters, reorth=reorth,
               ls_iters_first=ls_iters_first)
    if out["rc"] != 0:
        raise np.linalg.LinAlgError(f"RBGS breakdown ({out['rc']})")
    S = theta_apply(kind, k, seed_theta, out["Q"])
    return float(np.linalg.norm(np.eye(S.shape[1]) - S.T @ S, "fro"))


RITZ_WHICH = ("LR", "SR")


def ritz_select(mu, V, mp: int, which: str):
    """Step 2 of Alg. 8: the m_p extreme Ritz pairs of the projected matrix, as
    a real basis.  The paper leaves the selection and the scaling open; the
    conventions (shared with the GPU path, written separately there) are:

    * order: by real part, descending for "LR" and ascending for "SR"; among
      equal real parts the eigenvalue with positive imaginary part comes first,
      and each conjugate pair is considered once;
    * each eigenvector y is scaled to unit 2-norm with its largest-modulus entry
      (the first one, on ties) real and positive;
    * a real eigenvalue takes one column y, a conjugate pair a +- ib two
      columns Re y and Im y (only Re y if one slot is left).

    Returns (values (complex, per column), Y (N x mp, real), vecs (the complex
    unit eigenvector of each column's value: y, and conj(y) for the second
    column of a pair))."""
    mu = np.asarray(mu)
    cand = [i for i in range(mu.size) if mu[i].imag >= 0.0]
    if which == "LR":
        cand.sort(key=lambda i: (-mu[i].real, -mu[i].imag))
    elif which == "SR":
        cand.sort(key=lambda i: (mu[i].real, -mu[i].imag))
    else:
        raise ValueError("which must be 'LR' or 'SR'")
    N = V.shape[0]
    Y = np.zeros((N, mp), order="F")
    vals, vecs = [], []
    col = 0
    for i in cand:
        if col >= mp:
            break
        y = V[:, i].astype(np.complex128)
        y = y / np.linalg.norm(y)
        j = int(np.argmax(np.abs(y)))
        y = y * (np.conj(y[j]) / abs(y[j]))
        Y[:, col] = y.real
        vals.append(mu[i])
        vecs.append(y)
        col += 1
        if mu[i].imag > 0.0 and col < mp:
            Y[:, col] = y.imag
            vals.append(np.conj(mu[i]))
            vecs.append(np.conj(y))
            col += 1
    return np.array(vals), Y, vecs


def rayleigh_ritz(nx: int, ny: int, bx: float, by: float, B0, p: int, n_iter: int, which: str, kind: str, k: int,
                  seed: int, variant: int = 5, ls: str = "householder", ls_iters: int = 5, reorth: bool = False,
                  ls_iters_first: int = 0):
    """Alg. 8 (Sec. 5.4): randomized Rayleigh-Ritz with restarting.  Each
    iteration runs Alg. 7 from B, sets H = R_(1:p,2:p), takes the m_p extreme
    eigenpairs (mu, y) of H_(1:p-1,1:p-1) (numpy's eig as the library step;
    selection and scaling per ``ritz_select``), estimates each residual by
    ||H_(p,1:p-1) y|| and restarts from B = Q_(1:p-1) Y.  Step 5 scales the
    columns of the last B to unit 2-norm.

    Returns dict(values (complex, m_p), X (n x m_p), resid (m_p), Q, R of the
    last iteration)."""
    B = _f64(B0)
    n, mp = B.shape
    N = (p - 1) * mp
    out = None
    for _ in range(n_iter):
        out = rbgs_arnoldi(nx, ny, bx, by, B, p, kind, k, seed, variant=variant, ls=ls, ls_iters=ls_iters,
                           reorth=reorth, ls_iters_first=ls_iters_first)
        if out["rc"] != 0:
            raise np.linalg.LinAlgError(f"Arnoldi breakdown ({out['rc']})")
        H = out["R"][:, mp:]
        mu, V = np.linalg.eig(H[:N, :N])
        vals, Y, vecs = ritz_select(mu, V, mp, which)
        resid = np.array([np.linalg.norm(H[N:, :N] @ y) for y in vecs])
        B = np.asfortranarray(out["Q"][:, :N] @ Y)
    X = np.asfortranarray(B / np.linalg.norm(B, axis=0))
    return dict(values=vals, X=X, resid=resid, Q=out["Q"], R=out["R"])


def stencil5_dense(nx: int, ny: int, bx: float, by: float) -> np.ndarray:
    """The operator as a dense matrix, column by column through stencil5_apply."""
    n = nx * ny
    return stencil5_apply(nx, ny, bx, by, np.eye(n))


# ---- quality measures, computed in FP64 with the oracle's own Theta ----------

def sketched_orthogonality(Q, kind: str, k: int, seed: int):
    """(||I - (Theta Q)^T (Theta Q)||_F, same in the 2-norm)."""
    S = theta_apply(kind, k, seed, Q)
    E = np.eye(S.shape[1]) - S.T @ S
    return float(np.linalg.norm(E, "fro")), float(np.linalg.norm(E, 2))


def factorization_error(W, Q, R) -> float:
    """||W - Q R||_F / ||W||_F."""
    W = np.asarray(W, dtype=np.float64)
    return float(np.linalg.norm(W - np.asarray(Q, np.float64) @ np.asarray(R, np.float64)) / np.linalg.norm(W))


def cond(Q) -> float:
    s = np.linalg.svd(np.asarray(Q, dtype=np.float64), compute_uv=False)
    return float(s[0] / s[-1])
