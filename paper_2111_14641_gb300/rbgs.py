"""Thin Python binding of librbgs (ctypes).  Argument marshalling only: every
step of the computation runs in the CUDA library; there is no fallback.

Tensors are torch CUDA tensors in column-major layout: shape (rows, cols) with
stride (1, ld), ld >= rows (``colmajor(t)`` converts).  Work is enqueued on the
current torch CUDA stream unless ``stream`` is given.
"""
from __future__ import annotations

import ctypes
import re
from dataclasses import dataclass
from pathlib import Path

import torch

from . import build as _build

_HDR = Path(__file__).resolve().parent.parent / "include" / "rbgs.h"

SKETCH = {"gauss": 0, "rademacher": 1, "srht": 2, "sparse": 3}
PREC = {"fp64": 0, "fp32": 1, "tf32x3": 2, "f16x3": 3}
# Largest c + mb that rbgs_tall_update_noalloc accepts (its fixed scratch).
NOALLOC_MAX_K = int(re.search(r"#define RBGS_NOALLOC_MAX_K (\d+)", _HDR.read_text()).group(1))
STATUS = {0: "RBGS_OK", 1: "RBGS_EINVAL", 2: "RBGS_ENOMEM", 3: "RBGS_ECUDA", 4: "RBGS_EBREAKDOWN",
          5: "RBGS_ENOTCERTIFIED", 6: "RBGS_ETIMEOUT", 7: "RBGS_ENOCONV", 8: "RBGS_ENODEV",
          9: "RBGS_ETOOLARGE"}


class RbgsError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int32), ("ls_iters", ctypes.c_int32), ("reorth", ctypes.c_int32),
                ("certify", ctypes.c_int32), ("reorth_tol", ctypes.c_double), ("stream", ctypes.c_void_p),
                ("sync", ctypes.c_int32), ("timing", ctypes.c_int32), ("fine", ctypes.c_int32),
                ("interblock", ctypes.c_int32), ("ls", ctypes.c_int32), ("trsm", ctypes.c_int32)]


LS = {"richardson": 0, "cg": 1, "householder": 2}


class Problem(ctypes.Structure):
    _fields_ = [("W", ctypes.c_void_p), ("n", ctypes.c_int64), ("m", ctypes.c_int64), ("ldw", ctypes.c_int64),
                ("mb", ctypes.c_int64), ("k", ctypes.c_int64), ("seed", ctypes.c_uint64), ("Q", ctypes.c_void_p),
                ("ldq", ctypes.c_int64), ("R", ctypes.c_void_p), ("ldr", ctypes.c_int64), ("status", ctypes.c_int32),
                ("passes2", ctypes.c_int32)]


class Op(ctypes.Structure):
    """rbgs_op: the 5-point convection-diffusion operator (kind 0) or
    -div(a grad) with face coefficients (kind 1) on nx x ny interior points."""
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("nx", ctypes.c_int64),
                ("ny", ctypes.c_int64), ("bx", ctypes.c_double), ("by", ctypes.c_double),
                ("coef", ctypes.c_void_p)]


class UNet(ctypes.Structure):
    """rbgs_unet: the levels and per-level widths of the U-Net preconditioner;
    flags bit 0 keeps every convolution on the SIMT kernels."""
    _fields_ = [("levels", ctypes.c_int32), ("width", ctypes.c_int32 * 6), ("flags", ctypes.c_int32)]


def unet_shape(widths, simt: bool = False) -> UNet:
    w = (ctypes.c_int32 * 6)(*([int(x) for x in widths] + [0] * (6 - len(widths))))
    return UNet(len(widths), w, 1 if simt else 0)


def stencil_op(nx: int, ny: int, bx: float, by: float) -> Op:
    return Op(0, 0, nx, ny, bx, by, None)


def diffusion_faces(a: torch.Tensor, stream=None) -> torch.Tensor:
    """Face coefficients (harmonic means) of -div(a grad) from the node values
    a, a float64 CUDA tensor of (nx+2) x (ny+2) nodes with node (i, j) at
    i + (nx+2) j (a[j, i] of a row-major (ny+2, nx+2) tensor)."""
    lib = load()
    if a.dtype != torch.float64 or not a.is_contiguous():
        raise ValueError("a must be a contiguous float64 tensor")
    ny, nx = a.shape[0] - 2, a.shape[1] - 2
    fc = torch.empty((nx + 1) * (ny + 2) + (nx + 2) * (ny + 1), dtype=torch.float64, device=a.device)
    _check(lib.rbgs_diffusion_faces(nx, ny, a.data_ptr(), fc.data_ptr(), _stream_ptr(stream), 1),
           "rbgs_diffusion_faces")
    return fc


def diffusion_op(nx: int, ny: int, coef: torch.Tensor) -> Op:
    """rbgs_op of -div(a grad u) with the face coefficients coef (kept alive
    by the caller for as long as the operator is used)."""
    return Op(1, 0, nx, ny, 0.0, 0.0, coef.data_ptr())


class Stats(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("delta_tilde", ctypes.c_double), ("passes2", ctypes.c_int32),
                ("certified", ctypes.c_int32), ("tall_ms", ctypes.c_double), ("tall_bytes", ctypes.c_double),
                ("tall_launches", ctypes.c_int32), ("chol_rounds2", ctypes.c_int32),
                ("host_up_ms", ctypes.c_double), ("host_compute_ms", ctypes.c_double),
                ("host_total_ms", ctypes.c_double)]


@dataclass
class QRStats:
    delta: float
    delta_tilde: float
    passes2: int
    certified: bool
    tall_ms: float = 0.0
    tall_bytes: float = 0.0
    tall_launches: int = 0
    chol_rounds2: int = 0
    host_up_ms: float = 0.0
    host_compute_ms: float = 0.0
    host_total_ms: float = 0.0


_lib = None


def lib_path() -> Path:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load librbgs.so; raises if it is missing (no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not path.exists():
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"librbgs.so not built ({path}); run paper_2111_14641_gb300.build.build()")
    lib = ctypes.CDLL(str(path))
    i64, u64, vp, i32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int32
    lib.rbgs_opts_default.argtypes = [ctypes.POINTER(Opts)]
    lib.rbgs_qr.argtypes = [vp, i64, i64, i64, i64, ctypes.c_int, i64, u64, vp, i64, vp, i64,
                            ctypes.POINTER(Opts), ctypes.POINTER(Stats)]
    lib.rbgs_sketch_apply.argtypes = [ctypes.c_int, i64, i64, u64, i32, vp, i64, i64, vp, i64, vp, i32]
    lib.rbgs_tall_update.argtypes = [i32, i64, i64, i64, vp, i64, vp, i64, vp, i64, vp, i64, vp, i32]
    lib.rbgs_tall_update_noalloc.argtypes = [i32, i64, i64, i64, vp, i64, vp, i64, vp, i64, vp, i64, vp, i32]
    lib.rbgs_philox.argtypes = [u64, vp, vp, i64, vp, i32]
    opp = ctypes.POINTER(Op)
    lib.rbgs_op_apply.argtypes = [opp, i32, vp, i64, i64, vp, i64, vp, i32]
    lib.rbgs_diffusion_faces.argtypes = [i64, i64, vp, vp, vp, i32]
    unp = ctypes.POINTER(UNet)
    lib.rbgs_unet_num_params.argtypes = [unp]
    lib.rbgs_unet_num_params.restype = i64
    lib.rbgs_unet_forward.argtypes = [unp, vp, i64, i64, vp, vp, i32, vp, i32]
    lib.rbgs_unet_backward.argtypes = [unp, vp, i64, i64, vp, vp, vp, vp, i32]
    lib.rbgs_unet_residual_loss.argtypes = [i64, i64, vp, i64, vp, vp, vp, vp, vp, vp, i32]
    lib.rbgs_adam_step.argtypes = [i64, vp, vp, vp, vp, i64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, vp, i32]
    lib.rbgs_unet_precondition.argtypes = [unp, vp, i64, i32, vp, i64, i64, vp, i64, vp, i32]
    lib.rbgs_unet_scale_inputs.argtypes = [i64, i64, i32, vp, i64, vp, i64, vp, i32]
    lib.rbgs_block_fgmres.argtypes = [opp, unp, vp, vp, i64, vp, i64, i64, i64, ctypes.c_double, i64,
                                      ctypes.c_double, ctypes.c_int, i64, u64, ctypes.POINTER(Opts),
                                      ctypes.POINTER(ctypes.c_int64), vp, ctypes.POINTER(ctypes.c_int64)]
    lib.rbgs_block_arnoldi.argtypes = [opp, vp, i64, i64, i64, ctypes.c_int, i64, u64, vp, i64, vp, i64,
                                       ctypes.POINTER(Opts), ctypes.POINTER(Stats)]
    for fn in ("rbgs_block_gmres", "rbgs_block_fom"):
        getattr(lib, fn).argtypes = [opp, vp, i64, vp, i64, i64, i64, ctypes.c_double, i64, ctypes.c_int, i64, u64,
                                     ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_int64), vp]
    lib.rbgs_rayleigh_ritz.argtypes = [opp, vp, i64, i64, i64, i64, i32, ctypes.c_int, i64, u64, ctypes.POINTER(Opts),
                                       vp, i64, vp, vp, vp]
    lib.rbgs_qr_batched.argtypes = [ctypes.POINTER(Problem), i64, ctypes.c_int, ctypes.POINTER(Opts), i32]
    lib.rbgs_embedding_check.argtypes = [vp, i64, i64, i64, i64, ctypes.c_int, i64, u64, u64, ctypes.POINTER(Opts),
                                         vp]
    lib.rbgs_cholqr_postprocess.argtypes = [i32, i64, i64, vp, i64, vp, i64, i64, vp, i32]
    lib.rbgs_qr_graph_create.argtypes = [vp, i64, i64, i64, i64, ctypes.c_int, i64, u64, vp, i64, vp, i64,
                                         ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_void_p)]
    lib.rbgs_qr_graph_launch.argtypes = [vp, vp, i32]
    lib.rbgs_qr_batched_graph_create.argtypes = [ctypes.POINTER(Problem), i64, ctypes.c_int, ctypes.POINTER(Opts),
                                                 i32, ctypes.POINTER(ctypes.c_void_p)]
    lib.rbgs_qr_graph_destroy.argtypes = [vp]
    lib.rbgs_qr_host.argtypes = [vp, i64, i64, i64, i64, ctypes.c_int, i64, u64, vp, i64, vp, i64,
                                 ctypes.POINTER(Opts), ctypes.POINTER(Stats)]
    lib.rbgs_release_workspace.argtypes = []
    lib.rbgs_sparse_sign_columns.argtypes = [u64, i64, i64, i64, vp, vp]
    lib.rbgs_gaussian_entries.argtypes = [u64, i64, vp, vp, i64, vp]
    lib.rbgs_version.restype = ctypes.c_char_p
    lib.rbgs_launch_count.restype = ctypes.c_int64
    for name in ("rbgs_qr", "rbgs_sketch_apply", "rbgs_tall_update", "rbgs_tall_update_noalloc", "rbgs_philox",
                 "rbgs_release_workspace", "rbgs_op_apply", "rbgs_block_arnoldi", "rbgs_block_gmres",
                 "rbgs_block_fom", "rbgs_rayleigh_ritz", "rbgs_qr_batched", "rbgs_qr_host",
                 "rbgs_embedding_check", "rbgs_cholqr_postprocess", "rbgs_qr_graph_create",
                 "rbgs_qr_graph_launch", "rbgs_qr_graph_destroy", "rbgs_sparse_sign_columns",
                 "rbgs_gaussian_entries"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def header_functions() -> list[str]:
    """Names of the functions that include/rbgs.h declares."""
    txt = _HDR.read_text()
    return sorted(set(re.findall(r"^\s*(?:RBGS_API\s+)?(?:rbgs_status|void|const char\*)\s+(rbgs_\w+)\s*\(", txt, re.M)))


def colmajor(t: torch.Tensor) -> torch.Tensor:
    """Column-major copy (shape kept, stride (1, rows))."""
    return t.t().contiguous().t()


def _ld(t: torch.Tensor, name: str) -> int:
    """Leading dimension of a column-major 2-D tensor (the stride between columns)."""
    if t.dim() != 2:
        raise ValueError(f"{name} must be 2-D")
    rows, cols = t.shape
    if rows > 1 and t.stride(0) != 1:
        raise ValueError(f"{name} must be column-major (stride (1, ld)); use colmajor()")
    ld = t.stride(1)
    if cols <= 1 and ld < rows:
        ld = rows  # a single column: any ld >= rows addresses it
    return max(int(ld), 1)


def _stream_ptr(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _check(code: int, where: str):
    if code != 0:
        raise RbgsError(code, where)


def _prec_of(t: torch.Tensor, prec: str | None) -> str:
    if prec is None:
        return "fp64" if t.dtype == torch.float64 else "tf32x3"
    want = torch.float64 if prec == "fp64" else torch.float32
    if t.dtype != want:
        raise ValueError(f"precision {prec} needs {want}, got {t.dtype}")
    return prec


def _empty_cols(n: int, m: int, dtype, device) -> torch.Tensor:
    """An n x m column-major tensor whose leading dimension is a multiple of 4
    (the tensor-core paths read columns with 16-byte aligned copies)."""
    ld = (n + 3) // 4 * 4
    return torch.empty((m, ld), dtype=dtype, device=device).t()[:n]


def rbgs_qr(W: torch.Tensor, mb: int, sketch: str = "srht", k: int | None = None, seed: int = 0,
            prec: str | None = None, ls_iters: int = 2, reorth: int = 0, reorth_tol: float = 1e-8,
            certify: bool = False, Q: torch.Tensor | None = None, R: torch.Tensor | None = None, stream=None,
            sync: bool = True, timing: bool = False, fine: bool = False, interblock: int = 5, ls: str = "richardson",
            trsm: bool = False):
    """RBGS QR of W (n x m, column-major).  Returns (Q, R, QRStats | None).
    fine=True (FP32 / TF32X3 storage only) runs the sketch-space steps in FP64;
    interblock selects steps 4-5: 5 = Alg. 5 (implicit sketch), 4 = Alg. 4,
    1 / 3 = column by column (RGS / Alg. 3), 6 = Alg. 6 (l2 QR, then Alg. 4);
    trsm=True (interblock 4) scales by R_ii^{-1} with a row-wise triangular
    solve instead of the explicit inverse."""
    lib = load()
    prec = _prec_of(W, prec)
    n, m = W.shape
    k = 2 * m if k is None else k
    if Q is None:
        Q = _empty_cols(n, m, W.dtype, W.device)
    if R is None:
        R = torch.empty((m, m), dtype=torch.float64, device=W.device).t()
    o = Opts()
    lib.rbgs_opts_default(ctypes.byref(o))
    o.prec, o.ls_iters, o.reorth, o.certify = PREC[prec], ls_iters, reorth, int(certify)
    o.reorth_tol, o.stream, o.sync, o.timing = reorth_tol, _stream_ptr(stream), int(sync), int(timing)
    o.fine = int(fine)
    o.interblock = int(interblock)
    o.ls = LS[ls]
    o.trsm = int(bool(trsm))
    st = Stats()
    code = lib.rbgs_qr(W.data_ptr(), n, m, _ld(W, "W"), mb, SKETCH[sketch], k, seed, Q.data_ptr(), _ld(Q, "Q"),
                       R.data_ptr(), _ld(R, "R"), ctypes.byref(o), ctypes.byref(st) if sync else None)
    _check(code, "rbgs_qr")
    stats = (QRStats(st.delta, st.delta_tilde, st.passes2, bool(st.certified), st.tall_ms, st.tall_bytes,
                     st.tall_launches, st.chol_rounds2) if sync else None)
    return Q, R, stats


def embedding_check(Z: torch.Tensor, mb: int, sketch: str = "srht", k: int | None = None, seed_theta: int = 0,
                    seed_phi: int = 1, prec: str | None = None, ls_iters: int = 2, reorth: int = 0,
                    fine: bool = False, stream=None) -> float:
    """||I - (Theta Q_phi)^T (Theta Q_phi)||_F with Q_phi the RBGS factor of Z
    under an independent sketch Phi (the a posteriori check of Sec. 4)."""
    lib = load()
    prec = _prec_of(Z, prec)
    n, m = Z.shape
    k = 2 * m if k is None else k
    o = Opts()
    lib.rbgs_opts_default(ctypes.byref(o))
    o.prec, o.ls_iters, o.reorth, o.fine, o.stream = PREC[prec], ls_iters, reorth, int(fine), _stream_ptr(stream)
    out = ctypes.c_double(0.0)
    _check(lib.rbgs_embedding_check(Z.data_ptr(), n, m, _ld(Z, "Z"), mb, SKETCH[sketch], k, seed_theta, seed_phi,
                                     ctypes.byref(o), ctypes.cast(ctypes.pointer(out), ctypes.c_void_p)),
           "rbgs_embedding_check")
    return float(out.value)


class QRGraph:
    """rbgs_qr captured once as a CUDA graph on fixed W, Q, R (column-major
    CUDA tensors, kept alive by this object); launch() replays it on the
    current contents of W."""

    def __init__(self, W: torch.Tensor, mb: int, sketch: str = "srht", k: int | None = None, seed: int = 0,
                 prec: str | None = None, ls_iters: int = 2, reorth: int = 0, reorth_tol: float = 1e-8,
                 fine: bool = False, interblock: int = 5, ls: str = "richardson"):
        lib = load()
        prec = _prec_of(W, prec)
        n, m = W.shape
        k = 2 * m if k is None else k
        self.W = W
        self.Q = _empty_cols(n, m, W.dtype, W.device)
        self.R = torch.empty((m, m), dtype=torch.float64, device=W.device).t()
        o = Opts()
        lib.rbgs_opts_default(ctypes.byref(o))
        o.prec, o.ls_iters, o.reorth, o.reorth_tol = PREC[prec], ls_iters, reorth, reorth_tol
        o.fine, o.interblock, o.ls = int(fine), int(interblock), LS[ls]
        h = ctypes.c_void_p()
        _check(lib.rbgs_qr_graph_create(W.data_ptr(), n, m, _ld(W, "W"), mb, SKETCH[sketch], k, seed,
                                        self.Q.data_ptr(), _ld(self.Q, "Q"), self.R.data_ptr(), _ld(self.R, "R"),
                                        ctypes.byref(o), ctypes.byref(h)), "rbgs_qr_graph_create")
        self._h = h

    def launch(self, stream=None, sync: bool = True):
        _check(load().rbgs_qr_graph_launch(self._h, _stream_ptr(stream), int(sync)), "rbgs_qr_graph_launch")
        return self.Q, self.R

    def destroy(self):
        if self._h:
            load().rbgs_qr_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class BatchedQRGraph:
    """rbgs_qr_batched captured once as one CUDA graph on fixed W, Q, R of every
    problem (column-major CUDA tensors, kept alive by this object); launch()
    replays the whole batch with one graph launch and returns (Qs, Rs,
    statuses, passes2)."""

    def __init__(self, Ws: list, mbs, ks, seeds, sketch: str = "gauss", prec: str | None = None, ls_iters: int = 2,
                 reorth: int = 0, reorth_tol: float = 1e-8, fine: bool = False, interblock: int = 5,
                 nstreams: int = 8, trsm: bool = False):
        lib = load()
        cnt = len(Ws)
        pick = (lambda v, i: v[i] if isinstance(v, (list, tuple)) else v)
        prec = _prec_of(Ws[0], prec)
        self.Ws = list(Ws)
        self.Qs = [_empty_cols(W.shape[0], W.shape[1], W.dtype, W.device) for W in Ws]
        self.Rs = [torch.empty((W.shape[1], W.shape[1]), dtype=torch.float64, device=W.device).t() for W in Ws]
        self.probs = (Problem * cnt)()
        for i, W in enumerate(Ws):
            n, m = W.shape
            self.probs[i] = Problem(W.data_ptr(), n, m, _ld(W, "W"), int(pick(mbs, i)), int(pick(ks, i)),
                                    int(pick(seeds, i)), self.Qs[i].data_ptr(), _ld(self.Qs[i], "Q"),
                                    self.Rs[i].data_ptr(), _ld(self.Rs[i], "R"), 0, 0)
        o = Opts()
        lib.rbgs_opts_default(ctypes.byref(o))
        o.prec, o.ls_iters, o.reorth, o.reorth_tol = PREC[prec], ls_iters, reorth, reorth_tol
        o.fine, o.interblock, o.trsm = int(fine), int(interblock), int(bool(trsm))
        h = ctypes.c_void_p()
        _check(lib.rbgs_qr_batched_graph_create(self.probs, cnt, SKETCH[sketch], ctypes.byref(o), int(nstreams),
                                                ctypes.byref(h)), "rbgs_qr_batched_graph_create")
        self._h = h
        self.count = cnt

    def launch(self, stream=None, sync: bool = True):
        code = load().rbgs_qr_graph_launch(self._h, _stream_ptr(stream), int(sync))
        if code not in (0, 4, 6):
            _check(code, "rbgs_qr_graph_launch")
        return (self.Qs, self.Rs, [int(self.probs[i].status) for i in range(self.count)],
                [int(self.probs[i].passes2) for i in range(self.count)])

    def destroy(self):
        if self._h:
            load().rbgs_qr_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def cholqr_postprocess(Q: torch.Tensor, R: torch.Tensor, mb: int = 64, prec: str | None = None, stream=None):
    """In place: Q <- Q R'^{-1}, R <- R' R with R' = chol(Q^T Q) (the remark
    after Alg. 2), making Q l2-orthonormal.  Returns (Q, R)."""
    lib = load()
    prec = _prec_of(Q, prec)
    n, m = Q.shape
    _check(lib.rbgs_cholqr_postprocess(PREC[prec], n, m, Q.data_ptr(), _ld(Q, "Q"), R.data_ptr(), _ld(R, "R"), mb,
                                        _stream_ptr(stream), 1), "rbgs_cholqr_postprocess")
    return Q, R


def rbgs_qr_host(W: torch.Tensor, mb: int, sketch: str = "srht", k: int | None = None, seed: int = 0,
                 prec: str | None = None, ls_iters: int = 2, reorth: int = 0, reorth_tol: float = 1e-8,
                 Q: torch.Tensor | None = None, R: torch.Tensor | None = None, fine: bool = False,
                 interblock: int = 5, stream=None, timing: bool = False):
    """rbgs_qr on host (CPU) tensors, column-major; pinned memory lets the
    copies overlap the factorization.  Returns (Q, R, QRStats); with timing
    the stats carry the call's timeline (host_up_ms, host_compute_ms,
    host_total_ms)."""
    lib = load()
    if W.is_cuda:
        raise ValueError("W must be a host tensor")
    prec = _prec_of(W, prec)
    n, m = W.shape
    k = 2 * m if k is None else k
    pin = W.is_pinned()
    if Q is None:
        Q = torch.empty((m, n), dtype=W.dtype, pin_memory=pin).t()
    if R is None:
        R = torch.empty((m, m), dtype=torch.float64, pin_memory=pin).t()
    o = Opts()
    lib.rbgs_opts_default(ctypes.byref(o))
    o.prec, o.ls_iters, o.reorth, o.reorth_tol = PREC[prec], ls_iters, reorth, reorth_tol
    o.fine, o.interblock, o.stream = int(fine), int(interblock), _stream_ptr(stream)
    o.timing = int(timing)
    st = Stats()
    _check(lib.rbgs_qr_host(W.data_ptr(), n, m, _ld(W, "W"), mb, SKETCH[sketch], k, seed, Q.data_ptr(), _ld(Q, "Q"),
                            R.data_ptr(), _ld(R, "R"), ctypes.byref(o), ctypes.byref(st)), "rbgs_qr_host")
    return Q, R, QRStats(st.delta, st.delta_tilde, st.passes2, False, 0.0, 0.0, 0, st.chol_rounds2, st.host_up_ms,
                         st.host_compute_ms, st.host_total_ms)


def rbgs_qr_batched(Ws: list, mbs, ks, seeds, sketch: str = "gauss", prec: str | None = None, ls_iters: int = 2,
                    reorth: int = 0, reorth_tol: float = 1e-8, fine: bool = False, interblock: int = 5,
                    nstreams: int = 8, Qs: list | None = None, Rs: list | None = None, stream=None,
                    trsm: bool = False):
    """Independent RBGS factorizations of the column-major matrices Ws (one
    mb, k and seed per problem, or one value for all) on nstreams internal
    streams.  Returns (Qs, Rs, statuses, passes2)."""
    lib = load()
    cnt = len(Ws)
    pick = (lambda v, i: v[i] if isinstance(v, (list, tuple)) else v)
    prec = _prec_of(Ws[0], prec) if cnt else (prec or "fp64")
    if Qs is None:
        Qs = [_empty_cols(W.shape[0], W.shape[1], W.dtype, W.device) for W in Ws]
    if Rs is None:
        Rs = [torch.empty((W.shape[1], W.shape[1]), dtype=torch.float64, device=W.device).t() for W in Ws]
    probs = (Problem * max(cnt, 1))()
    for i, W in enumerate(Ws):
        n, m = W.shape
        probs[i] = Problem(W.data_ptr(), n, m, _ld(W, "W"), int(pick(mbs, i)), int(pick(ks, i)), int(pick(seeds, i)),
                           Qs[i].data_ptr(), _ld(Qs[i], "Q"), Rs[i].data_ptr(), _ld(Rs[i], "R"), 0, 0)
    o = Opts()
    lib.rbgs_opts_default(ctypes.byref(o))
    o.prec, o.ls_iters, o.reorth, o.reorth_tol = PREC[prec], ls_iters, reorth, reorth_tol
    o.fine, o.interblock, o.stream = int(fine), int(interblock), _stream_ptr(stream)
    o.trsm = int(bool(trsm))
    code = lib.rbgs_qr_batched(probs, cnt, SKETCH[sketch], ctypes.byref(o), int(nstreams))
    if code not in (0, 4, 6):  # per-problem breakdowns and timeouts are reported in the statuses
        _check(code, "rbgs_qr_batched")
    return Qs, Rs, [int(probs[i].status) for i in range(cnt)], [int(probs[i].passes2) for i in range(cnt)]


def sketch_apply(X: torch.Tensor, sketch: str, k: int, seed: int, prec: str | None = None, stream=None,
                 sync: bool = True) -> torch.Tensor:
    """Y = Theta X (k x ncols, float64)."""
    lib = load()
    prec = _prec_of(X, prec)
    n, c = X.shape
    Y = torch.empty((c, k), dtype=torch.float64, device=X.device).t()
    code = lib.rbgs_sketch_apply(SKETCH[sketch], k, n, seed, PREC[prec], X.data_ptr(), _ld(X, "X"), c, Y.data_ptr(),
                                 k, _stream_ptr(stream), int(sync))
    _check(code, "rbgs_sketch_apply")
    return Y


def tall_update(Qprev: torch.Tensor | None, X: torch.Tensor, G: torch.Tensor, prec: str | None = None,
                out: torch.Tensor | None = None, stream=None, sync: bool = True) -> torch.Tensor:
    """Qout = [Qprev | X] G."""
    lib = load()
    prec = _prec_of(X, prec)
    n, mb = X.shape
    c = 0 if Qprev is None else Qprev.shape[1]
    if out is None:
        out = torch.empty((mb, n), dtype=X.dtype, device=X.device).t()
    Gc = colmajor(G.to(device=X.device, dtype=torch.float64))
    code = lib.rbgs_tall_update(PREC[prec], n, c, mb, 0 if Qprev is None else Qprev.data_ptr(),
                                n if Qprev is None else _ld(Qprev, "Qprev"), X.data_ptr(), _ld(X, "X"),
                                Gc.data_ptr(), _ld(Gc, "G"), out.data_ptr(), _ld(out, "out"), _stream_ptr(stream),
                                int(sync))
    _check(code, "rbgs_tall_update")
    return out


def tall_update_noalloc(Qprev: torch.Tensor | None, X: torch.Tensor, G: torch.Tensor, out: torch.Tensor,
                        prec: str | None = None, stream=None, sync: bool = True) -> torch.Tensor:
    """Qout = [Qprev | X] G like tall_update, through the entry point that
    allocates no device memory (scratch is a fixed buffer inside the library;
    c + mb <= NOALLOC_MAX_K).  G must already be a column-major float64 CUDA
    tensor and out must be given, so this call allocates nothing either."""
    lib = load()
    prec = _prec_of(X, prec)
    n, mb = X.shape
    c = 0 if Qprev is None else Qprev.shape[1]
    if not (G.is_cuda and G.dtype == torch.float64):
        raise ValueError("G must be a float64 CUDA tensor")
    code = lib.rbgs_tall_update_noalloc(PREC[prec], n, c, mb, 0 if Qprev is None else Qprev.data_ptr(),
                                        n if Qprev is None else _ld(Qprev, "Qprev"), X.data_ptr(), _ld(X, "X"),
                                        G.data_ptr(), _ld(G, "G"), out.data_ptr(), _ld(out, "out"),
                                        _stream_ptr(stream), int(sync))
    _check(code, "rbgs_tall_update_noalloc")
    return out


def op_apply(op: Op, X: torch.Tensor, prec: str | None = None, stream=None) -> torch.Tensor:
    """Y = A X (column-major CUDA tensors; float64 for fp64, else float32)."""
    lib = load()
    prec = _prec_of(X, prec)
    n, c = X.shape
    Y = torch.empty((c, n), dtype=X.dtype, device=X.device).t()
    _check(lib.rbgs_op_apply(ctypes.byref(op), PREC[prec], X.data_ptr(), _ld(X, "X"), c, Y.data_ptr(), n,
                             _stream_ptr(stream), 1), "rbgs_op_apply")
    return Y


def _krylov_opts(prec, ls_iters, reorth, reorth_tol, fine, stream, interblock=5, trsm=False):
    o = Opts()
    load().rbgs_opts_default(ctypes.byref(o))
    o.prec, o.ls_iters, o.reorth, o.reorth_tol = PREC[prec], ls_iters, reorth, reorth_tol
    o.stream, o.fine = _stream_ptr(stream), int(fine)
    o.interblock, o.trsm = int(interblock), int(bool(trsm))
    return o


def block_arnoldi(op: Op, B: torch.Tensor, p: int, sketch: str = "srht", k: int | None = None, seed: int = 0,
                  prec: str | None = None, ls_iters: int = 2, reorth: int = 0, reorth_tol: float = 1e-8,
                  fine: bool = False, Q: torch.Tensor | None = None, R: torch.Tensor | None = None, stream=None,
                  interblock: int = 5, trsm: bool = False):
    """Alg. 7: returns (Q, R) with A Q[:, :(p-1) mb] = Q R[:, mb:]."""
    lib = load()
    prec = _prec_of(B, prec)
    n, mb = B.shape
    m = p * mb
    k = 2 * m if k is None else k
    if Q is None:
        Q = torch.empty((m, n), dtype=B.dtype, device=B.device).t()
    if R is None:
        R = torch.empty((m, m), dtype=torch.float64, device=B.device).t()
    o = _krylov_opts(prec, ls_iters, reorth, reorth_tol, fine, stream, interblock, trsm)
    st = Stats()
    _check(lib.rbgs_block_arnoldi(ctypes.byref(op), B.data_ptr(), _ld(B, "B"), mb, p, SKETCH[sketch], k, seed,
                                  Q.data_ptr(), _ld(Q, "Q"), R.data_ptr(), _ld(R, "R"), ctypes.byref(o),
                                  ctypes.byref(st)), "rbgs_block_arnoldi")
    return Q, R


def _block_solve(fn: str, op: Op, B: torch.Tensor, X: torch.Tensor | None, p: int, rtol: float, max_cycles: int,
                 sketch: str, k: int | None, seed: int, prec: str, ls_iters: int, reorth: int, reorth_tol: float,
                 fine: bool, stream, raise_on_noconv: bool, interblock: int = 5, trsm: bool = False):
    lib = load()
    n, mb = B.shape
    if B.dtype != torch.float64:
        raise ValueError("B must be float64")
    if X is None:
        X = torch.zeros((mb, n), dtype=torch.float64, device=B.device).t()
    k = 2 * p * mb if k is None else k
    o = _krylov_opts(prec, ls_iters, reorth, reorth_tol, fine, stream, interblock, trsm)
    cyc = ctypes.c_int64(0)
    rel = (ctypes.c_double * mb)()
    code = getattr(lib, fn)(ctypes.byref(op), B.data_ptr(), _ld(B, "B"), X.data_ptr(), _ld(X, "X"), mb, p,
                            float(rtol), int(max_cycles), SKETCH[sketch], k, seed, ctypes.byref(o),
                            ctypes.byref(cyc), ctypes.cast(rel, ctypes.c_void_p))
    if code == 7 and not raise_on_noconv:
        code = 0
    _check(code, fn)
    return X, int(cyc.value), [float(v) for v in rel]


def block_gmres(op: Op, B: torch.Tensor, X: torch.Tensor | None = None, p: int = 10, rtol: float = 1e-8,
                max_cycles: int = 100, sketch: str = "srht", k: int | None = None, seed: int = 0,
                prec: str = "fp64", ls_iters: int = 2, reorth: int = 0, reorth_tol: float = 1e-8,
                fine: bool = False, stream=None, raise_on_noconv: bool = False, interblock: int = 5,
                trsm: bool = False):
    """Restarted randomized block GMRES (Sec. 5.2): returns (X, cycles, relres)."""
    return _block_solve("rbgs_block_gmres", op, B, X, p, rtol, max_cycles, sketch, k, seed, prec, ls_iters, reorth,
                        reorth_tol, fine, stream, raise_on_noconv, interblock, trsm)


def block_fom(op: Op, B: torch.Tensor, X: torch.Tensor | None = None, p: int = 10, rtol: float = 1e-8,
              max_cycles: int = 100, sketch: str = "srht", k: int | None = None, seed: int = 0,
              prec: str = "fp64", ls_iters: int = 2, reorth: int = 0, reorth_tol: float = 1e-8,
              fine: bool = False, stream=None, raise_on_noconv: bool = False, interblock: int = 5,
              trsm: bool = False):
    """Restarted randomized block FOM (Sec. 5.3): returns (X, cycles, relres)."""
    return _block_solve("rbgs_block_fom", op, B, X, p, rtol, max_cycles, sketch, k, seed, prec, ls_iters, reorth,
                        reorth_tol, fine, stream, raise_on_noconv, interblock, trsm)


RITZ_WHICH = {"LR": 0, "SR": 1}


def rayleigh_ritz(op: Op, B0: torch.Tensor, p: int = 10, n_iter: int = 1, which: str = "LR", sketch: str = "srht",
                  k: int | None = None, seed: int = 0, prec: str = "fp64", ls_iters: int = 2, reorth: int = 0,
                  reorth_tol: float = 1e-8, fine: bool = False, X: torch.Tensor | None = None, stream=None,
                  interblock: int = 5, trsm: bool = False):
    """Randomized Rayleigh-Ritz with restarting (Alg. 8, Sec. 5.4).  B0: n x mb
    float64 on the device.  Returns (values (complex, mb), X (n x mb float64,
    unit columns), resid (mb estimates ||H_(p,1:p-1) y||))."""
    lib = load()
    n, mb = B0.shape
    if B0.dtype != torch.float64:
        raise ValueError("B0 must be float64")
    if X is None:
        X = torch.empty((mb, n), dtype=torch.float64, device=B0.device).t()
    k = 2 * p * mb if k is None else k
    o = _krylov_opts(prec, ls_iters, reorth, reorth_tol, fine, stream, interblock, trsm)
    re, im, rs = (ctypes.c_double * mb)(), (ctypes.c_double * mb)(), (ctypes.c_double * mb)()
    _check(lib.rbgs_rayleigh_ritz(ctypes.byref(op), B0.data_ptr(), _ld(B0, "B0"), mb, p, n_iter, RITZ_WHICH[which],
                                  SKETCH[sketch], k, seed, ctypes.byref(o), X.data_ptr(), _ld(X, "X"),
                                  ctypes.cast(re, ctypes.c_void_p), ctypes.cast(im, ctypes.c_void_p),
                                  ctypes.cast(rs, ctypes.c_void_p)), "rbgs_rayleigh_ritz")
    vals = [complex(re[j], im[j]) for j in range(mb)]
    return vals, X, [float(v) for v in rs]


def sparse_sign_columns(seed: int, k: int, j0: int, count: int):
    """Rows (count x z) and negative flags of the nonzeros of columns j0 ..
    j0 + count - 1 of the sparse-sign Theta, z = min(8, k), as numpy arrays
    (the generator the sketch kernels evaluate, run on the host)."""
    import numpy as np

    lib = load()
    z = min(8, int(k))
    rows = np.zeros((count, z), dtype=np.int64)
    neg = np.zeros((count, z), dtype=np.int32)
    _check(lib.rbgs_sparse_sign_columns(int(seed), int(k), int(j0), int(count), rows.ctypes.data, neg.ctypes.data),
           "rbgs_sparse_sign_columns")
    return rows, neg


def gaussian_entries(seed: int, k: int, r, j):
    """Entries Theta(r[t], j[t]) of the Gaussian Theta (k rows) as a float64
    numpy array, from the generator the sketch kernels evaluate, run on the
    host."""
    import numpy as np

    lib = load()
    r = np.ascontiguousarray(r, dtype=np.int64)
    j = np.ascontiguousarray(j, dtype=np.int64)
    if r.shape != j.shape:
        raise ValueError("r and j must have the same shape")
    out = np.zeros(r.shape, dtype=np.float64)
    _check(lib.rbgs_gaussian_entries(int(seed), int(k), r.ctypes.data, j.ctypes.data, int(r.size), out.ctypes.data),
           "rbgs_gaussian_entries")
    return out


def philox(ctr: torch.Tensor, seed: int, stream=None) -> torch.Tensor:
    """Philox4x32-10 blocks for counters ctr (count x 4, int32/uint32 bits, CUDA)."""
    lib = load()
    c = ctr.contiguous()
    out = torch.empty_like(c)
    code = lib.rbgs_philox(seed, c.data_ptr(), out.data_ptr(), c.shape[0], _stream_ptr(stream), 1)
    _check(code, "rbgs_philox")
    return out


def release_workspace():
    _check(load().rbgs_release_workspace(), "rbgs_release_workspace")


def launch_count() -> int:
    """Kernels launched by librbgs in this process so far."""
    return int(load().rbgs_launch_count())


def version() -> str:
    return load().rbgs_version().decode()


# ------------------------------------------------- the learned preconditioner --

def _images(t: torch.Tensor, n: int, name: str):
    """n x batch FP32 CUDA tensor with leading dimension n (image b = column b)."""
    if t.dtype != torch.float32 or t.shape[0] != n or (t.shape[1] > 1 and t.stride(1) != n) or t.stride(0) != 1:
        raise ValueError(f"{name} must be a float32 n x batch tensor with leading dimension n")
    return t.shape[1]


def unet_num_params(widths) -> int:
    n = load().rbgs_unet_num_params(ctypes.byref(unet_shape(widths)))
    if n < 0:
        raise ValueError("invalid U-Net shape")
    return int(n)


def unet_forward(widths, params: torch.Tensor, N: int, x: torch.Tensor, save: bool = False, stream=None,
                 sync: bool = True, simt: bool = False) -> torch.Tensor:
    """y = U-Net(x) for the columns of x (N^2 x batch, float32)."""
    lib = load()
    b = _images(x, N * N, "x")
    y = torch.empty((b, N * N), dtype=torch.float32, device=x.device).t()
    _check(lib.rbgs_unet_forward(ctypes.byref(unet_shape(widths, simt)), params.data_ptr(), N, b, x.data_ptr(),
                                 y.data_ptr(), int(save), _stream_ptr(stream), int(sync)), "rbgs_unet_forward")
    return y


def unet_backward(widths, params: torch.Tensor, N: int, x: torch.Tensor, gy: torch.Tensor,
                  grads: torch.Tensor | None = None, stream=None, sync: bool = True, simt: bool = False) -> torch.Tensor:
    """d sum(gy * y) / d params of the last forward with save=True."""
    lib = load()
    b = _images(x, N * N, "x")
    _images(gy, N * N, "gy")
    if grads is None:
        grads = torch.empty(params.numel(), dtype=torch.float32, device=params.device)
    _check(lib.rbgs_unet_backward(ctypes.byref(unet_shape(widths, simt)), params.data_ptr(), N, b, x.data_ptr(),
                                  gy.data_ptr(), grads.data_ptr(), _stream_ptr(stream), int(sync)),
           "rbgs_unet_backward")
    return grads


def unet_residual_loss(N: int, coef: torch.Tensor, field: torch.Tensor, x: torch.Tensor, y: torch.Tensor,
                       gy: torch.Tensor | None = None, loss: torch.Tensor | None = None, stream=None,
                       sync: bool = True):
    """(loss (device float64 scalar tensor), gy) of the residual-norm loss;
    coef: (fields, stride) float64 face coefficients, field: int32 per image."""
    lib = load()
    b = _images(x, N * N, "x")
    if gy is None:
        gy = torch.empty((b, N * N), dtype=torch.float32, device=x.device).t()
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float64, device=x.device)
    _check(lib.rbgs_unet_residual_loss(N, b, coef.data_ptr(), coef.stride(0), field.data_ptr(), x.data_ptr(),
                                       y.data_ptr(), gy.data_ptr(), loss.data_ptr(), _stream_ptr(stream), int(sync)),
           "rbgs_unet_residual_loss")
    return loss, gy


def adam_step(params: torch.Tensor, grads: torch.Tensor, m: torch.Tensor, v: torch.Tensor, t: int, lr: float = 1e-3,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, stream=None, sync: bool = True):
    lib = load()
    _check(lib.rbgs_adam_step(params.numel(), params.data_ptr(), grads.data_ptr(), m.data_ptr(), v.data_ptr(), int(t),
                              lr, beta1, beta2, eps, _stream_ptr(stream), int(sync)), "rbgs_adam_step")


def unet_scale_inputs(Q: torch.Tensor, X: torch.Tensor | None = None, prec: str | None = None, stream=None,
                      sync: bool = True) -> torch.Tensor:
    """X = Q's columns scaled to unit root mean square (float32, ld n)."""
    lib = load()
    prec = _prec_of(Q, prec)
    n, c = Q.shape
    if X is None:
        X = torch.empty((c, n), dtype=torch.float32, device=Q.device).t()
    _check(lib.rbgs_unet_scale_inputs(n, c, PREC[prec], Q.data_ptr(), _ld(Q, "Q"), X.data_ptr(), _ld(X, "X"),
                                      _stream_ptr(stream), int(sync)), "rbgs_unet_scale_inputs")
    return X


def unet_precondition(widths, params: torch.Tensor, N: int, Q: torch.Tensor, prec: str | None = None,
                      stream=None) -> torch.Tensor:
    """Z = M(Q) (float64 or float32 columns of N^2 rows)."""
    lib = load()
    prec = _prec_of(Q, prec)
    n, c = Q.shape
    Z = torch.empty((c, n), dtype=Q.dtype, device=Q.device).t()
    _check(lib.rbgs_unet_precondition(ctypes.byref(unet_shape(widths)), params.data_ptr(), N, PREC[prec],
                                      Q.data_ptr(), _ld(Q, "Q"), c, Z.data_ptr(), n, _stream_ptr(stream), 1),
           "rbgs_unet_precondition")
    return Z


def block_fgmres(op: Op, widths, params: torch.Tensor | None, B: torch.Tensor, X: torch.Tensor | None = None,
                 p: int = 10, rtol: float = 1e-8, max_cycles: int = 100, accept: float = 0.9, sketch: str = "srht",
                 k: int | None = None, seed: int = 0, prec: str = "fp64", ls_iters: int = 2, reorth: int = 0,
                 reorth_tol: float = 1e-8, fine: bool = False, stream=None, interblock: int = 5,
                 trsm: bool = False):
    """Restarted randomized block flexible GMRES with the U-Net preconditioner
    (widths=None: plain block GMRES).  Returns (X, cycles, relres, fallbacks)."""
    lib = load()
    n, mb = B.shape
    if X is None:
        X = torch.zeros((mb, n), dtype=torch.float64, device=B.device).t()
    k = 2 * p * mb if k is None else k
    o = _krylov_opts(prec, ls_iters, reorth, reorth_tol, fine, stream, interblock, trsm)
    cyc, fb = ctypes.c_int64(0), ctypes.c_int64(0)
    rel = (ctypes.c_double * mb)()
    net = ctypes.byref(unet_shape(widths)) if widths is not None else None
    code = lib.rbgs_block_fgmres(ctypes.byref(op), net, params.data_ptr() if params is not None else None,
                                 B.data_ptr(), _ld(B, "B"), X.data_ptr(), _ld(X, "X"), mb, p, rtol, max_cycles,
                                 accept, SKETCH[sketch], k, seed, ctypes.byref(o), ctypes.byref(cyc),
                                 ctypes.cast(rel, ctypes.c_void_p), ctypes.byref(fb))
    if code not in (0, 7):
        _check(code, "rbgs_block_fgmres")
    return X, int(cyc.value), [float(r) for r in rel], int(fb.value)

