"""Many independent factorizations in one call (rbgs_qr_batched): every problem
equals its single rbgs_qr result bit for bit, whatever the number of streams,
matches the oracle, and a breakdown stays local to its problem."""
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


SHAPES = [(2000, 16, 4), (3100, 24, 8), (4096, 40, 8), (2500, 12, 4), (5000, 32, 16), (2048, 20, 8), (3000, 9, 4)]


@pytest.mark.parametrize("prec", ["fp64", "f16x3"])
@pytest.mark.parametrize("nstreams", [1, 3, 8])
def test_batched_equals_single_calls_and_oracle(rb, prec, nstreams):
    td = torch.float64 if prec == "fp64" else torch.float32
    Ws = [synth.svd_matrix(n, m, 1e3, 40 + i) for i, (n, m, _) in enumerate(SHAPES)]
    if prec != "fp64":
        Ws = [W.astype(np.float32).astype(np.float64) for W in Ws]
    mbs = [mb for _, _, mb in SHAPES]
    ks = [2 * m for _, m, _ in SHAPES]
    seeds = [100 + i for i in range(len(SHAPES))]
    Wd = [dev(W, td) for W in Ws]
    Qs, Rs, status, passes2 = rb.rbgs_qr_batched(Wd, mbs, ks, seeds, "gauss", prec=prec, ls_iters=2, reorth=1,
                                                  fine=prec != "fp64", nstreams=nstreams)
    assert status == [0] * len(SHAPES)
    assert passes2 == [(m + mb - 1) // mb - 1 for _, m, mb in SHAPES]
    for i, (n, m, mb) in enumerate(SHAPES):
        Q1, R1, _ = rb.rbgs_qr(Wd[i], mbs[i], "gauss", ks[i], seeds[i], prec=prec, ls_iters=2, reorth=1,
                               fine=prec != "fp64")
        assert torch.equal(Qs[i], Q1) and torch.equal(Rs[i], R1)
        ref = oracle.rbgs(Ws[i], mb, "gauss", ks[i], seeds[i], variant=5, ls="richardson", ls_iters=2, reorth=True,
                          ls_iters_first=1)
        R = host(Rs[i])
        tol = 1e-10 if prec == "fp64" else 1e-2
        assert np.abs(R - ref["R"]).max() <= tol * np.abs(ref["R"]).max()
        assert oracle.factorization_error(Ws[i], host(Qs[i]), R) < (1e-14 if prec == "fp64" else 2e-6)


def test_batched_breakdown_stays_local(rb):
    """A zero column makes its problem's Cholesky pivot vanish: that problem
    reports RBGS_EBREAKDOWN, the others are unaffected."""
    Ws = [synth.svd_matrix(n, m, 1e2, 60 + i) for i, (n, m, _) in enumerate(SHAPES[:4])]
    Ws[2] = Ws[2].copy()
    Ws[2][:, 5] = 0.0
    Wd = [dev(W) for W in Ws]
    mbs = [mb for _, _, mb in SHAPES[:4]]
    ks = [2 * m for _, m, _ in SHAPES[:4]]
    Qs, Rs, status, _ = rb.rbgs_qr_batched(Wd, mbs, ks, 5, "gauss", prec="fp64", nstreams=2)
    assert status[2] == 4 and [s for i, s in enumerate(status) if i != 2] == [0, 0, 0]
    for i in (0, 1, 3):
        Q1, R1, _ = rb.rbgs_qr(Wd[i], mbs[i], "gauss", ks[i], 5, prec="fp64")
        assert torch.equal(Qs[i], Q1) and torch.equal(Rs[i], R1)


def test_batched_rejects_a_bad_problem_before_any_work(rb):
    Wd = [dev(synth.gaussian(100, 8, 1)), dev(synth.gaussian(120, 8, 2))]
    with pytest.raises(rb.RbgsError):
        rb.rbgs_qr_batched(Wd, [4, 4], [16, 200], 0, "gauss", prec="fp64")   # k > n in the second problem


@pytest.mark.parametrize("prec,pinned", [("fp64", True), ("f16x3", True), ("f16x3", False), ("fp32", True)])
def test_host_buffer_path_equals_device_path(rb, prec, pinned):
    """rbgs_qr_host (host W, Q, R; copies overlapped with the factorization)
    gives bit for bit the device path's result, ragged last block included."""
    n, m, mb, k = 5001, 70, 16, 160
    td = torch.float64 if prec == "fp64" else torch.float32
    W = synth.svd_matrix(n, m, 1e3, 21)
    Wh = torch.from_numpy(np.ascontiguousarray(W.T)).to(td).t()
    if pinned:
        Wh = Wh.t().contiguous().pin_memory().t()
    Qh, Rh, st = rb.rbgs_qr_host(Wh, mb, "srht", k, 3, prec=prec, ls_iters=1, reorth=1, fine=prec != "fp64")
    Wd = Wh.t().contiguous().cuda().t()
    if prec != "fp64":  # the tensor-core paths need a leading dimension that is a multiple of 4
        buf = torch.zeros((m, (n + 3) // 4 * 4), dtype=td, device="cuda")
        buf[:, :n] = Wd.t()
        Wd = buf.t()[:n]
    Qd, Rd, std = rb.rbgs_qr(Wd, mb, "srht", k, 3, prec=prec, ls_iters=1, reorth=1, fine=prec != "fp64")
    assert torch.equal(Qh, Qd.cpu()) and torch.equal(Rh, Rd.cpu())
    assert st.passes2 == std.passes2 == (m + mb - 1) // mb - 1


@pytest.mark.parametrize("prec,n,m,mb,kind,k,interblock", [("fp64", 10000, 100, 10, "gauss", 200, 5),
                                                           ("f16x3", 20000, 128, 32, "srht", 256, 5),
                                                           ("fp32", 8000, 60, 16, "srht", 160, 4),
                                                           ("fp64", 6000, 40, 8, "gauss", 80, 6)])
def test_graph_replay_equals_direct_call(rb, prec, n, m, mb, kind, k, interblock):
    """A captured factorization replays bit for bit the direct rbgs_qr, and a
    replay after W changes factorizes the new contents (2 W: R doubles)."""
    td = torch.float64 if prec == "fp64" else torch.float32
    W = synth.svd_matrix(n, m, 1e3, 31)
    if prec != "fp64":
        W = W.astype(np.float32).astype(np.float64)
    Wd = dev(W, td)
    kw = dict(prec=prec, ls_iters=2, reorth=1, fine=prec != "fp64", interblock=interblock)
    g = rb.QRGraph(Wd, mb, kind, k, 6, **kw)
    for _ in range(2):
        Qg, Rg = g.launch()
    Q1, R1, _ = rb.rbgs_qr(Wd, mb, kind, k, 6, **kw)
    assert torch.equal(Qg, Q1) and torch.equal(Rg, R1)
    Wd.mul_(2.0)
    Qg2, Rg2 = g.launch()
    assert torch.allclose(Rg2, 2.0 * R1, rtol=1e-12, atol=0) and torch.allclose(Qg2, Q1, rtol=1e-12, atol=1e-14)
    g.destroy()


def test_graph_refuses_the_column_by_column_variants(rb):
    Wd = dev(synth.gaussian(2000, 16, 3))
    with pytest.raises(rb.RbgsError):
        rb.QRGraph(Wd, 4, "gauss", 32, 0, prec="fp64", interblock=3)


@pytest.mark.parametrize("prec,interblock,trsm", [("fp64", 5, False), ("f16x3", 5, False), ("f16x3", 4, True)])
@pytest.mark.parametrize("nstreams", [1, 4])
def test_batched_graph_replays_the_batch(rb, prec, interblock, trsm, nstreams):
    """The batch captured as one CUDA graph: a replay gives the batched call's
    results bit for bit, and a replay after new contents of every W gives the
    factorization of the new matrices (again equal to the batched call)."""
    td = torch.float64 if prec == "fp64" else torch.float32
    Wd = [dev(synth.svd_matrix(n, m, 1e3, 60 + i), td) for i, (n, m, _) in enumerate(SHAPES)]
    mbs = [mb for _, _, mb in SHAPES]
    ks = [2 * m for _, m, _ in SHAPES]
    seeds = [300 + i for i in range(len(SHAPES))]
    kw = dict(ls_iters=1, reorth=1, fine=2 if prec != "fp64" else 0, interblock=interblock, trsm=trsm)
    g = rb.BatchedQRGraph(Wd, mbs, ks, seeds, "gauss", prec=prec, nstreams=nstreams, **kw)
    for round_ in range(2):
        if round_:
            for i, (n, m, _) in enumerate(SHAPES):
                Wd[i].copy_(dev(synth.svd_matrix(n, m, 1e2, 90 + i), td))
        Qg, Rg, st, p2 = g.launch()
        Qs = [q.clone() for q in Qg]
        Rs = [r.clone() for r in Rg]
        assert st == [0] * len(SHAPES)
        Qb, Rb, stb, _ = rb.rbgs_qr_batched(Wd, mbs, ks, seeds, "gauss", prec=prec, nstreams=nstreams, **kw)
        assert stb == [0] * len(SHAPES)
        for i in range(len(SHAPES)):
            assert torch.equal(Qs[i], Qb[i]) and torch.equal(Rs[i], Rb[i]), (round_, i)
    g.destroy()


def test_near_duplicate_blocks_of_32_do_not_break_down(rb):
    """Problems 3, 12 and 26 of the many-small-problems workload put up to four
    near-duplicate columns (relative perturbation 1e-7) into one block of 32,
    so the sketch of the projected block has a condition number near 1e7-1e8
    and an unshifted FP64 Cholesky factor of its Gram matrix meets a
    non-positive pivot.  With the row-wise solve (Alg. 4, opts.trsm) the first
    Cholesky round takes the shifted Cholesky QR shift: every status is OK,
    W = QR holds at the FP32 level and cond(Q) = O(1)."""
    specs = synth.batch_specs(32)
    pick = [3, 12, 26]
    Ws = [synth.near_duplicate_matrix_torch(specs[i][0], specs[i][1], 11 + i, device="cuda", dtype=torch.float32)
          for i in pick]
    mbs = [specs[i][2] for i in pick]
    ks = [2 * specs[i][1] for i in pick]
    seeds = [7 + i for i in pick]
    kw = dict(ls_iters=1, reorth=1, fine=2, interblock=4, trsm=True)
    Qs, Rs, status, _ = rb.rbgs_qr_batched(Ws, mbs, ks, seeds, "gauss", prec="f16x3", nstreams=2, **kw)
    assert status == [0, 0, 0]
    for W, Q, R in zip(Ws, Qs, Rs):
        Wd, Qd = W.double(), Q.double()
        fe = float(torch.linalg.norm(Wd - Qd @ R) / torch.linalg.norm(Wd))
        sv = torch.linalg.svdvals(Qd)
        assert fe < 1e-6 and float(sv[0] / sv[-1]) < 10.0, (fe, float(sv[0] / sv[-1]))
    # a single call on the same problem gives the same factors
    Q1, R1, _ = rb.rbgs_qr(Ws[0], mbs[0], "gauss", ks[0], seeds[0], prec="f16x3", **kw)
    assert torch.equal(Q1, Qs[0]) and torch.equal(R1, Rs[0])
