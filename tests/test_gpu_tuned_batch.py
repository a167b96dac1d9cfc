"""The autotuned batch (rbgs_qr_batched_auto): every problem runs with the
configuration chosen for its shape class, and each result matches the oracle
whichever variant was chosen."""
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


def dev(A, dtype):
    A = np.asarray(A)
    return torch.from_numpy(np.ascontiguousarray(A.T)).to("cuda", dtype).t()


def test_autotuned_batch_matches_the_oracle(rb, tmp_path):
    from paper_2111_14641_gb300 import autotune as at

    shapes = [(3000, 32, 8), (20000, 48, 16), (3100, 32, 8), (24000, 48, 16), (2900, 32, 8)]
    Ws = [synth.svd_matrix(n, m, 1e3, 70 + i).astype(np.float32).astype(np.float64)
          for i, (n, m, _) in enumerate(shapes)]
    Wd = [dev(W, torch.float32) for W in Ws]
    mbs = [mb for _, _, mb in shapes]
    ks = [3 * m for _, m, _ in shapes]
    cache = str(tmp_path / "tuned.json")
    tuner = at.BatchTuner(streams=(1, 4), sample=2, reps=1, cache_file=cache,
                          device_name=torch.cuda.get_device_name())
    Qs, Rs, st, p2, cfg = at.rbgs_qr_batched_auto(Wd, mbs, ks, 5, "gauss", tuner=tuner, ls_iters=2, reorth=1,
                                                  fine=True)
    assert st == [0] * len(shapes)
    assert p2 == [m // mb - 1 for _, m, mb in shapes]
    assert cfg[0] == cfg[2] == cfg[4] and cfg[1] == cfg[3]
    assert all(c[0] in at.FP32_VARIANTS and c[1] in (1, 4) for c in cfg)
    assert len(tuner.cache) == 2
    for i, (n, m, mb) in enumerate(shapes):
        R = Rs[i].double().cpu().numpy()
        Q = Qs[i].double().cpu().numpy()
        ref = oracle.rbgs(Ws[i], mb, "gauss", ks[i], 5, variant=5, ls="richardson", ls_iters=2, reorth=True,
                          ls_iters_first=1)
        assert np.allclose(np.tril(R, -1), 0.0) and np.all(np.diag(R) > 0)
        assert np.abs(R - ref["R"]).max() <= 1e-2 * np.abs(ref["R"]).max()
        assert oracle.factorization_error(Ws[i], Q, R) < 2e-6
    # the cached choice is reused without timing
    tuner2 = at.BatchTuner(streams=(1, 4), cache_file=cache, device_name=torch.cuda.get_device_name())
    _, _, st2, _, cfg2 = at.rbgs_qr_batched_auto(Wd, mbs, ks, 5, "gauss", tuner=tuner2, ls_iters=2, reorth=1,
                                                 fine=True)
    assert cfg2 == cfg and st2 == st and tuner2.trials == {}
