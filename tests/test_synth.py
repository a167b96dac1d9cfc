"""The seeded input recipes, checked on the CPU against their stated shapes and
structure (they serve both the oracle and the GPU path, and hold none of the
method's arithmetic)."""
import numpy as np
import pytest

import synth


def test_batch_specs_follow_the_recipe():
    specs = synth.batch_specs(256)
    assert len(specs) == 256
    ns = np.array([s[0] for s in specs])
    assert ns.min() >= 20000 and ns.max() <= 200000
    assert {s[1] for s in specs} == {64, 128, 192, 256}
    assert {s[2] for s in specs} == {16, 32}
    assert specs == synth.batch_specs(256)  # seeded


def test_near_duplicate_columns():
    """Every 8th column is an earlier column plus noise of relative size 1e-7,
    so the FP32 matrix is numerically rank deficient; the others are N(0, 1)."""
    torch = pytest.importorskip("torch")
    n, m = 4000, 64
    W = synth.near_duplicate_matrix_torch(n, m, 5, device="cpu", dtype=torch.float64).numpy()
    Wn = W / np.linalg.norm(W, axis=0)
    for j in range(m):
        d = np.linalg.norm(Wn[:, :j] - Wn[:, [j]], axis=0).min() if j else np.inf
        if j % 8 == 0 and j:
            assert 1e-8 < d < 1e-6, (j, d)
        else:
            assert d > 0.5, (j, d)
    sv = np.linalg.svd(W, compute_uv=False)
    assert sv[0] / sv[-1] > 1e6
    assert np.abs(np.linalg.norm(W[:, 1], axis=0) / np.sqrt(n) - 1) < 0.05


def test_svd_matrix_has_the_stated_spectrum():
    W = synth.svd_matrix(2000, 40, 1e8, seed=7)
    sv = np.linalg.svd(W, compute_uv=False)
    np.testing.assert_allclose(sv, synth.sigmas(40, 1e8), rtol=1e-6)
    assert sv[0] / sv[-1] == pytest.approx(1e8, rel=1e-6)
