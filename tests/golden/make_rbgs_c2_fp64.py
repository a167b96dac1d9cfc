"""Writes tests/golden/rbgs_c2_fp64.json: the CPU oracle's RBGS factorization
of the full-size mixed-precision workload, sampled, for the full-size GPU
parity tests.  It calls only the oracle and the seeded input generator.

Workload: n = 1,000,000, m = 1000, m_p = 50, SRHT k = 2000 (seed 1), W the
FP32 matrix of ``synth.hadamard_svd_matrix`` (sigma log-spaced from 1 to
1e-6, seed 7), which the CPU and the device build bit for bit.  The oracle
runs Alg. 2 in FP64 with steps 4-5 by Alg. 5, step 2 by one Richardson
iteration, and the second projection pass on every block (the options the
benchmark times).

Stored: W's bit checksum (to confirm the GPU factors the same matrix), R's
diagonal, sixteen whole columns of R with the condition number kappa_j of
R_{1:j,1:j} (= cond(Theta W_{:,1:j}), which scales the forward error of
column j), four whole rows of Q, the quality measures (||W - QR||_F/||W||_F,
||I - (Theta Q)^T (Theta Q)|| in the Frobenius and 2-norm, cond(Q)), and how
long the oracle took on how many threads of which CPU.

Run:  python tests/golden/make_rbgs_c2_fp64.py   (minutes; about 30 GB of RAM)
"""
import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
import oracle  # noqa: E402
import synth  # noqa: E402

N, M, MB, K, SEED_THETA, SEED_W, COND = 1_000_000, 1000, 50, 2000, 1, 7, 1e6
R_COLS = [0, 1, 49, 50, 99, 149, 250, 399, 499, 500, 650, 799, 899, 949, 950, 999]
Q_ROWS = [0, 1, 123457, 999999]


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu model")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def main():
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    W32 = synth.hadamard_svd_matrix(N, M, COND, SEED_W)
    checksum = synth.bit_checksum(W32)
    W = np.asfortranarray(W32.astype(np.float64))
    del W32
    t0 = time.perf_counter()
    out = oracle.rbgs(W, MB, "srht", K, SEED_THETA, variant=5, ls="richardson", ls_iters=1, reorth=True,
                      ls_iters_first=1)
    seconds = time.perf_counter() - t0
    assert out["rc"] == 0, out["rc"]
    Q, R = out["Q"], out["R"]
    # quality, in FP64 with the oracle's own Theta
    num = den = 0.0
    for r0 in range(0, N, 100_000):
        Wc = W[r0:r0 + 100_000]
        E = Wc - Q[r0:r0 + 100_000] @ R
        num += float((E * E).sum())
        den += float((Wc * Wc).sum())
    del W
    d_fro, d_two = oracle.sketched_orthogonality(Q, "srht", K, SEED_THETA)
    ev = np.linalg.eigvalsh(Q.T @ Q)
    cols = {}
    for j in R_COLS:
        sv = np.linalg.svd(R[: j + 1, : j + 1], compute_uv=False)
        cols[str(j)] = {"kappa": float(sv[0] / sv[-1]), "R": [float(x) for x in R[: j + 1, j]]}
    doc = {
        "what": "oracle RBGS (Alg. 2, steps 4-5 by Alg. 5, Richardson l = 1, second pass on every block) in FP64 "
                "of synth.hadamard_svd_matrix(1e6, 1000, 1e6, seed 7), SRHT k = 2000 seed 1; written by "
                "tests/golden/make_rbgs_c2_fp64.py from the oracle only",
        "n": N, "m": M, "mb": MB, "k": K, "sketch": "srht", "seed_theta": SEED_THETA, "seed_w": SEED_W,
        "cond": COND, "w_bit_checksum": checksum,
        "passes2": out["passes2"], "delta": float(out["delta"]), "delta_tilde": float(out["delta_tilde"]),
        "quality": {"rel_factorization_error": float(np.sqrt(num / den)), "sketched_orthogonality_fro": d_fro,
                    "sketched_orthogonality_2": d_two, "cond_Q": float(np.sqrt(ev.max() / ev.min()))},
        "kappa_R": float(np.linalg.cond(R)),
        "R_diag": [float(x) for x in np.diag(R)],
        "R_cols": cols,
        "Q_rows": {str(i): [float(x) for x in Q[i]] for i in Q_ROWS},
        "oracle_seconds": seconds, "oracle_threads": threads, "cpu": cpu_model(),
    }
    with open(os.path.join(HERE, "rbgs_c2_fp64.json"), "w") as f:
        json.dump(doc, f, indent=0)
    print(f"oracle {seconds:.1f} s on {threads} threads; quality {doc['quality']}")


if __name__ == "__main__":
    main()
