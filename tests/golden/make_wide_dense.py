"""Write tests/golden/wide_dense_sample.npz: the oracle's direct sum (Eq.
(direct_sum)) over all 1M sources of the wide-strip workload (medium
k = (1, 8, 2), d = 1, seed 0, 16 dense N(0,1) density vectors) at 8 sampled
targets.  This is the benchmark's own input; the sample checks its dense
16-vector output element by element.

Calls only oracle/ and workloads/ (seeded inputs).  About 15 minutes on 8
cores (one target per thread).  Run from the repo root:
    python tests/golden/make_wide_dense.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
import workloads  # noqa: E402

N, NVEC, SEED, NTGT = 1_000_000, 16, 0, 8


def fingerprint(x, y, q):
    """A few input values and sums, so that a change in the seeded generator is detected."""
    return np.concatenate([x[:4], y[:4], [x.sum(), y.sum()], q[:, :2].ravel().view(np.float64),
                           [q.real.sum(), q.imag.sum()]])


def main():
    x, y, q = workloads.wide_uniform(N, NVEC, seed=SEED)
    tg = np.sort(np.random.default_rng(SEED + 1).choice(N, NTGT, replace=False))
    t = time.time()
    u = oracle.direct_apply(workloads.MEDIUM_B, x, y, q, targets=tg, nthreads=NTGT)
    print(f"{NTGT} targets x {N} sources x {NVEC} vectors in {time.time() - t:.1f} s")
    np.savez_compressed(os.path.join(ROOT, "tests", "golden", "wide_dense_sample.npz"), u=u, targets=tg,
                        medium=np.array(workloads.MEDIUM_B), seed=SEED, fingerprint=fingerprint(x, y, q))


if __name__ == "__main__":
    main()
