"""Write tests/golden/small_direct.npz: the oracle's direct sum (Eq. (direct_sum))
for the 1000-point uniform workload in medium A (seed 0, one density vector).

Calls only oracle/ and workloads/ (seeded inputs).  Run from the repo root:
    python tests/golden/make_small_direct.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
import workloads  # noqa: E402


def main():
    x, y, q = workloads.small_uniform()
    t = time.time()
    u = oracle.direct_apply(workloads.MEDIUM_A, x, y, q)
    print(f"direct sum of {x.size} points in {time.time() - t:.1f} s")
    np.savez_compressed(os.path.join(ROOT, "tests", "golden", "small_direct.npz"), u=u,
                        medium=np.array(workloads.MEDIUM_A), seed=0)


if __name__ == "__main__":
    main()
