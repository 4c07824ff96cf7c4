"""Writes the oracle's full-size reference reconstructions used by the GPU
parity tests: the 512 x 512 (0.8 mm), 738-bin fan-beam slices with 800 and
200 views, 30 split-Bregman x 8 CG iterations (inputs from the seeded
generator, rounded to FP32 as the GPU receives them).  Calls only the FP64 oracle; takes ~15 min on 8 cores.

    python tests/golden/make_golden.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1310_1434_gb300 import inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    for w in (inputs.AIR512_V200, inputs.AIR512_V800):
        out = os.path.join(HERE, f"{w.name}_oracle.npz")
        _, _, Y = inputs.make_case(w)
        Y = Y.astype(np.float32).astype(np.float64)     # the input the GPU sees
        g = oracle.Geometry(**{k: getattr(w.geom, k) for k in oracle.Geometry.__dataclass_fields__})
        t = time.time()
        X, resid = oracle.solve(g, Y, w.lam, w.mu, w.n_outer, w.n_cg, return_resid=True)
        np.savez_compressed(out, X=X.astype(np.float32), resid=resid, lam=w.lam, mu=w.mu,
                            n_outer=w.n_outer, n_cg=w.n_cg, threads=oracle.threads(),
                            seconds=time.time() - t)
        print(w.name, f"{time.time() - t:.1f}s", float(np.linalg.norm(X)), flush=True)


if __name__ == "__main__":
    main()
