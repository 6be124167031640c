"""Write tests/golden/flops_per_face.txt: the algorithmic FP64 operation count per face
of the benchmark workloads, counted by the CPU oracle's op-counting scalar (one per
+, -, *, /, sqrt, compare/min/max/abs) on seeded samples of the initial states.

Calls only oracle/ and the seeded input generators.  Run:
    python tests/golden/gen_flops.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as orc  # noqa: E402
from paper_2010_13289_gb300 import problems as PB  # noqa: E402


def sample(shape, axis, m, rng):
    idx = np.zeros((m, 3), dtype=np.int32)
    for a, n in enumerate(shape):
        idx[:, a] = rng.integers(0, n + 1 if a == axis else n, m)
    return idx


def count(name, prim, shape, dx, K, lim, m=20000, seed=0):
    g = orc.make_grid(shape, dx, (orc.BC_PERIODIC,) * len(shape))
    S = orc.make_scheme(K, limiter=lim)
    U = orc.init_state(g, prim)
    rng = np.random.default_rng(seed)
    per_axis = []
    for a in range(len(shape)):
        idx = sample(shape, a, m, rng)
        per_axis.append(orc.face_flops_at(g, S, U, a, idx) / m)
    return "%s K=%d lim=%s %s" % (name, K, "MP" if lim == 0 else "TVD5", " ".join("%.1f" % f for f in per_axis))


def main():
    lines = ["# Mean counted FP64 operations per face (per axis), oracle op counter, 20000",
             "# seeded faces per axis of the initial state.  Written by tests/golden/gen_flops.py.",
             "# workload K limiter flops_axis0 [flops_axis1 [flops_axis2]]"]
    prim, dx = PB.broadband_2d(2048, 2)
    lines.append(count("broadband_2d_2048", prim, (2048, 2048), (dx, dx), 6, 0))
    lines.append(count("broadband_2d_2048", prim, (2048, 2048), (dx, dx), 8, 1))
    del prim
    prim, dx = PB.solenoidal_3d(256, 3)
    lines.append(count("solenoidal_3d_256", prim, (256, 256, 256), (dx, dx, dx), 8, 0, m=6000))
    del prim
    sizes, prims, dxs = PB.batch_riemann(512, 4)
    tot, nf = 0, 0
    rng = np.random.default_rng(1)
    for j in rng.choice(512, 16, replace=False):
        n = int(sizes[j])
        g = orc.make_grid((n,), (dxs[j],), (orc.BC_TRANSMISSIVE,))
        S = orc.make_scheme(6)
        U = orc.init_state(g, prims[j])
        tot += orc.face_flops(g, S, U, 0)
        nf += n + 1
    lines.append("riemann_1d_batch K=6 lim=MP %.1f" % (tot / nf))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "flops_per_face.txt")
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
