"""Write tests/golden/le_blanc_900_envelope.txt: how far the CPU oracle's own Le Blanc run
(Section 4.4.2, Eq. Leblanc: 900 cells, gamma = 5/3, TENO8-MP with the minmod curvature and
beta = 1, positivity limiter, CFL 0.4, t = 6) moves when its initial state is perturbed by
1 or 4 units in the last place (seeded random signs): the relative L1 distance per
component from the unperturbed run, for each of 8 perturbations.  The run holds
rounding-decided events, so a different rounding of the same arithmetic can land up to
this far from the oracle; the GPU parity test takes its tolerance from the largest of them.

Calls only oracle/ and the seeded input generators.  Run:
    python tests/golden/gen_le_blanc_envelope.py
"""
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as orc  # noqa: E402
from paper_2010_13289_gb300 import problems as PB  # noqa: E402

N = 900
PERTURBATIONS = [(seed, ulps) for ulps in (1, 4) for seed in range(4)]


def run(pert):
    prim, dx = PB.le_blanc_1d(N)
    g = orc.make_grid((N,), (dx,), (orc.BC_TRANSMISSIVE,), gamma=PB.LE_BLANC_GAMMA)
    s = orc.make_scheme(8, orc.LIM_MP, mp_curv=orc.CURV_MM, mp_beta=1.0, positivity=1)
    U0 = orc.init_state(g, prim)
    if pert is not None:
        seed, ulps = pert
        sign = np.random.default_rng(seed).choice([-1.0, 1.0], U0.shape)
        U0 = U0 * (1.0 + ulps * 2.0 ** -52 * sign)
    U, t, steps, _ = orc.advance(g, s, U0, 6.0, 0.4)
    return U


def main():
    orc.build()
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        res = pool.map(run, [None] + PERTURBATIONS)
    base = res[0]
    lines = ["# Le Blanc, 900 cells, TENO8-MP (minmod curvature, beta = 1), positivity limiter, t = 6",
             "# (Section 4.4.2, Eq. Leblanc): relative L1 distance per component (rho, rho u, E) of the",
             "# oracle's run from an initial state perturbed by `ulps` units in the last place with",
             "# seeded random signs.  Written by gen_le_blanc_envelope.py (oracle only).",
             "# seed ulps l1_rho l1_mom l1_E"]
    for (seed, ulps), U in zip(PERTURBATIONS, res[1:]):
        l1 = np.abs(U - base).sum(1) / np.abs(base).sum(1)
        lines.append("%d %d %.6e %.6e %.6e" % (seed, ulps, l1[0], l1[1], l1[2]))
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "le_blanc_900_envelope.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
