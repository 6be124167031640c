"""Cases of the full-run parity tests (test_gpu_fullrun.py) and the oracle side of them.
Imported by spawned worker processes, so it imports neither torch nor the CUDA library."""
from paper_2010_13289_gb300 import problems as PB

RUNS = {
    # name: (generator, n, seed, K, limiter, steps)
    "broadband_2d_128_teno6_mp": ("broadband_2d", 128, 2, 6, 0, 60),
    "broadband_2d_128_teno8_tvd5": ("broadband_2d", 128, 2, 8, 1, 60),
    "solenoidal_3d_32_teno8_mp": ("solenoidal_3d", 32, 3, 8, 0, 20),
}


def initial(name):
    gen, n, seed, K, lim, steps = RUNS[name]
    if gen == "broadband_2d":
        prim, dx = PB.broadband_2d(n, seed)
        return prim, (n, n), (dx, dx)
    prim, dx = PB.solenoidal_3d(n, seed)
    return prim, (n, n, n), (dx, dx, dx)


def oracle_run(name):
    """Runs in a spawned process: the oracle from the seeded state, `steps` SSP-RK3 steps
    at CFL 0.4 (dt from each step's state), no end time."""
    import oracle as orc
    prim, shape, dx = initial(name)
    gen, n, seed, K, lim, steps = RUNS[name]
    g = orc.make_grid(shape, dx, (orc.BC_PERIODIC,) * len(shape))
    so = orc.make_scheme(K, limiter=lim)
    U0 = orc.init_state(g, prim)
    U, t, nst, bad = orc.advance(g, so, U0, 1e300, 0.4, steps)
    return U, t, nst, bad
