"""Full-run parity of multi-dimensional workloads: the GPU solver (device-side CFL dt,
SSP-RK3 through tenom_advance) against the CPU oracle advanced from the same seeded
state, relative L1 <= 1e-10 per conserved component over the whole run.  The paper states
the method dimension by dimension (Section 4: Eq. approximateEq along each axis), so the
2D and 3D operators are checked through whole runs, not only one face sweep at a time.

Reduced sizes of the benchmarked workloads, so that the oracle finishes in seconds:
  2D broadband field with circular jumps at 128^2, TENO6-MP and TENO8-TVD5, 60 steps;
  3D solenoidal field (rms Mach 0.6) at 32^3, TENO8-MP, 20 steps.
The three oracle runs start together in spawned processes before the first GPU call."""
import concurrent.futures as cf
import math
import multiprocessing as mp

import numpy as np
import pytest

from fullrun_cases import RUNS, initial, oracle_run
from parity import bound_counts, central_terms, compare_faces

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

@pytest.fixture(scope="module")
def oracle_results():
    ex = cf.ProcessPoolExecutor(max_workers=len(RUNS), mp_context=mp.get_context("spawn"))
    futs = {name: ex.submit(oracle_run, name) for name in RUNS}
    yield futs
    ex.shutdown(wait=True)


@pytest.fixture(scope="module")
def T(oracle_results):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2010_13289_gb300 import tenom
    tenom.lib()
    return tenom


@pytest.mark.parametrize("name", sorted(RUNS))
def test_full_run_relative_l1(T, orc, oracle_results, name):
    gen, n, seed, K, lim, steps = RUNS[name]
    prim, shape, dx = initial(name)
    S = T.Solver(shape, dx, (T.BC_PERIODIC,) * len(shape), T.make_scheme(K, limiter=lim))
    U = S.init_state(torch.from_numpy(prim).cuda())
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    S.advance(U, steps, t_end=math.inf, cfl=0.4, t_dev=t)
    Ug = U.cpu().numpy()
    Uo, to, nst, bad = oracle_results[name].result(timeout=1800)
    assert bad == 0 and nst == steps
    assert t.item() == pytest.approx(to, rel=1e-13)
    axes = tuple(range(1, Uo.ndim))
    l1 = np.sum(np.abs(Ug - Uo), axis=axes) / np.sum(np.abs(Uo), axis=axes)
    assert np.all(l1 <= 1e-10), (name, l1)
    # the end states' face decisions: counted, and away from the cutoff identical
    g = orc.make_grid(shape, dx, (orc.BC_PERIODIC,) * len(shape))
    so = orc.make_scheme(K, limiter=lim)
    Ugd = torch.from_numpy(Uo).cuda()
    for a in range(len(shape)):
        Fg, flg = S.face_dump(Ugd, a)
        Fo, flo, cut, noise, badf, scale = orc.faces(g, so, Uo, a, with_scale=True)
        scale = np.maximum(scale, central_terms(Uo, a, K, 0))
        st = compare_faces(Fg.cpu().numpy(), flg.cpu().numpy(), Fo, flo, cut, noise, scale,
                           label="%s end state axis %d" % (name, a))
        bound_counts(st)
    assert S.status() == 0
    S.close()
