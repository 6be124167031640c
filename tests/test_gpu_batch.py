"""Batched persistent path (many independent 1D problems of uneven size): results equal the
separate per-problem launches and the CPU oracle; finished problems are masked."""
import numpy as np
import pytest

from paper_2010_13289_gb300 import problems as PB

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2010_13289_gb300 import tenom
    tenom.lib()
    return tenom


def make_batch(T, nprob, seed, nmin, nmax, K=6, lim=0):
    sizes, prims, dxs = PB.batch_riemann(nprob, seed, nmin, nmax)
    B = T.Batch(sizes, dxs, T.make_scheme(K, limiter=lim))
    prim = np.zeros((3, B.total))
    for j in range(nprob):
        prim[:, B.off[j]:B.off[j + 1]] = prims[j]
    U = B.init_state(torch.from_numpy(prim).cuda())
    return B, U, sizes, prims, dxs


def separate(T, sizes, prims, dxs, steps, K=6, lim=0, t_end=float("inf")):
    outs = []
    for n, p, dx in zip(sizes, prims, dxs):
        S = T.Solver((int(n),), (dx,), (T.BC_TRANSMISSIVE,), T.make_scheme(K, limiter=lim))
        U = S.init_state(torch.from_numpy(p).cuda())
        t = torch.zeros(1, dtype=torch.float64, device="cuda")
        S.advance(U, steps, t_end=t_end, cfl=0.4, t_dev=t)
        outs.append(U.cpu().numpy())
        S.close()
    return outs


@pytest.mark.parametrize("K,lim,graph", [(6, 0, True), (8, 1, True), (6, 0, False)])
def test_batch_equals_separate_launches(T, K, lim, graph):
    B, U, sizes, prims, dxs = make_batch(T, 24, 11 + K, 16, 700, K, lim)
    B.step(U, nsteps=6, graph=graph)
    ref = separate(T, sizes, prims, dxs, 6, K, lim)
    Ub = U.cpu().numpy()
    for j in range(B.P):
        got = Ub[:, B.off[j]:B.off[j + 1]]
        np.testing.assert_allclose(got, ref[j], rtol=1e-13, atol=1e-14)
    assert B.status() == 0


@pytest.mark.parametrize("tile", [64, 128, 256])
def test_tiles_give_identical_results(T, tile):
    B, U, *_ = make_batch(T, 12, 5, 20, 500)
    B2, U2, *_ = make_batch(T, 12, 5, 20, 500)
    B.set_tiling(128, 2)
    B2.set_tiling(tile, 1)
    B.step(U, nsteps=3)
    B2.step(U2, nsteps=3)
    d = (U - U2).abs().max().item()
    print("tile", tile, "max abs diff", d, "bitwise", torch.equal(U, U2))
    np.testing.assert_allclose(U2.cpu().numpy(), U.cpu().numpy(), rtol=1e-13, atol=1e-14)


def test_autotune_keeps_results(T):
    B, U, *_ = make_batch(T, 40, 9, 64, 2000)
    B2, U2, *_ = make_batch(T, 40, 9, 64, 2000)
    tile, ctas = B.autotune(U)
    assert tile in (64, 128, 256) and 1 <= ctas <= 8
    B.step(U, nsteps=2)
    B2.step(U2, nsteps=2)
    np.testing.assert_allclose(U2.cpu().numpy(), U.cpu().numpy(), rtol=1e-13, atol=1e-14)


def test_batch_full_run_matches_oracle_and_masks_finished(T, orc):
    """Each problem runs to its own t_end = 0.15 with its own CFL steps; the oracle's result
    per problem agrees to 1e-10 relative L1, and steps after t_end change nothing."""
    B, U, sizes, prims, dxs = make_batch(T, 6, 21, 32, 256)
    B.set_time(0.0, 0.15)
    steps = []
    ref = []
    for n, p, dx in zip(sizes, prims, dxs):
        g = orc.make_grid((int(n),), (dx,), (orc.BC_TRANSMISSIVE,))
        Uo, t, st, bad = orc.advance(g, orc.make_scheme(6), orc.init_state(g, p), 0.15, 0.4)
        steps.append(st)
        ref.append(Uo)
    B.step(U, nsteps=max(steps))
    t = B.times()
    np.testing.assert_allclose(t, 0.15, rtol=1e-14)
    Ub = U.cpu().numpy()
    for j in range(B.P):
        got = Ub[:, B.off[j]:B.off[j + 1]]
        l1 = np.sum(np.abs(got - ref[j]), axis=1) / np.sum(np.abs(ref[j]), axis=1)
        assert np.all(l1 <= 1e-10), (j, l1)
    before = U.clone()
    B.step(U, nsteps=3)
    assert torch.equal(U, before)
    np.testing.assert_allclose(B.times(), 0.15, rtol=1e-14)
