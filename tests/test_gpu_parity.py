"""Parity of the CUDA path (through the C ABI) with the CPU oracle on identical seeded
inputs.  Runs on a GB300 (-m gpu)."""
import math

import numpy as np
import pytest

from paper_2010_13289_gb300 import problems as PB
from parity import (CUT_TOL, NOISE_K, bound_counts, central_terms, central_terms_at, compare_cells, compare_faces,
                    compare_rhs, dilate, switch_cells)

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


def schemes(T, orc, K, lim, **kw):
    return T.make_scheme(K, limiter=lim, **kw), orc.make_scheme(K, limiter=lim, **kw)


def setup(T, orc, shape, bc, K, lim, prim, dx=None, **kw):
    dim = len(shape)
    dx = dx or tuple(1.0 / n for n in shape)
    sg, so = schemes(T, orc, K, lim, **kw)
    S = T.Solver(shape, dx, bc, sg)
    g = orc.make_grid(shape, dx, bc)
    Uo = orc.init_state(g, prim)
    Ug = S.init_state(torch.from_numpy(np.ascontiguousarray(prim)).cuda())
    return S, g, so, Uo, Ug


CASES = [
    # (shape x-first, bc, K, limiter, jumps)
    ((300,), (1,), 6, 0, True),
    ((300,), (0,), 8, 1, True),
    ((257,), (1,), 8, 0, True),
    ((70, 45), (0, 0), 6, 0, True),
    ((70, 45), (1, 0), 8, 1, True),
    ((33, 40), (0, 1), 8, 0, True),
    ((64, 64), (0, 0), 6, 1, False),
    ((20, 13, 11), (0, 0, 0), 8, 0, True),
    ((20, 13, 11), (1, 0, 1), 6, 1, True),
    ((9, 8, 17), (0, 1, 0), 6, 0, True),
]


@pytest.mark.parametrize("shape,bc,K,lim,jumps", CASES)
def test_face_flux_parity(T, orc, shape, bc, K, lim, jumps):
    """Per-face Fhat (1e-13 relative) and per-field/side flags on every axis."""
    prim = PB.random_state(tuple(reversed(shape)), seed=sum(shape) + K + lim, jumps=jumps)
    S, g, so, Uo, Ug = setup(T, orc, shape, bc, K, lim, prim)
    np.testing.assert_allclose(Ug.cpu().numpy(), Uo, rtol=1e-15, atol=1e-15)
    Fs = []
    sw = []
    for a in range(len(shape)):
        Fg, flg = S.face_dump(Ug, a)
        Fo, flo, cut, noise, bad, scale = orc.faces(g, so, Uo, a, with_scale=True)
        scale = np.maximum(scale, central_terms(Uo, a, so.K, g.bc[a]))
        assert bad == 0
        st = compare_faces(Fg.cpu().numpy(), flg.cpu().numpy(), Fo, flo, cut, noise, scale,
                           label="%s axis %d" % (shape, a))
        # near-cutoff switches are rare; noise-decided ones sit where a characteristic field
        # is flat to rounding (transmissive ghost copies, the acoustic fields across a
        # contact): up to 4 % of the faces on the small 3D grids with transmissive axes
        bound_counts(st, noise_frac=0.05)
        Fs.append(Fo)
        sw.append((flg.cpu().numpy() != flo).reshape(flo.shape[:-2] + (-1,)).any(axis=-1))
    ro, _ = orc.rhs(g, so, Uo)
    rg = S.rhs(Ug).cpu().numpy()
    ex = switch_cells(sw, ro.shape[1:])
    compare_rhs(rg, ro, Fs, [1.0 / n for n in shape], exclude=ex, label="rhs %s" % (shape,))
    assert S.status() == 0


def face_parity_checks(T, orc, S, g, so, Uo, Ug, shape):
    for a in range(len(shape)):
        Fg, flg = S.face_dump(Ug, a)
        Fo, flo, cut, noise, bad, scale = orc.faces(g, so, Uo, a, with_scale=True)
        scale = np.maximum(scale, central_terms(Uo, a, so.K, g.bc[a]))
        assert bad == 0
        st = compare_faces(Fg.cpu().numpy(), flg.cpu().numpy(), Fo, flo, cut, noise, scale,
                           label="%s axis %d" % (shape, a))
        bound_counts(st, noise_frac=0.05)
    assert S.status() == 0


# Scheme options beyond the two benchmarked ones: the Van Albada limiter (TENO-M-VA,
# Section 3.2.3), the MP variants with the 2-argument minmod curvature and beta = 2 / 1
# (Sections 3.2.2, 4), the classical renormalised TENO weights (Eq. weight_renormalize),
# non-maximal-order d_k (no central-formula shortcut), the constant and adaptive C_T on the
# other stencil width, a larger MP alpha.
VARIANTS = [
    ((70, 45), (0, 0), 6, 2, {}),
    ((70, 45), (1, 0), 8, 2, {}),
    ((20, 13, 11), (0, 1, 0), 8, 2, {}),
    ((300,), (1,), 6, 2, {}),
    ((70, 45), (0, 0), 6, 0, {"mp_curv": 1, "mp_beta": 2.0}),
    ((70, 45), (0, 1), 8, 0, {"mp_curv": 1, "mp_beta": 1.0}),
    ((70, 45), (0, 0), 6, 0, {"mp_alpha": 2.0}),
    ((70, 45), (0, 0), 6, 0, {"weights": 1}),
    ((70, 45), (1, 1), 8, 0, {"weights": 1}),
    ((70, 45), (0, 0), 6, 0, {"d": (0.4, 0.3, 0.1, 0.2)}),
    ((70, 45), (0, 0), 8, 1, {"d": (0.3, 0.25, 0.1, 0.2, 0.05, 0.1)}),
    ((70, 45), (0, 0), 8, 0, {"ct_mode": 0, "ct_const": 1e-6}),
    ((70, 45), (0, 0), 6, 1, {"ct_mode": 1}),
]


@pytest.mark.parametrize("shape,bc,K,lim,kw", VARIANTS)
def test_face_flux_parity_scheme_variants(T, orc, shape, bc, K, lim, kw):
    prim = PB.random_state(tuple(reversed(shape)), seed=sum(shape) + 7 * K + lim, jumps=True)
    S, g, so, Uo, Ug = setup(T, orc, shape, bc, K, lim, prim, **kw)
    face_parity_checks(T, orc, S, g, so, Uo, Ug, shape)
    S.close()


def step_switch_region(T, orc, S, g, so, Uo, dto, shape, K, label):
    """Cells that a cutoff decision set by rounding can reach within one SSP-RK3 step: at
    each stage state (the oracle's), the faces whose GPU and oracle flags differ (each
    such difference is checked to be near the cutoff or noise-decided, and counted), their
    neighbour cells, dilated by two stencil half-widths plus one cell per later stage."""
    L0, _ = orc.rhs(g, so, Uo)
    U1 = Uo + dto * L0
    L1, _ = orc.rhs(g, so, U1)
    U2 = 0.75 * Uo + 0.25 * (U1 + dto * L1)
    region = np.zeros(Uo.shape[1:], dtype=bool)
    for st_i, X in enumerate((Uo, U1, U2)):
        Xg = torch.from_numpy(np.ascontiguousarray(X)).cuda()
        sw = []
        for a in range(len(shape)):
            Fg, flg = S.face_dump(Xg, a)
            Fo, flo, cut, noise, bad, scale = orc.faces(g, so, X, a, with_scale=True)
            scale = np.maximum(scale, central_terms(X, a, so.K, g.bc[a]))
            st = compare_faces(Fg.cpu().numpy(), flg.cpu().numpy(), Fo, flo, cut, noise, scale,
                               label="%s stage %d axis %d" % (label, st_i + 1, a))
            bound_counts(st)
            sw.append((flg.cpu().numpy() != flo).reshape(flo.shape[:-2] + (-1,)).any(axis=-1))
        region |= dilate(switch_cells(sw, Uo.shape[1:]), K + 3 - st_i)
    return region


def test_van_albada_steps_match_and_adjoint_is_refused(T, orc):
    """TENO-M-VA through SSP-RK3 steps agrees with the oracle; its adjoint is reported as
    not supported (the Van Albada flux is not a selection among linear forms)."""
    shape = (48, 40)
    prim = PB.random_state((40, 48), seed=21, jumps=True)
    S, g, so, Uo, Ug = setup(T, orc, shape, (0, 0), 6, T.LIM_VA, prim)
    dto = orc.max_dt(g, Uo, 0.4)
    dt = torch.tensor([dto], dtype=torch.float64, device="cuda")
    U1o, _ = orc.rk3_step(g, so, Uo, dto)
    U1g = S.rk3_step(Ug.clone(), dt).cpu().numpy()
    ex = step_switch_region(T, orc, S, g, so, Uo, dto, shape, 6, "VA step")
    assert float(ex.mean()) < 0.1, float(ex.mean())
    compare_cells(U1g, U1o, exclude=ex, rel=1e-13, label="VA step")
    with pytest.raises(T.TenomError) as ei:
        S.rhs_vjp(Ug, Ug.clone())
    assert ei.value.status == T.TENOM_E_UNSUPPORTED
    with pytest.raises(T.TenomError):
        S.rk3_step_adjoint(Ug, dt, Ug.clone())
    with pytest.raises(T.TenomError):
        S.rk3_step_record(Ug.clone(), dt, S.new_tape(linear=True))
    S.close()


@pytest.mark.parametrize("K,lim", [(6, 0), (8, 1), (8, 0)])
def test_rk3_step_and_max_dt_parity(T, orc, K, lim):
    shape = (48, 40)
    prim = PB.random_state((40, 48), seed=5 + K, jumps=True)
    S, g, so, Uo, Ug = setup(T, orc, shape, (0, 0), K, lim, prim)
    dto = orc.max_dt(g, Uo, 0.4)
    dtg = S.max_dt(Ug, 0.4).item()
    assert dtg == pytest.approx(dto, rel=1e-14)
    dt = torch.tensor([dto], dtype=torch.float64, device="cuda")
    U1o, _ = orc.rk3_step(g, so, Uo, dto)
    U1g = S.rk3_step(Ug.clone(), dt).cpu().numpy()
    # cells within reach of a rounding-decided cutoff switch are set aside (counted, at most
    # a tenth of the grid); every other cell agrees to 1e-13
    ex = step_switch_region(T, orc, S, g, so, Uo, dto, shape, K, "rk3 K=%d lim=%d" % (K, lim))
    assert float(ex.mean()) < 0.1, float(ex.mean())
    compare_cells(U1g, U1o, exclude=ex, rel=1e-13, label="rk3 step K=%d lim=%d" % (K, lim))


def c1_oracle_run(orc, n=256, seed=1, K=6, lim=0):
    prim, dx = PB.riemann_1d(n, seed)
    g = orc.make_grid((n,), (dx,), (orc.BC_TRANSMISSIVE,))
    so = orc.make_scheme(K, limiter=lim)
    U0 = orc.init_state(g, prim)
    U, t, steps, bad = orc.advance(g, so, U0, 0.15, 0.4)
    return prim, dx, U, steps


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_riemann_full_run_parity(T, orc, seed):
    """1D seeded Riemann problem, 256 cells, TENO6-MP, to t = 0.15: relative L1 <= 1e-10."""
    prim, dx, Uo, steps = c1_oracle_run(orc, seed=seed)
    S = T.Solver((256,), (dx,), (T.BC_TRANSMISSIVE,), T.make_scheme(6))
    U = S.init_state(torch.from_numpy(prim).cuda())
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    S.advance(U, steps + 2, t_end=0.15, cfl=0.4, t_dev=t)
    assert t.item() == pytest.approx(0.15, rel=1e-14)
    Ug = U.cpu().numpy()
    l1 = np.sum(np.abs(Ug - Uo), axis=1) / np.sum(np.abs(Uo), axis=1)
    assert np.all(l1 <= 1e-10), l1
    assert S.status() == 0


def test_advance_host_matches_device(T, orc):
    """The host-buffer entry point gives the device path's result (and the oracle's)."""
    prim, dx, Uo, steps = c1_oracle_run(orc, seed=4)
    S = T.Solver((256,), (dx,), (T.BC_TRANSMISSIVE,), T.make_scheme(6))
    g = orc.make_grid((256,), (dx,), (orc.BC_TRANSMISSIVE,))
    U0 = orc.init_state(g, prim)
    out = np.zeros_like(U0)
    t = S.advance_host(np.ascontiguousarray(U0), out, t=0.0, t_end=0.15, cfl=0.4, nsteps=steps + 1)
    assert t == pytest.approx(0.15, rel=1e-14)
    l1 = np.sum(np.abs(out - Uo), axis=1) / np.sum(np.abs(Uo), axis=1)
    assert np.all(l1 <= 1e-10), l1


def test_init_state_parity(T, orc):
    prim = PB.random_state((7, 9, 11), 3, jumps=True)
    g = orc.make_grid((11, 9, 7), (0.1, 0.1, 0.1), (0, 0, 0))
    S = T.Solver((11, 9, 7), (0.1, 0.1, 0.1), (0, 0, 0), T.make_scheme(8))
    Ug = S.init_state(torch.from_numpy(prim).cuda()).cpu().numpy()
    np.testing.assert_allclose(Ug, orc.init_state(g, prim), rtol=2e-16, atol=0)


@pytest.mark.parametrize("shape,bc,K", [((4,), (0,), 8), ((1,), (1,), 6), ((5, 1), (0, 1), 6),
                                        ((6, 4, 1), (0, 0, 1), 8)])
def test_degenerate_sizes(T, orc, shape, bc, K):
    """Tiny periodic axes (n = K/2, stencils wrap several times) and single-cell axes."""
    prim = PB.random_state(tuple(reversed(shape)), 9, jumps=False)
    S, g, so, Uo, Ug = setup(T, orc, shape, bc, K, 0, prim)
    for a in range(len(shape)):
        Fg, flg = S.face_dump(Ug, a)
        Fo, flo, cut, noise, bad, scale = orc.faces(g, so, Uo, a, with_scale=True)
        scale = np.maximum(scale, central_terms(Uo, a, so.K, g.bc[a]))
        st = compare_faces(Fg.cpu().numpy(), flg.cpu().numpy(), Fo, flo, cut, noise, scale,
                           label="degenerate %s axis %d" % (shape, a))
        bound_counts(st)


def test_invalid_arguments_rejected(T):
    g = T.make_grid((0,), (0.1,), (0,))
    ctx = T.ctypes.c_void_p()
    s = T.make_scheme(6)
    assert T.lib().tenom_create(T.ctypes.byref(ctx), T.ctypes.byref(g), T.ctypes.byref(s), None) == T.TENOM_E_INVALID
    g = T.make_grid((16,), (0.1,), (0,))
    s.K = 7
    assert T.lib().tenom_create(T.ctypes.byref(ctx), T.ctypes.byref(g), T.ctypes.byref(s), None) == T.TENOM_E_INVALID
    S = T.Solver((16,), (0.1,), (0,), T.make_scheme(6))
    with pytest.raises(T.TenomError):
        S.face_dump(S.tensor(), 1)


def test_nonphysical_state_sets_status_word(T):
    """A negative pressure in the input is reported through the sticky status word (the
    kernels do not trap)."""
    n = 64
    prim = np.ones((3, n))
    prim[1] = 0.0
    prim[2, 10] = -0.5
    S = T.Solver((n,), (1.0 / n,), (T.BC_PERIODIC,), T.make_scheme(6))
    U = S.init_state(torch.from_numpy(prim).cuda())
    S.rhs(U)
    torch.cuda.synchronize()
    st = S.status(reset=True)
    assert st & T.ST_P
    assert S.status() == 0


def sample_faces(rng, shape, axis, m):
    """m random face multi-indices (x, y, z) of an axis."""
    idx = np.zeros((m, 3), dtype=np.int32)
    for a, n in enumerate(shape):
        hi = n + 1 if a == axis else n
        idx[:, a] = rng.integers(0, hi, m)
    return idx


def check_sampled(T, orc, S, g, so, Ug, Uo, shape, m, seed, label="", smooth=False):
    rng = np.random.default_rng(seed)
    for a in range(len(shape)):
        Fg, flg = S.face_dump(Ug, a)
        Fg = Fg.cpu().numpy()
        flg = flg.cpu().numpy()
        idx = sample_faces(rng, shape, a, m)
        Fo, flo, cut, noise, bad, scale = orc.faces_at(g, so, Uo, a, idx, with_scale=True)
        scale = np.maximum(scale.T, central_terms_at(Uo, a, so.K, g.bc[a], idx)).T
        sel = tuple(idx[:, d] for d in reversed(range(len(shape))))
        Fgs = np.stack([Fg[v][sel] for v in range(len(shape) + 2)])
        st = compare_faces(Fgs, flg[sel], Fo.T, flo, cut, noise, scale.T, label="%s sampled axis %d" % (label, a))
        bound_counts(st)
        if smooth:  # no characteristic field of these smooth-plus-jump fields is flat to rounding
            assert st["noise_faces"] == 0, st
        # the face fluxes of all faces must be finite
        assert np.isfinite(Fg).all()
        del Fg, flg


def test_full_size_2d_sampled(T, orc):
    """2048^2 broadband field with circular jumps (TENO6-MP and TENO8-TVD5) at full size,
    in the bench's launch configuration: 4000 sampled faces per axis against the oracle."""
    prim, dx = PB.broadband_2d(2048, 2)
    for K, lim in ((6, 0), (8, 1)):
        S, g, so, Uo, Ug = setup(T, orc, (2048, 2048), (0, 0), K, lim, prim, dx=(dx, dx))
        check_sampled(T, orc, S, g, so, Ug, Uo, (2048, 2048), 4000, K, label="broadband 2048^2 K=%d" % K,
                      smooth=True)
        S.close()


def test_full_size_3d_sampled(T, orc):
    """256^3 solenoidal field (TENO8-MP) at full size: 3000 sampled faces per axis."""
    prim, dx = PB.solenoidal_3d(256, 3)
    S, g, so, Uo, Ug = setup(T, orc, (256, 256, 256), (0, 0, 0), 8, 0, prim, dx=(dx, dx, dx))
    del prim
    check_sampled(T, orc, S, g, so, Ug, Uo, (256, 256, 256), 3000, 3, label="solenoidal 256^3", smooth=True)


FILTER_CASES = [
    ("random", (300,), (1,), 6, 0), ("random", (300,), (0,), 8, 1), ("random", (70, 45), (1, 0), 8, 0),
    ("random", (20, 13, 11), (0, 1, 0), 6, 1), ("random", (33, 40), (0, 0), 8, 1),
    ("broadband", (2048, 2048), (0, 0), 6, 0), ("broadband", (2048, 2048), (0, 0), 8, 1),
    ("solenoidal", (96, 96, 96), (0, 0, 0), 8, 0),
]


@pytest.mark.parametrize("kind,shape,bc,K,lim", FILTER_CASES)
def test_certified_fp32_cutoff_filter_equals_fp64_decisions(T, kind, shape, bc, K, lim):
    """The cutoff decisions taken through the certified FP32 filter (default) are identical to
    FP64-only decisions, and so are the face fluxes, bit for bit."""
    if kind == "random":
        prim = PB.random_state(tuple(reversed(shape)), seed=sum(shape) + 3 * K + lim, jumps=True)
        dx = tuple(1.0 / n for n in shape)
    elif kind == "broadband":
        prim, h = PB.broadband_2d(shape[0], 2)
        dx = (h, h)
    else:
        prim, h = PB.solenoidal_3d(shape[0], 3)
        dx = (h, h, h)
    S1 = T.Solver(shape, dx, bc, T.make_scheme(K, limiter=lim))
    S2 = T.Solver(shape, dx, bc, T.make_scheme(K, limiter=lim, decisions=T.DECIDE_FP64))
    U = S1.init_state(torch.from_numpy(prim).cuda())
    for a in range(len(shape)):
        F1, f1 = S1.face_dump(U, a)
        F2, f2 = S2.face_dump(U, a)
        assert torch.equal(f1, f2), int((f1 != f2).sum())
        assert torch.equal(F1, F2)
    S1.close()
    S2.close()


def test_taylor_green_parity_and_conservation(T, orc):
    """Inviscid Taylor-Green vortex (Eq. TGV) at 16^3, TENO8A-M-MP: face fluxes and flags of
    every axis agree with the oracle (the symmetric field makes many characteristic
    stencils flat, so many cutoff decisions are set by rounding: those are the
    noise-decided faces of the parity rules); over 40 GPU steps mass, momentum and energy
    sums stay at rounding level (flux form, periodic) and the kinetic energy stays bounded
    by its initial value (no exchange beyond the weak pressure work of this low-Mach flow)."""
    n = 16
    prim, dx = PB.taylor_green_3d(n)
    shape = (n, n, n)
    S, g, so, Uo, Ug = setup(T, orc, shape, (0, 0, 0), 8, 0, prim, dx=(dx, dx, dx))
    for a in range(3):
        Fg, flg = S.face_dump(Ug, a)
        Fo, flo, cut, noise, bad, scale = orc.faces(g, so, Uo, a, with_scale=True)
        scale = np.maximum(scale, central_terms(Uo, a, so.K, g.bc[a]))
        assert bad == 0
        # the symmetric field makes face values vanish exactly on its symmetry planes, where
        # both sides return rounding noise of terms that cancel before the back-projection:
        # these faces are measured against 1e-3 of the component's largest value
        st = compare_faces(Fg.cpu().numpy(), flg.cpu().numpy(), Fo, flo, cut, noise, scale, label="TGV axis %d" % a,
                           floor=True)
        bound_counts(st, noise_frac=0.1, floor=True)
    dt = S.max_dt(Ug, 0.4)
    U = Ug.clone()
    ke = lambda X: float((0.5 * (X[1] ** 2 + X[2] ** 2 + X[3] ** 2) / X[0]).sum())
    tot0, ke0 = U.sum(dim=(1, 2, 3)), ke(U)
    for _ in range(40):
        S.rk3_step(U, dt)
    scale = U.abs().sum(dim=(1, 2, 3))
    assert float(((U.sum(dim=(1, 2, 3)) - tot0).abs() / scale).max()) < 1e-13
    assert ke(U) <= ke0 * (1 + 1e-3)
    assert S.status() == 0


STATS_CASES = [((70, 45), (0, 0), 6, 0), ((70, 45), (1, 0), 8, 1), ((20, 13, 11), (0, 0, 1), 8, 0),
               ((300,), (1,), 6, 0), ((64, 48), (0, 0), 6, 2)]


@pytest.mark.parametrize("shape,bc,K,lim", STATS_CASES)
def test_decision_stats_match_oracle(T, orc, shape, bc, K, lim):
    """The logging pass (tenom_decision_stats) counts what the oracle decides: per split side
    the nonsmooth candidates per k (Eq. cut-off), the all-smooth sides, the adaptive [beta]
    histogram (Eq. cut-off_adjust) and the near-cutoff sides, equal to the oracle's counts
    up to the sides whose decision the parity rules excuse (near the cutoff or set by
    rounding); the limiter's sides and changes are consistent with them."""
    prim = PB.random_state(tuple(reversed(shape)), seed=sum(shape) + 11 * K + lim, jumps=True)
    S, g, so, Uo, Ug = setup(T, orc, shape, bc, K, lim, prim)
    for a in range(len(shape)):
        cnt = S.decision_stats(Ug, a)
        c = T.stats_dict(cnt.cpu().numpy(), K)
        Fo, flo, cut, noise, bad, scale = orc.faces(g, so, Uo, a, with_scale=True)
        scale = np.maximum(scale, central_terms(Uo, a, so.K, g.bc[a]))
        fl = flo.reshape(-1).astype(np.int64)
        cu, no = cut.reshape(-1), noise.reshape(-1)
        excused = int(((cu <= CUT_TOL) | (cu <= NOISE_K * no)).sum())
        assert c["sides"] == fl.size
        bits = fl & 63
        total_ns = 0
        for k in range(K - 2):
            o = int((((bits >> k) & 1) == 0).sum())
            assert abs(c["nonsmooth_k%d" % k] - o) <= excused, (k, c, o, excused)
            total_ns += c["nonsmooth_k%d" % k]
        assert total_ns > 0  # the jumps make some candidates nonsmooth
        allsm = int((bits == (1 << (K - 2)) - 1).sum())
        assert abs(c["all_smooth"] - allsm) <= excused, (c, allsm)
        assert c["limited_sides"] == c["sides"] - c["all_smooth"]
        assert 0 < c["limiter_changed"] <= total_ns
        assert c["certified"] > 0.25 * c["sides"] and c["certified_disagree"] <= excused
        if K == 8:
            hist = [int((((fl >> 6) & 3) == j).sum()) for j in range(4)]
            for j in range(4):
                assert abs(c["ct_exp_%d" % (7 + j)] - hist[j]) <= excused, (c, hist)
        near = int((cu <= CUT_TOL).sum())
        assert abs(c["near_cutoff_sides"] + c["near_integer_beta"] - near) <= 1 + near, (c, near)
        assert c["nonfinite"] == 0
    # the counters add up over calls
    cnt = S.decision_stats(Ug, 0)
    S.decision_stats(Ug, 0, counters=cnt)
    c2 = T.stats_dict(cnt.cpu().numpy(), K)
    c1 = T.stats_dict(S.decision_stats(Ug, 0).cpu().numpy(), K)
    assert all(c2[k] == 2 * c1[k] for k in c1)
    S.close()
