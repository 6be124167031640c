"""Parity of the CUDA path (through the C ABI) with the CPU oracle on identical seeded
inputs.  Runs on a GB300 (-m gpu)."""
import math

import numpy as np
import pytest

from paper_2010_13289_gb300 import problems as PB
from parity import compare_faces, compare_rhs, switch_cells

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
        assert bad == 0
        st = compare_faces(Fg.cpu().numpy(), flg.cpu().numpy(), Fo, flo, cut, noise, scale,
                           label="%s axis %d" % (shape, a))
        # near-cutoff switches are rare; noise-decided ones sit where a characteristic field
        # is flat to rounding (transmissive ghost copies, degenerate fields)
        assert st["near_cutoff_faces"] <= max(2, 0.01 * st["faces"]), st
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
        assert bad == 0
        st = compare_faces(Fg.cpu().numpy(), flg.cpu().numpy(), Fo, flo, cut, noise, scale,
                           label="%s axis %d" % (shape, a))
        assert st["near_cutoff_faces"] <= max(2, 0.01 * st["faces"]), st
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
    err = np.abs(U1g - U1o) / np.maximum(np.abs(U1o), 1e-3 * np.abs(U1o).max(axis=(1, 2), keepdims=True))
    assert float(np.mean(err > 1e-12)) < 0.01 and np.median(err) < 1e-15
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
    err = np.abs(U1g - U1o) / np.maximum(np.abs(U1o), 1e-3 * np.abs(U1o).max(axis=(1, 2), keepdims=True))
    # a rare cutoff switch changes a few cells by more; everything else agrees to 1e-12
    frac_bad = float(np.mean(err > 1e-12))
    assert frac_bad < 0.01, (frac_bad, err.max())
    assert np.median(err) < 1e-15


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
        compare_faces(Fg.cpu().numpy(), flg.cpu().numpy(), Fo, flo, cut, noise, scale, label="%s" % (shape,))


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


def check_sampled(T, orc, S, g, so, Ug, Uo, shape, m, seed):
    rng = np.random.default_rng(seed)
    for a in range(len(shape)):
        Fg, flg = S.face_dump(Ug, a)
        Fg = Fg.cpu().numpy()
        flg = flg.cpu().numpy()
        idx = sample_faces(rng, shape, a, m)
        Fo, flo, cut, noise, bad, scale = orc.faces_at(g, so, Uo, a, idx, with_scale=True)
        sel = tuple(idx[:, d] for d in reversed(range(len(shape))))
        Fgs = np.stack([Fg[v][sel] for v in range(len(shape) + 2)])
        compare_faces(Fgs, flg[sel], Fo.T, flo, cut, noise, scale.T, label="sampled axis %d" % a)
        # the face fluxes of all faces must be finite
        assert np.isfinite(Fg).all()
        del Fg, flg


def test_full_size_2d_sampled(T, orc):
    """2048^2 broadband field with circular jumps (TENO6-MP and TENO8-TVD5) at full size,
    in the bench's launch configuration: 4000 sampled faces per axis against the oracle."""
    prim, dx = PB.broadband_2d(2048, 2)
    for K, lim in ((6, 0), (8, 1)):
        S, g, so, Uo, Ug = setup(T, orc, (2048, 2048), (0, 0), K, lim, prim, dx=(dx, dx))
        check_sampled(T, orc, S, g, so, Ug, Uo, (2048, 2048), 4000, K)
        S.close()


def test_full_size_3d_sampled(T, orc):
    """256^3 solenoidal field (TENO8-MP) at full size: 3000 sampled faces per axis."""
    prim, dx = PB.solenoidal_3d(256, 3)
    S, g, so, Uo, Ug = setup(T, orc, (256, 256, 256), (0, 0, 0), 8, 0, prim, dx=(dx, dx, dx))
    del prim
    check_sampled(T, orc, S, g, so, Ug, Uo, (256, 256, 256), 3000, 3)


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
        assert bad == 0
        compare_faces(Fg.cpu().numpy(), flg.cpu().numpy(), Fo, flo, cut, noise, scale, label="TGV axis %d" % a)
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
