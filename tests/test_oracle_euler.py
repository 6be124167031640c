"""Pins of the oracle's Euler layer (characteristic decomposition, LLF splitting,
conservative difference, SSP-RK3; Section 4) against mathematics and the paper's
test problems.  CPU only."""
import numpy as np
import pytest

from conftest import read_golden
from paper_2010_13289_gb300 import problems as PB


def grid1(orc, n, dx, bc=None):
    return orc.make_grid((n,), (dx,), (orc.BC_TRANSMISSIVE if bc is None else bc,))


def rand_U(orc, g, rng):
    nv = g.dim + 2
    prim = np.empty(nv)
    prim[0] = rng.uniform(0.2, 2.0)
    prim[1:nv - 1] = rng.uniform(-1, 1, nv - 2)
    prim[nv - 1] = rng.uniform(0.2, 2.0)
    G1 = orc.make_grid((1,) * g.dim, (1.0,) * g.dim, (0,) * g.dim, g.gamma)
    return orc.init_state(G1, prim.reshape((nv,) + (1,) * g.dim)).ravel()


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_left_right_eigenvectors_inverse_and_roe_property(orc, dim):
    """L = R^{-1}, and the Roe matrix A = R diag(lambda) L satisfies
    A (U_R - U_L) = F(U_R) - F(U_L) (Roe's defining property, Section 4)."""
    g = orc.make_grid((4,) * dim, (1.0,) * dim, (0,) * dim)
    rng = np.random.default_rng(dim)
    for _ in range(10):
        UL, UR = rand_U(orc, g, rng), rand_U(orc, g, rng)
        for a in range(dim):
            R, L = orc.roe_eigen(g, UL, UR, a)
            np.testing.assert_allclose(L @ R, np.eye(dim + 2), atol=1e-13)
            # eigenvalues from the Roe state: (u-c, u, .., u, u+c)
            sL, sR = np.sqrt(UL[0]), np.sqrt(UR[0])
            uL, uR = UL[1:dim + 1] / UL[0], UR[1:dim + 1] / UR[0]
            pL = 0.4 * (UL[-1] - 0.5 * UL[0] * uL @ uL)
            pR = 0.4 * (UR[-1] - 0.5 * UR[0] * uR @ uR)
            HL, HR = (UL[-1] + pL) / UL[0], (UR[-1] + pR) / UR[0]
            u = (sL * uL + sR * uR) / (sL + sR)
            H = (sL * HL + sR * HR) / (sL + sR)
            c = np.sqrt(0.4 * (H - 0.5 * u @ u))
            lam = np.full(dim + 2, u[a])
            lam[0] -= c
            lam[-1] += c
            A = R @ np.diag(lam) @ L
            dF = orc.phys_flux(g, UR, a) - orc.phys_flux(g, UL, a)
            np.testing.assert_allclose(A @ (UR - UL), dF, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("dim,K", [(1, 6), (2, 8), (3, 6)])
def test_uniform_state_flux_is_physical_flux(orc, dim, K):
    """Consistency: on a uniform state the LLF halves add to G (f+ + f- = f) and the
    back-projection returns the physical flux exactly (to rounding)."""
    n = 6
    g = orc.make_grid((n,) * dim, (0.1,) * dim, (0,) * dim)
    rng = np.random.default_rng(5)
    U1 = rand_U(orc, g, rng)
    U = np.empty((dim + 2,) + (n,) * dim)
    for q in range(dim + 2):
        U[q] = U1[q]
    S = orc.make_scheme(K)
    for a in range(dim):
        F, fl, _, _, bad = orc.faces(g, S, U, a)
        assert bad == 0
        want = orc.phys_flux(g, U1, a)
        for q in range(dim + 2):
            np.testing.assert_allclose(F[q], want[q], rtol=1e-13, atol=1e-14)
        rhs, _ = orc.rhs(g, S, U)
        assert np.max(np.abs(rhs)) < 1e-12


def state2d(orc, n, seed, jumps=True):
    prim = PB.random_state((n, n), seed, jumps)
    g = orc.make_grid((n, n), (1.0 / n, 1.0 / n), (0, 0))
    return g, orc.init_state(g, prim)


@pytest.mark.parametrize("K,lim", [(6, 0), (8, 1)])
def test_periodic_conservation(orc, K, lim):
    """Eq. approximateEq in flux form: with periodic boundaries sum_i U_i is conserved by
    every RK3 step up to rounding."""
    g, U = state2d(orc, 24, 3)
    S = orc.make_scheme(K, limiter=lim)
    tot0 = U.reshape(4, -1).sum(axis=1)
    dt = orc.max_dt(g, U, 0.4)
    U1, bad = orc.rk3_step(g, S, U, dt)
    assert bad == 0
    tot1 = U1.reshape(4, -1).sum(axis=1)
    scale = np.abs(U).reshape(4, -1).sum(axis=1)
    assert np.all(np.abs(tot1 - tot0) <= 1e-14 * scale)


def test_transmissive_conservation_is_boundary_flux(orc):
    """Transmissive boundaries: d/dt sum_i U_i dx = F_{1/2} - F_{N+1/2} exactly."""
    prim, dx = PB.riemann_1d(64, 1)
    g = grid1(orc, 64, dx)
    U = orc.init_state(g, prim)
    S = orc.make_scheme(6)
    r, _ = orc.rhs(g, S, U)
    F, _, _, _, _ = orc.faces(g, S, U, 0)
    np.testing.assert_allclose(r.sum(axis=1) * dx, F[:, 0] - F[:, -1], rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("K,lim", [(6, 0), (8, 0), (6, 1)])
def test_mirror_symmetry(orc, K, lim):
    """x -> -x, u -> -u maps solutions to solutions: the mirrored initial state gives the
    mirrored state after several RK3 steps (the f- side is the mirrored f+ stencil)."""
    prim, dx = PB.riemann_1d(64, 7)
    g = grid1(orc, 64, dx)
    S = orc.make_scheme(K, limiter=lim)
    U = orc.init_state(g, prim)
    Um = U[:, ::-1].copy()
    Um[1] *= -1
    for _ in range(5):
        dt = orc.max_dt(g, U, 0.4)
        U, _ = orc.rk3_step(g, S, U, dt)
        Um, _ = orc.rk3_step(g, S, Um, dt)
    back = Um[:, ::-1].copy()
    back[1] *= -1
    np.testing.assert_allclose(back, U, rtol=1e-12, atol=1e-13)


def test_dimension_consistency_and_rotation(orc):
    """2D data uniform in y reproduces the 1D result (x-momentum and energy) and a 90 degree
    rotation of the data permutes the result (dimension-by-dimension, Section 4)."""
    n = 32
    prim1, dx = PB.riemann_1d(n, 11)
    S = orc.make_scheme(6)
    g1 = orc.make_grid((n,), (dx,), (orc.BC_PERIODIC,))
    U1 = orc.init_state(g1, prim1)
    r1, _ = orc.rhs(g1, S, U1)
    ny = 8
    prim2 = np.zeros((4, ny, n))
    prim2[0] = prim1[0]
    prim2[1] = prim1[1]
    prim2[3] = prim1[2]
    g2 = orc.make_grid((n, ny), (dx, 0.1), (0, 0))
    U2 = orc.init_state(g2, prim2)
    r2, _ = orc.rhs(g2, S, U2)
    for j in range(ny):
        np.testing.assert_allclose(r2[0, j], r1[0], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(r2[1, j], r1[1], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(r2[3, j], r1[2], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(r2[2, j], 0.0, atol=1e-12)
    # rotation: swap the roles of x and y
    g, U = state2d(orc, 16, 19)
    rA, _ = orc.rhs(g, S, U)
    Ut = np.stack([U[0].T, U[2].T, U[1].T, U[3].T])
    rB, _ = orc.rhs(g, S, Ut)
    back = np.stack([rB[0].T, rB[2].T, rB[1].T, rB[3].T])
    np.testing.assert_allclose(back, rA, rtol=1e-11, atol=1e-11)


def test_exact_riemann_wave_relations(orc):
    """The exact solver's waves satisfy the Rankine-Hugoniot conditions (shocks), keep the
    Riemann invariant u + 2c/(g-1) (left fan) constant, and have continuous p and u at
    the contact; checked on the seeded states and the printed Lax/Sod states."""
    gam = 1.4
    cases = [PB.riemann_states(s) for s in range(1, 9)]
    for row in read_golden("shock_tubes.txt"):
        v = [float(x) for x in row[1:7]]
        cases.append(((v[0], v[1], v[2]), (v[3], v[4], v[5])))
    xi = np.linspace(-6, 6, 24001)
    for L, R in cases:
        rho, u, p, star = orc.exact_riemann(L, R, gam, xi)
        ps, us = star
        E = p / (gam - 1) + 0.5 * rho * u * u
        # far field
        assert rho[0] == L[0] and rho[-1] == R[0]
        # contact: pressure and velocity equal on both sides
        il = np.searchsorted(xi, us) - 5
        ir = np.searchsorted(xi, us) + 5
        assert p[il] == pytest.approx(ps) and p[ir] == pytest.approx(ps)
        assert u[il] == pytest.approx(us) and u[ir] == pytest.approx(us)
        for side, far, idx in (("L", L, il), ("R", R, ir)):
            if ps > far[2]:
                # shock: mass, momentum, energy fluxes conserved in the shock frame
                rs = rho[idx]
                Es = ps / (gam - 1) + 0.5 * rs * us * us
                Ef = far[2] / (gam - 1) + 0.5 * far[0] * far[1] ** 2
                Ssh = (rs * us - far[0] * far[1]) / (rs - far[0])
                m1 = rs * (us - Ssh) - far[0] * (far[1] - Ssh)
                m2 = (rs * us * us + ps - Ssh * rs * us) - (far[0] * far[1] ** 2 + far[2] - Ssh * far[0] * far[1])
                m3 = ((Es + ps) * us - Ssh * Es) - ((Ef + far[2]) * far[1] - Ssh * Ef)
                assert abs(m2) < 1e-10 * (1 + ps) and abs(m3) < 1e-10 * (1 + Es)
                assert abs(m1) < 1e-10
            else:
                # rarefaction: isentropic, Riemann invariant constant through the fan
                assert p[idx] / rho[idx] ** gam == pytest.approx(far[2] / far[0] ** gam, rel=1e-10)
        c = np.sqrt(gam * p / rho)
        fan = (xi < us) & (p < L[2]) & (p > ps) if ps < L[2] else np.zeros_like(xi, bool)
        if fan.any():
            inv = u[fan] + 2 * c[fan] / (gam - 1)
            assert np.allclose(inv, L[1] + 2 * np.sqrt(gam * L[2] / L[0]) / (gam - 1), rtol=1e-12)


def shock_tube_error(orc, n, L, R, t_end, K=6, lim=0):
    """Run on the extended domain [-1, 2] (transmissive) so no wave reaches a boundary and
    return the L1 errors of rho, u, p against the exact solution on [0, 1]."""
    x0, x1 = -1.0, 2.0
    N = 3 * n
    prim, dx = PB.riemann_1d(N, 0, x0=x0, x1=x1, xc=0.5, states=(L, R))
    g = grid1(orc, N, dx)
    S = orc.make_scheme(K, limiter=lim)
    U, t, steps, bad = orc.advance(g, S, orc.init_state(g, prim), t_end, 0.4)
    assert bad == 0 and t == pytest.approx(t_end)
    x = x0 + (np.arange(N) + 0.5) * dx
    inside = (x > 0) & (x < 1)
    rho_e, u_e, p_e, _ = orc.exact_riemann(L, R, 1.4, (x[inside] - 0.5) / t_end)
    rho = U[0, inside]
    u = U[1, inside] / rho
    p = 0.4 * (U[2, inside] - 0.5 * rho * u * u)
    return np.array([np.mean(np.abs(rho - rho_e)), np.mean(np.abs(u - u_e)), np.mean(np.abs(p - p_e))])


@pytest.mark.parametrize("name", ["sod", "lax"])
def test_shock_tubes_converge_to_exact(orc, name):
    """Section 4.2.1 shock tubes: the TENO6-M-MP solution approaches the exact Riemann
    solution under refinement (L1 error of rho, u, p decreasing 100 -> 200 -> 400)."""
    row = [r for r in read_golden("shock_tubes.txt") if r[0] == name][0]
    v = [float(x) for x in row[1:]]
    L, R, t_end = tuple(v[0:3]), tuple(v[3:6]), v[6]
    errs = [shock_tube_error(orc, n, L, R, t_end) for n in (100, 200, 400)]
    assert np.all(errs[1] < errs[0]) and np.all(errs[2] < errs[1]), errs
    assert errs[0][0] < 0.02


@pytest.mark.slow
def test_seeded_riemann_converges(orc):
    """The 256-cell seeded shock-tube workload (seed 1) versus the exact solution:
    error decreases under 128 -> 256 -> 512."""
    L, R = PB.riemann_states(1)
    errs = [shock_tube_error(orc, n, L, R, 0.15) for n in (128, 256, 512)]
    assert np.all(errs[1] < errs[0]) and np.all(errs[2] < errs[1]), errs


@pytest.mark.parametrize("K,expect", [(6, 6.0), (8, 8.0)])
def test_spatial_order_gaussian_pulse(orc, K, expect):
    """Section 4.1.1 (Gaussian pulse, u_t + u_x = 0, periodic): the error of the spatial
    operator -(f_{i+1/2} - f_{i-1/2})/dx against -u'(x_i) converges at the design order
    K (all stencils smooth, Section 3.3)."""
    S = orc.make_scheme(K)
    errs, ns = [], [160, 320, 640]
    for n in ns:
        u, dx = PB.gaussian_pulse(n)
        x = (np.arange(n) + 0.5) * dx
        r = orc.scalar_rhs(S, u, dx)
        exact = 600.0 * (x - 0.5) * u
        errs.append(np.max(np.abs(r - exact)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > expect - 0.6), orders


def test_gaussian_pulse_time_integrated_order(orc):
    """Gaussian pulse to t = 1 with SSP-RK3 and dt ~ dx^2 so the time error is below the
    spatial one: L_inf error decreases at (at least) close to 6th order for TENO6-M."""
    S = orc.make_scheme(6)
    errs = []
    for n in (80, 160):
        u0, dx = PB.gaussian_pulse(n)
        nsteps = int(np.ceil(1.0 / (0.4 * dx * dx * 20)))
        dt = 1.0 / nsteps
        u = orc.scalar_advance(S, u0, dx, dt, nsteps)
        errs.append(np.max(np.abs(u - u0)))
    assert np.log2(errs[0] / errs[1]) > 5.0, errs


def test_euler_entropy_wave_order(orc):
    """Smooth advected entropy wave of the Euler equations (rho = 1 + 0.2 sin, u = p = 1):
    the spatial operator's error in d(rho)/dt converges at order 6 through the whole
    characteristic path."""
    S = orc.make_scheme(6)
    errs = []
    for n in (64, 128, 256):
        prim, dx = PB.smooth_1d(n, 3)
        g = grid1(orc, n, dx, orc.BC_PERIODIC)
        U = orc.init_state(g, prim)
        r, _ = orc.rhs(g, S, U)
        x = (np.arange(n) + 0.5) * dx
        rng = np.random.default_rng(3)
        phi = rng.uniform(0, 2 * np.pi)
        exact = -0.2 * 2 * np.pi * np.cos(2 * np.pi * x + phi)
        errs.append(np.max(np.abs(r[0] - exact)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 5.4), orders


def square_wave(n):
    x = (np.arange(n) + 0.5) / n
    return np.where((x > 0.3) & (x < 0.6), 1.0, 0.0), 1.0 / n


def test_mp_no_new_extrema(orc):
    """Section 3.2.2: with every candidate limited (forced delta = 0) and CFL <= 1/(1+alpha)
    the MP scheme creates no new extrema on a square wave (Suresh-Huynh)."""
    S = orc.make_scheme(6, ct_const=2.0)
    u, dx = square_wave(100)
    dt = 0.4 * dx
    for _ in range(30):
        u = orc.scalar_advance(S, u, dx, dt, 1)
        assert u.max() <= 1.0 + 1e-13 and u.min() >= -1e-13


def test_tvd5_total_variation_diminishing(orc):
    """Section 3.2.1: forced delta = 0 turns TENO-M-TVD5 into the high-order TVD scheme;
    its total variation does not grow at CFL 0.4."""
    S = orc.make_scheme(6, limiter=1, ct_const=2.0)
    rng = np.random.default_rng(47)
    u = np.cumsum(rng.normal(size=120)) * 0.1
    u = np.concatenate([u, u[::-1]])
    dx = 1.0 / u.size
    tv = np.sum(np.abs(np.diff(np.concatenate([u, u[:1]]))))
    for _ in range(20):
        u = orc.scalar_advance(S, u, dx, 0.4 * dx, 1)
        tv1 = np.sum(np.abs(np.diff(np.concatenate([u, u[:1]]))))
        assert tv1 <= tv * (1 + 1e-13)
        tv = tv1


def test_teno_m_removes_overshoot_that_teno_keeps(orc):
    """Section 4.1.2 (half-ellipse): TENO-M-MP stays within the data bounds on a
    square wave where plain TENO6 with renormalised weights may not (qualitative claim;
    here we check TENO-M-MP only)."""
    S = orc.make_scheme(6)
    u, dx = square_wave(200)
    for _ in range(50):
        u = orc.scalar_advance(S, u, dx, 0.4 * dx, 1)
    assert u.max() <= 1.0 + 1e-3 and u.min() >= -1e-3


def test_jvp_matches_central_differences(orc):
    """The dual-number oracle (branches frozen) equals central finite differences of the
    plain oracle on smooth data (where no branch switches under the perturbation)."""
    n = 32
    prim = PB.random_state((n,), 5, jumps=False)  # every characteristic field varies
    g = grid1(orc, n, 1.0 / n, orc.BC_PERIODIC)
    rng = np.random.default_rng(1)
    for K in (6, 8):
        S = orc.make_scheme(K)
        U = orc.init_state(g, prim)
        dt = orc.max_dt(g, U, 0.4)
        v = rng.normal(size=U.shape)
        _, jv, _ = orc.rk3_step_jvp(g, S, U, v, dt)
        eps = 1e-6
        fl0 = orc.faces(g, S, U, 0)[1]
        for sgn in (1, -1):  # no branch switches inside the FD stencil
            assert np.array_equal(orc.faces(g, S, U + sgn * eps * v, 0)[1], fl0)
        up, _ = orc.rk3_step(g, S, U + eps * v, dt)
        um, _ = orc.rk3_step(g, S, U - eps * v, dt)
        fd = (up - um) / (2 * eps)
        assert np.max(np.abs(fd - jv)) < 1e-8 * np.max(np.abs(jv))


def test_flop_counter(orc):
    """The op-counting run visits every face: per-face count is identical for identical
    smooth faces and positive."""
    n = 16
    g = orc.make_grid((n,), (1.0 / n,), (orc.BC_PERIODIC,))
    U = np.zeros((3, n))
    U[0] = 1.0
    U[2] = 2.5
    S = orc.make_scheme(6)
    tot = orc.face_flops(g, S, U, 0)
    assert tot > 0 and tot % (n + 1) == 0
