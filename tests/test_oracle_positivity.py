"""Pins of the oracle's positivity-preserving flux limiter (Section 4.4, which applies the
limiter of Hu, Adams & Shu 2013) against what its definition and the mathematics fix:
it leaves admissible steps untouched, its flux lies on the segment between the first-order
Lax-Friedrichs flux and the high-order flux, the one-sided states it is built on keep
density and pressure at or above the floor, and with it TENO8-MP runs the Le Blanc problem
to t = 6 close to the exact Riemann solution, where without it the run breaks down.  CPU
only.  The Euler flux and the Lax-Friedrichs flux are written out here in numpy, from
their textbook definitions, independently of the oracle."""
import numpy as np
import pytest

from paper_2010_13289_gb300 import problems as PB

EPS = 1e-13


def euler_flux(U, a, gamma):
    """Physical flux along axis a of conserved states U[nv, ...], with |u_a| + c."""
    D = U.shape[0] - 2
    rho = U[0]
    vel = U[1:1 + D] / rho
    p = (gamma - 1.0) * (U[-1] - 0.5 * rho * (vel ** 2).sum(0))
    F = np.empty_like(U)
    F[0] = U[1 + a]
    for d in range(D):
        F[1 + d] = U[1 + d] * vel[a] + (p if d == a else 0.0)
    F[-1] = (U[-1] + p) * vel[a]
    return F, np.abs(vel[a]) + np.sqrt(gamma * p / rho)


def pressure(W, gamma):
    D = W.shape[0] - 2
    return (gamma - 1.0) * (W[-1] - 0.5 * (W[1:1 + D] ** 2).sum(0) / W[0])


def face_neighbours(U, a, n, periodic):
    """States left and right of every face of axis a (face f between cells f-1 and f)."""
    ax = U.ndim - 1 - a
    left = np.arange(-1, n) % n if periodic else np.clip(np.arange(-1, n), 0, n - 1)
    right = np.arange(0, n + 1) % n if periodic else np.clip(np.arange(0, n + 1), 0, n - 1)
    return np.take(U, left, axis=ax), np.take(U, right, axis=ax)


def evolved_states(orc, shape, seed, steps, bc=None):
    """Seeded near-vacuum state advanced `steps` limited SSP-RK3 steps (CFL 0.4): states
    on which the limiter is active."""
    D = len(shape)
    bc = orc.BC_PERIODIC if bc is None else bc
    g = orc.make_grid(tuple(reversed(shape)), (0.1,) * D, (bc,) * D, gamma=1.4)
    s = orc.make_scheme(6, orc.LIM_MP, positivity=1)
    U = orc.init_state(g, PB.near_vacuum(shape, seed))
    out = []
    for _ in range(steps):
        dt = orc.max_dt(g, U, 0.4)
        out.append((U.copy(), dt))
        U, _ = orc.rk3_step(g, s, U, dt)
    return g, s, out


@pytest.mark.parametrize("shape,seed,periodic", [((128,), 1, True), ((24, 20), 0, True), ((10, 12, 8), 2, True),
                                                  ((128,), 3, False), ((24, 20), 4, False)])
def test_limited_flux_on_segment_and_one_sided_states_admissible(orc, shape, seed, periodic):
    """Per face: F = F^LF + theta (F^H - F^LF) with one theta in [0, 1]; the one-sided
    states U_L - mu F and U_R + mu F (mu = 2 D dt/dx) keep density and pressure at or above
    min(1e-13, the value with F^LF); theta < 1 only where F^H itself breaks that floor.
    On transmissive grids the cell outside a boundary face is the edge cell's copy."""
    D = len(shape)
    g, s, states = evolved_states(orc, shape, seed, 6, None if periodic else orc.BC_TRANSMISSIVE)
    nlim = 0
    for U, dt in states:
        for a in range(D):
            n = shape[D - 1 - a]
            FH = orc.faces(g, s, U, a)[0]
            F, _ = orc.faces_limited(g, s, U, a, dt)
            UL, UR = face_neighbours(U, a, n, periodic)
            FLl, sl = euler_flux(UL, a, g.gamma)
            FLr, sr = euler_flux(UR, a, g.gamma)
            FLF = 0.5 * (FLl + FLr - np.maximum(sl, sr) * (UR - UL))
            mu = 2.0 * D * dt / 0.1
            changed = np.any(F != FH, axis=0)
            nlim += changed.sum()
            # one theta per face, in [0, 1]
            dH = FH - FLF
            k = np.argmax(np.abs(dH), axis=0)
            den = np.take_along_axis(dH, k[None], 0)[0]
            num = np.take_along_axis(F - FLF, k[None], 0)[0]
            theta = np.where(den != 0.0, num / np.where(den != 0.0, den, 1.0), 1.0)
            assert np.all(theta[changed] >= -1e-9) and np.all(theta[changed] <= 1.0 + 1e-9)
            scale = np.abs(FH) + np.abs(FLF)
            resid = np.abs(F - FLF - theta * dH)
            assert np.all(resid[:, changed] <= 1e-9 * scale[:, changed] + 1e-300)
            # floors of the one-sided states
            for W0, sg in ((UL, -1.0), (UR, 1.0)):
                Wlf, W, Wh = W0 + sg * mu * FLF, W0 + sg * mu * F, W0 + sg * mu * FH
                r_floor = np.minimum(EPS, Wlf[0])
                p_floor = np.minimum(EPS, pressure(Wlf, g.gamma))
                tol_r = 1e-12 * np.abs(W0[0]) + 1e-12 * mu * np.abs(F[0])
                assert np.all(W[0] >= r_floor - tol_r)
                Emag = np.abs(W0[-1]) + mu * np.abs(F[-1])
                assert np.all(pressure(W, g.gamma) >= p_floor - 1e-11 * Emag)
            # minimal intervention: unchanged wherever F^H keeps both floors on both sides
            ok = np.ones(changed.shape, dtype=bool)
            for W0, sg in ((UL, -1.0), (UR, 1.0)):
                Wlf, Wh = W0 + sg * mu * FLF, W0 + sg * mu * FH
                ok &= Wh[0] >= np.minimum(EPS, Wlf[0])
                ok &= pressure(Wh, g.gamma) >= np.minimum(EPS, pressure(Wlf, g.gamma))
            assert not np.any(changed & ok)
    assert nlim > 0  # the cases do exercise the limiter


@pytest.mark.parametrize("dim", [1, 2])
def test_limiter_leaves_admissible_steps_bit_exact(orc, dim):
    """On a smooth state far from vacuum every theta is 1: the limited SSP-RK3 step equals
    the unlimited one bit for bit."""
    shape = (48,) if dim == 1 else (20, 24)
    g = orc.make_grid(tuple(reversed(shape)), (1.0 / 48,) * dim, (orc.BC_PERIODIC,) * dim)
    U = orc.init_state(g, PB.random_state(shape, 11, jumps=False))
    dt = orc.max_dt(g, U, 0.4)
    A, _ = orc.rk3_step(g, orc.make_scheme(6, orc.LIM_MP, positivity=1), U, dt)
    B, _ = orc.rk3_step(g, orc.make_scheme(6, orc.LIM_MP), U, dt)
    assert np.array_equal(A, B)


def test_periodic_conservation_with_limiter(orc):
    """The limiter only changes face fluxes, so the periodic sums of mass, momentum and
    energy stay constant to rounding."""
    shape = (24, 20)
    g, s, states = evolved_states(orc, shape, 0, 4)
    U, dt = states[-1]
    V, _ = orc.rk3_step(g, s, U, dt)
    tot0, tot1 = U.reshape(4, -1).sum(1), V.reshape(4, -1).sum(1)
    mag = np.abs(U).reshape(4, -1).sum(1)
    assert np.all(np.abs(tot1 - tot0) <= 1e-13 * mag)


def test_le_blanc_teno8_mp_with_limiter_matches_exact(orc):
    """Le Blanc (Section 4.4.2, Eq. Leblanc), 300 cells, gamma = 5/3, TENO8-MP with the
    minmod curvature and beta = 1 as Section 4.4 sets them: with the limiter the run reaches
    t = 6 with positive density and pressure, and the density and velocity are close to
    the exact Riemann solution in L1 (measured 2.0e-3 and 2.2e-2; a misplaced shock or
    a lost contact costs O(1e-2) and O(1e-1)); without the limiter it breaks down."""
    n = 300
    prim, dx = PB.le_blanc_1d(n)
    g = orc.make_grid((n,), (dx,), (orc.BC_TRANSMISSIVE,), gamma=PB.LE_BLANC_GAMMA)
    on = orc.make_scheme(8, orc.LIM_MP, mp_curv=orc.CURV_MM, mp_beta=1.0, positivity=1)
    U0 = orc.init_state(g, prim)
    U, t, steps, _ = orc.advance(g, on, U0, 6.0, 0.4)
    assert t == 6.0 and np.isfinite(U).all()
    rho, u = U[0], U[1] / U[0]
    p = pressure(U, g.gamma)
    assert rho.min() > 0 and p.min() > 0
    x = (np.arange(n) + 0.5) * dx
    ex = orc.exact_riemann(PB.LE_BLANC_LEFT, PB.LE_BLANC_RIGHT, g.gamma, (x - 3.0) / 6.0)
    assert np.abs(rho - ex[0]).mean() < 3e-3
    assert np.abs(u - ex[1]).mean() < 3e-2
    off = orc.make_scheme(8, orc.LIM_MP, mp_curv=orc.CURV_MM, mp_beta=1.0)
    V, t2, _, _ = orc.advance(g, off, U0, 6.0, 0.4, max_steps=200)
    pv = pressure(V, g.gamma)
    assert not (np.isfinite(V).all() and V[0].min() > 0 and pv.min() > 0)
