"""Frozen-branch adjoint (reverse mode through the CUDA path) against the dual-number
(forward-mode, branches frozen) CPU oracle via the dot-product identity
<w, J v> = <J^T w, v>, and against central finite differences of the GPU forward."""
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


def setup(T, orc, shape, bc, K, lim, seed, jumps=False):
    prim = PB.random_state(tuple(reversed(shape)), seed, jumps=jumps)
    dx = tuple(1.0 / n for n in shape)
    S = T.Solver(shape, dx, bc, T.make_scheme(K, limiter=lim))
    g = orc.make_grid(shape, dx, bc)
    so = orc.make_scheme(K, limiter=lim)
    Uo = orc.init_state(g, prim)
    Ug = torch.from_numpy(Uo).cuda()
    return S, g, so, Uo, Ug


def flags_agree(S, orc, g, so, Uo, Ug):
    for a in range(S.dim):
        _, flg = S.face_dump(Ug, a)
        flo = orc.faces(g, so, Uo, a)[1]
        if not np.array_equal(flg.cpu().numpy(), flo):
            return False
    return True


# The identity needs the GPU and the oracle to freeze the same branches; transmissive ghost
# copies make some cutoff decisions rounding-dependent (flat stencils), so the multi-D
# cases use periodic boundaries (flags_agree() checks the premise).
CASES = [((64,), (0,), 6, 0, 1), ((64,), (0,), 8, 1, 2), ((40,), (1,), 8, 0, 3),
         ((24, 20), (0, 0), 6, 0, 4), ((24, 20), (0, 0), 8, 1, 5), ((12, 10, 8), (0, 0, 0), 8, 0, 6),
         ((12, 10, 8), (0, 0, 0), 6, 1, 7)]


@pytest.mark.parametrize("shape,bc,K,lim,seed", CASES)
def test_rhs_vjp_dot_product_vs_dual_oracle(T, orc, shape, bc, K, lim, seed):
    S, g, so, Uo, Ug = setup(T, orc, shape, bc, K, lim, seed)
    assert flags_agree(S, orc, g, so, Uo, Ug)
    rng = np.random.default_rng(seed)
    v = rng.normal(size=Uo.shape)
    w = rng.normal(size=Uo.shape)
    _, Jv, bad = orc.rhs_jvp(g, so, Uo, v)
    assert bad == 0
    JTw = S.rhs_vjp(Ug, torch.from_numpy(w).cuda()).cpu().numpy()
    lhs, rhs = float(np.sum(w * Jv)), float(np.sum(JTw * v))
    scale = float(np.sum(np.abs(w * Jv)))
    assert abs(lhs - rhs) <= 1e-10 * scale, (lhs, rhs, scale)


@pytest.mark.parametrize("shape,bc,K,lim,seed", CASES)
def test_rhs_vjp_from_linearisation_vs_dual_oracle(T, orc, shape, bc, K, lim, seed):
    """The linearisation tape: rhs_record gives the forward's L(U) and a tape from which
    rhs_vjp_lin is the same L'^T w (dot-product identity against the dual-number oracle,
    and against the flags path, which rebuilds the reconstructions, to rounding)."""
    S, g, so, Uo, Ug = setup(T, orc, shape, bc, K, lim, seed)
    assert flags_agree(S, orc, g, so, Uo, Ug)
    lin = S.new_lin()
    R = S.rhs_record(Ug, lin)
    np.testing.assert_allclose(R.cpu().numpy(), S.rhs(Ug).cpu().numpy(), rtol=1e-13, atol=1e-13)
    rng = np.random.default_rng(seed)
    v = rng.normal(size=Uo.shape)
    w = rng.normal(size=Uo.shape)
    _, Jv, bad = orc.rhs_jvp(g, so, Uo, v)
    assert bad == 0
    wt = torch.from_numpy(w).cuda()
    JTw = S.rhs_vjp_lin(Ug, lin, wt).cpu().numpy()
    lhs, rhs = float(np.sum(w * Jv)), float(np.sum(JTw * v))
    scale = float(np.sum(np.abs(w * Jv)))
    assert abs(lhs - rhs) <= 1e-10 * scale, (lhs, rhs, scale)
    JTw_flags = S.rhs_vjp(Ug, wt).cpu().numpy()
    assert np.max(np.abs(JTw - JTw_flags)) <= 1e-11 * np.max(np.abs(JTw_flags))


@pytest.mark.parametrize("shape,bc,K,lim,seed", CASES[:1] + CASES[3:4] + CASES[4:5] + CASES[5:6])
def test_rk3_step_adjoint_vs_dual_oracle(T, orc, shape, bc, K, lim, seed):
    S, g, so, Uo, Ug = setup(T, orc, shape, bc, K, lim, seed)
    dt = 0.5 * orc.max_dt(g, Uo, 0.4)
    rng = np.random.default_rng(seed + 100)
    v = rng.normal(size=Uo.shape)
    ub = rng.normal(size=Uo.shape)
    _, Jv, bad = orc.rk3_step_jvp(g, so, Uo, v, dt)
    dt_dev = torch.tensor([dt], dtype=torch.float64, device="cuda")
    JTu = S.rk3_step_adjoint(Ug, dt_dev, torch.from_numpy(ub).cuda()).cpu().numpy()
    # the taped variant gives the same numbers (up to the order of the atomic additions)
    tape = S.new_tape()
    U1 = Ug.clone()
    S.rk3_step_record(U1, dt_dev, tape)
    JTu2 = S.rk3_step_adjoint(Ug, dt_dev, torch.from_numpy(ub).cuda(), tape=tape).cpu().numpy()
    np.testing.assert_allclose(JTu2, JTu, rtol=1e-13, atol=1e-14)
    # the linearisation tape: same step, same adjoint to rounding
    tl = S.new_tape(linear=True)
    U2 = Ug.clone()
    S.rk3_step_record(U2, dt_dev, tl)
    np.testing.assert_allclose(U2.cpu().numpy(), U1.cpu().numpy(), rtol=1e-13, atol=1e-13)
    JTu3 = S.rk3_step_adjoint(Ug, dt_dev, torch.from_numpy(ub).cuda(), tape=tl).cpu().numpy()
    assert np.max(np.abs(JTu3 - JTu)) <= 1e-11 * np.max(np.abs(JTu))
    for J in (JTu, JTu3):
        lhs, rhs = float(np.sum(ub * Jv)), float(np.sum(J * v))
        scale = float(np.sum(np.abs(ub * Jv)))
        assert abs(lhs - rhs) <= 1e-10 * scale, (lhs, rhs, scale)


@pytest.mark.parametrize("tape", ["flags", "linear"])
def test_rollout_autograd_with_checkpoints_vs_dual_oracle(T, orc, tape):
    """torch.autograd through a 7-step rollout checkpointed every 3 steps, with either tape."""
    from paper_2010_13289_gb300.autograd import rollout
    shape, bc, K, lim, seed = (24, 20), (0, 0), 6, 0, 4
    S, g, so, Uo, Ug = setup(T, orc, shape, bc, K, lim, seed)
    dt = 0.5 * orc.max_dt(g, Uo, 0.4)
    nsteps = 7
    rng = np.random.default_rng(11)
    v = rng.normal(size=Uo.shape)
    c = rng.normal(size=Uo.shape)
    U, dU = Uo.copy(), v.copy()
    for _ in range(nsteps):
        U, dU, _ = orc.rk3_step_jvp(g, so, U, dU, dt)
    U0 = Ug.clone().requires_grad_(True)
    UN = rollout(U0, S, dt, nsteps, checkpoint_every=3, tape=tape)
    np.testing.assert_allclose(UN.detach().cpu().numpy(), U, rtol=1e-11, atol=1e-12)
    loss = (UN * torch.from_numpy(c).cuda()).sum()
    loss.backward()
    grad = U0.grad.cpu().numpy()
    lhs, rhs = float(np.sum(c * dU)), float(np.sum(grad * v))
    scale = float(np.sum(np.abs(c * dU)))
    assert abs(lhs - rhs) <= 1e-10 * scale, (lhs, rhs, scale)


def pressure_window_loss(U, gamma, win, dxdy):
    rho, mx, my, E = U[0], U[1], U[2], U[3]
    p = (gamma - 1.0) * (E - 0.5 * (mx * mx + my * my) / rho)
    return (p[win] * dxdy).sum()


def lattice_fd_check(S, U, fwd, vjp, radius, spacing, seed, eps=(1e-7, 2e-8), box=False):
    """Per-cell central differences on a lattice of cells whose dependency supports (radius
    `radius`: a cross for one operator evaluation, a box for a multi-stage step) are disjoint.  For lattice cell i with random weights w_i,
    FD_i = sum_v w_iv (f_iv(U + e d) - f_iv(U - e d)) / 2e at two steps e; AD_i = sum over
    the support of i of (f'^T w)_j d_j.  A cell whose two FD values agree crossed no branch
    switch ("away from switch faces"); returns (#cells, #switch-free cells, worst relative
    error of those cells)."""
    n = S.shape[0]
    rng = np.random.default_rng(seed)
    d = torch.from_numpy(rng.normal(size=S.state_shape)).cuda() * U.abs().mean(dim=(1, 2), keepdim=True)
    idx = np.arange(radius, n - radius, spacing)
    w = np.zeros(S.state_shape)
    for y in idx:
        for x in idx:
            w[:, y, x] = rng.normal(size=S.nv)
    wt = torch.from_numpy(w).cuda()
    g = (vjp(U, wt) * d).cpu().numpy().sum(axis=0)
    fds = []
    for e in eps:
        diff = ((fwd((U + e * d).contiguous()) - fwd((U - e * d).contiguous())) / (2 * e)).cpu().numpy()
        fds.append((w * diff).sum(axis=0))
    good, worst, cells = 0, 0.0, 0
    for y in idx:
        for x in idx:
            cells += 1
            if box:  # several stages: the support fills a box
                ad = float(g[y - radius:y + radius + 1, x - radius:x + radius + 1].sum())
            else:    # one operator evaluation: the cross of the two sweeps
                ad = float(g[y - radius:y + radius + 1, x].sum() + g[y, x - radius:x + radius + 1].sum() - g[y, x])
            f1, f2 = fds[0][y, x], fds[1][y, x]
            if abs(f1 - f2) <= 1e-7 * abs(f1):
                good += 1
                worst = max(worst, abs(f1 - ad) / abs(ad))
    return cells, good, worst


@pytest.mark.parametrize("circles", [4, 0])
@pytest.mark.parametrize("linear", [False, True])
def test_operator_and_step_adjoint_vs_central_differences(T, circles, linear):
    """Central differences of the GPU forward against the adjoint, cell by cell away from
    switch faces, to 1e-6 relative: the operator L (support radius 3) and one SSP-RK3
    step (radius 9), on the broadband field with and without circular jumps; reverse from
    the flags or from the linearisation tape."""
    n = 128
    prim, dx = PB.broadband_2d(n, 5, kmax=8, ncircle=circles)
    S = T.Solver((n, n), (dx, dx), (0, 0), T.make_scheme(6))
    U = S.init_state(torch.from_numpy(prim).cuda())

    def op_vjp(X, w):
        if not linear:
            return S.rhs_vjp(X, w)
        lin = S.new_lin()
        S.rhs_record(X, lin)
        return S.rhs_vjp_lin(X, lin, w)

    def step_vjp(X, w):
        if not linear:
            return S.rk3_step_adjoint(X, dt, w)
        tape = S.new_tape(linear=True)
        S.rk3_step_record(X.clone(), dt, tape)
        return S.rk3_step_adjoint(X, dt, w, tape=tape)

    cells, good, worst = lattice_fd_check(S, U, S.rhs, op_vjp, 3, 8, 1 + circles)
    assert good >= 0.8 * cells and worst <= 1e-6, (cells, good, worst)
    dt = torch.tensor([S.max_dt(U, 0.4).item()], dtype=torch.float64, device="cuda")
    cells, good, worst = lattice_fd_check(S, U, lambda X: S.rk3_step(X, dt), step_vjp, 9, 20, 2 + circles, box=True)
    assert good >= 0.8 * cells and worst <= 1e-6, (cells, good, worst)


def test_rollout_gradient_wrt_initial_density_vs_central_differences(T):
    """The adjoint workload's gradient at small size: 2D periodic broadband field with
    circular jumps (64^2), TENO6-MP, 20 steps at fixed dt, loss = integral of p over a
    16 x 16 window, gradient with respect to the initial density (u, v, p fixed) through
    torch.autograd with checkpoints every 5 steps.  Over 20 steps the forward crosses
    branch switches (cutoff, limiter, LLF argmax): on this field a decision lies within
    about 3e-8 of its switch along most directions, so central differences at steps of
    3e-8 and above carry a jump (errors 2e-3 .. 7e-2 of |grad|), while at 1e-8 these four
    directions stay on one side and agree to their rounding floor (measured 3e-7 .. 9e-7 of
    |grad|); the bound is three times that.  Exactness is established by the dual-number
    identities and the per-cell checks above."""
    from paper_2010_13289_gb300.autograd import rollout
    n, steps, gam = 64, 20, 1.4
    prim, dx = PB.broadband_2d(n, 5, kmax=8)
    S = T.Solver((n, n), (dx, dx), (0, 0), T.make_scheme(6))
    primd = torch.from_numpy(prim).cuda()
    dt = S.max_dt(S.init_state(primd), 0.4).item()
    win = (slice(24, 40), slice(10, 26))

    def loss_of(rho0, grad=False):
        pr = primd.clone()
        pr[0] = rho0
        U0 = S.init_state(pr)
        if grad:
            U0.requires_grad_(True)
        UN = rollout(U0, S, dt, steps, checkpoint_every=5)
        L = pressure_window_loss(UN, gam, win, dx * dx)
        return L, U0

    L, U0 = loss_of(primd[0], grad=True)
    L.backward()
    Ub = U0.grad
    u, v = primd[1], primd[2]
    grad_rho = Ub[0] + u * Ub[1] + v * Ub[2] + 0.5 * (u * u + v * v) * Ub[3]
    gnorm = float(torch.linalg.norm(grad_rho))
    rng = np.random.default_rng(7)
    for k in range(4):
        d = torch.from_numpy(rng.normal(size=(n, n))).cuda()
        d /= torch.linalg.norm(d)
        eps = 1e-8
        Lp, _ = loss_of(primd[0] + eps * d)
        Lm, _ = loss_of(primd[0] - eps * d)
        fd = (Lp - Lm).item() / (2 * eps)
        ad = float((grad_rho * d).sum())
        # unit directions: the error is measured against the gradient norm (a direction
        # nearly orthogonal to the gradient has a derivative below the FD rounding floor)
        assert abs(fd - ad) <= 3e-6 * gnorm, (k, fd, ad, gnorm)
