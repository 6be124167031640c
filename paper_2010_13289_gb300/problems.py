"""Seeded synthetic initial conditions in primitive variables (rho, u_1..u_D, p).

This module holds no arithmetic of the reconstruction method: it only draws the
initial fields.  Both the CUDA path and the CPU oracle are fed from here.  Every
array is FP64, laid out [nvar][nz][ny][nx] (x fastest, leading singleton axes
dropped for lower dimensions).

Workloads (shaped like the paper's Section 4 problems):
  riemann_1d        seeded shock tube on [0,1] (Sod/Lax-like, Section 4.2.1)
  broadband_2d      periodic [0,1]^2: random-phase Fourier modes 1 <= |k| <= kmax,
                    rms 1e-2, plus 4 circular density/pressure jumps (ratio 2-10)
  solenoidal_3d     periodic [0,2pi]^3: solenoidal random-phase velocity with
                    E(k) ~ k^4 exp(-2 (k/4)^2), rms Mach 0.6, rho = 1, p = 1/gamma
  batch_sizes       log-uniform sizes 128..8192 for batched 1D problems
  gaussian_pulse    exp(-300 (x - 0.5)^2) on [0,1] (Section 4.1.1)
  taylor_green_3d   inviscid Taylor-Green vortex (Section 4.3.1)
  le_blanc_1d       Le Blanc shock tube on [0,9], gamma = 5/3 (Section 4.4.2)
  near_vacuum       seeded blocks of density 1e-3..1 and pressure 1e-10..1e-1
"""
import numpy as np

GAMMA = 1.4


def riemann_states(seed):
    """Left/right (rho, u, p): rho, p ~ U[0.1, 1], u ~ U[-1, 1]."""
    rng = np.random.default_rng(seed)
    rl, rr = rng.uniform(0.1, 1.0, 2)
    ul, ur = rng.uniform(-1.0, 1.0, 2)
    pl, pr = rng.uniform(0.1, 1.0, 2)
    return (rl, ul, pl), (rr, ur, pr)


def riemann_1d(n, seed, x0=0.0, x1=1.0, xc=0.5, states=None):
    """Primitive field [3][n] of a Riemann problem with interface at xc; cell i at
    x_i = x0 + (i + 1/2) dx.  Returns (prim, dx)."""
    left, right = riemann_states(seed) if states is None else states
    dx = (x1 - x0) / n
    x = x0 + (np.arange(n) + 0.5) * dx
    prim = np.empty((3, n))
    lm = x < xc
    for q in range(3):
        prim[q] = np.where(lm, left[q], right[q])
    return prim, dx


def _fourier_field(rng, shape, kmax):
    """Real periodic field: sum over integer wavevectors 1 <= |k| <= kmax of unit
    amplitude cosines with random phases, normalised to unit rms."""
    ks = [np.fft.fftfreq(n, 1.0 / n) for n in shape]
    grids = np.meshgrid(*ks, indexing="ij")
    kk = np.sqrt(sum(g * g for g in grids))
    mask = (kk >= 1.0) & (kk <= kmax)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=shape)
    spec = np.where(mask, np.exp(1j * phase), 0.0)
    f = np.real(np.fft.ifftn(spec))
    rms = np.sqrt(np.mean(f * f))
    return f / rms if rms > 0 else f


def broadband_2d(n, seed, kmax=32, amp=1e-2, ncircle=4, gamma=GAMMA):
    """2D periodic field on [0,1]^2, n x n points.  Base (1, 0, 0, 1/gamma) (c = 1);
    independent random-phase perturbations of rho, u, v, p with rms amp (relative for
    rho and p, absolute for u and v); then ncircle circles (centres U[0,1]^2, radii
    U[0.05, 0.15], periodic distance, sharp at points) in which rho and p are
    multiplied by ratios U[2, 10], applied one after another.  Returns (prim[4][n][n], dx)."""
    rng = np.random.default_rng(seed)
    kmax = min(kmax, n // 4)
    shape = (n, n)  # (y, x)
    dx = 1.0 / n
    base = [1.0, 0.0, 0.0, 1.0 / gamma]
    prim = np.empty((4, n, n))
    for q in range(4):
        f = _fourier_field(rng, shape, kmax) * amp
        prim[q] = base[q] * (1.0 + f) if q in (0, 3) else f
    x = (np.arange(n) + 0.5) * dx
    X, Y = np.meshgrid(x, x, indexing="xy")
    for _ in range(ncircle):
        cx, cy = rng.uniform(0.0, 1.0, 2)
        rad = rng.uniform(0.05, 0.15)
        ratio = rng.uniform(2.0, 10.0)
        ddx = np.abs(X - cx)
        ddx = np.minimum(ddx, 1.0 - ddx)
        ddy = np.abs(Y - cy)
        ddy = np.minimum(ddy, 1.0 - ddy)
        inside = ddx * ddx + ddy * ddy < rad * rad
        prim[0][inside] *= ratio
        prim[3][inside] *= ratio
    return prim, dx


def solenoidal_3d(n, seed, mach=0.6, k0=4.0, gamma=GAMMA):
    """3D periodic field on [0, 2 pi]^3, n^3 points: rho = 1, p = 1/gamma (c = 1),
    solenoidal random-phase velocity with energy spectrum E(k) ~ k^4 exp(-2 (k/k0)^2)
    (Helmholtz-projected in Fourier space), scaled to rms |u| / c = mach.
    Returns (prim[5][n][n][n], dx)."""
    rng = np.random.default_rng(seed)
    dx = 2.0 * np.pi / n
    k1 = np.fft.fftfreq(n, 1.0 / n)
    KZ, KY, KX = np.meshgrid(k1, k1, k1, indexing="ij")
    kk = np.sqrt(KX * KX + KY * KY + KZ * KZ)
    E = kk ** 4 * np.exp(-2.0 * (kk / k0) ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        amp = np.where(kk > 0, np.sqrt(E / (4.0 * np.pi * kk * kk)), 0.0)
    comps = []
    for _ in range(3):
        ph = rng.uniform(0.0, 2.0 * np.pi, size=kk.shape)
        comps.append(amp * np.exp(1j * ph))
    # project out the component along k (solenoidal part)
    with np.errstate(divide="ignore", invalid="ignore"):
        kdot = (KX * comps[0] + KY * comps[1] + KZ * comps[2]) / np.where(kk > 0, kk * kk, 1.0)
    comps = [comps[0] - KX * kdot, comps[1] - KY * kdot, comps[2] - KZ * kdot]
    vel = [np.real(np.fft.ifftn(c)) for c in comps]  # order (u_x, u_y, u_z)
    rms = np.sqrt(np.mean(vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2))
    prim = np.empty((5, n, n, n))
    prim[0] = 1.0
    for d in range(3):
        prim[1 + d] = vel[d] * (mach / rms)
    prim[4] = 1.0 / gamma
    return prim, dx


def taylor_green_3d(n, gamma=GAMMA):
    """Inviscid Taylor-Green vortex (Section 4.3.1, Eq. TGV): on [0, 2 pi]^3, n^3 points at
    cell centres, rho = 1, u = sin x cos y cos z, v = -cos x sin y cos z, w = 0,
    p = 100 + ((cos 2x + cos 2y)(2 + cos 2z) - 2)/16.  Returns (prim[5][n][n][n], dx)."""
    dx = 2.0 * np.pi / n
    x = (np.arange(n) + 0.5) * dx
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    prim = np.empty((5, n, n, n))
    prim[0] = 1.0
    prim[1] = np.sin(X) * np.cos(Y) * np.cos(Z)
    prim[2] = -np.cos(X) * np.sin(Y) * np.cos(Z)
    prim[3] = 0.0
    prim[4] = 100.0 + ((np.cos(2 * X) + np.cos(2 * Y)) * (2.0 + np.cos(2 * Z)) - 2.0) / 16.0
    return prim, dx


LE_BLANC_GAMMA = 5.0 / 3.0
LE_BLANC_LEFT = (1.0, 0.0, 2.0 / 3.0 * 1e-1)
LE_BLANC_RIGHT = (1e-3, 0.0, 2.0 / 3.0 * 1e-10)


def le_blanc_1d(n):
    """Le Blanc problem (Section 4.4.2, Eq. Leblanc): on [0, 9], (rho, u, p) = (1, 0, 2/3 1e-1)
    for x < 3 and (1e-3, 0, 2/3 1e-10) for x >= 3, n cells; gamma = 5/3, run to t = 6.
    Returns (prim[3][n], dx)."""
    return riemann_1d(n, 0, x0=0.0, x1=9.0, xc=3.0, states=(LE_BLANC_LEFT, LE_BLANC_RIGHT))


def near_vacuum(shape, seed, block=4):
    """Seeded state of piecewise-constant blocks (block^D cells) with log-uniform density
    in [1e-3, 1], pressure in [1e-10, 1e-1] and velocity components in [-1, 1]: every block
    edge is a strong jump next to near-vacuum.  shape = (nz, ny, nx) trailing dims.
    Returns prim[D+2][*shape]."""
    rng = np.random.default_rng(seed)
    D = len(shape)
    nb = [-(-n // block) for n in shape]
    rho = 10.0 ** rng.uniform(-3.0, 0.0, nb)
    p = 10.0 ** rng.uniform(-10.0, -1.0, nb)
    vel = rng.uniform(-1.0, 1.0, [D] + nb)
    def expand(a):
        for ax in range(D):
            a = np.repeat(a, block, axis=ax)
        return a[tuple(slice(0, n) for n in shape)]
    prim = np.empty((D + 2,) + tuple(shape))
    prim[0] = expand(rho)
    for d in range(D):
        prim[1 + d] = expand(vel[d])
    prim[D + 1] = expand(p)
    return prim


def batch_sizes(nprob, seed, nmin=128, nmax=8192):
    """Sizes N_j = round(exp(U[ln nmin, ln nmax])) of independent 1D problems."""
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(np.log(nmin), np.log(nmax), nprob))).astype(np.int64)


def batch_riemann(nprob, seed, nmin=128, nmax=8192):
    """Ragged batch of seeded 1D Riemann problems on [0,1]: (sizes, list of prim[3][n_j], dx_j)."""
    sizes = batch_sizes(nprob, seed, nmin, nmax)
    rng = np.random.default_rng(seed + 7919)
    seeds = rng.integers(0, 2**31 - 1, nprob)
    prims, dxs = [], []
    for n, s in zip(sizes, seeds):
        p, dx = riemann_1d(int(n), int(s))
        prims.append(p)
        dxs.append(dx)
    return sizes, prims, np.array(dxs)


def gaussian_pulse(n):
    """u(x, 0) = exp(-300 (x - 0.5)^2) at x_i = (i + 1/2)/n on [0,1] (Section 4.1.1)."""
    x = (np.arange(n) + 0.5) / n
    return np.exp(-300.0 * (x - 0.5) ** 2), 1.0 / n


def smooth_1d(n, seed, amp=0.2):
    """Smooth periodic 1D Euler state on [0,1]: rho = 1 + amp sin(2 pi x + phi),
    u = 1, p = 1 (an advected entropy wave).  Returns (prim, dx)."""
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0, 2 * np.pi)
    dx = 1.0 / n
    x = (np.arange(n) + 0.5) * dx
    prim = np.empty((3, n))
    prim[0] = 1.0 + amp * np.sin(2 * np.pi * x + phi)
    prim[1] = 1.0
    prim[2] = 1.0
    return prim, dx


def random_state(shape, seed, jumps=True):
    """Generic seeded positive state for parity tests: smooth broadband background plus
    (optionally) random sharp jumps.  shape = (nz, ny, nx) trailing dims; D = len(shape).
    Returns prim[D+2][*shape]."""
    rng = np.random.default_rng(seed)
    D = len(shape)
    prim = np.empty((D + 2,) + tuple(shape))
    coords = np.meshgrid(*[(np.arange(n) + 0.5) / n for n in shape], indexing="ij")
    for q in range(D + 2):
        f = np.zeros(shape)
        for _ in range(4):
            k = rng.integers(1, 4, D)
            ph = rng.uniform(0, 2 * np.pi)
            f += rng.uniform(0.05, 0.2) * np.sin(2 * np.pi * sum(k[j] * coords[j] for j in range(D)) + ph)
        if q == 0 or q == D + 1:
            prim[q] = 1.0 + 0.5 * f
        else:
            prim[q] = f
    if jumps:
        for _ in range(3):
            c = [rng.uniform(0, 1) for _ in range(D)]
            r = rng.uniform(0.1, 0.3)
            d2 = sum((coords[j] - c[j]) ** 2 for j in range(D))
            inside = d2 < r * r
            ratio = rng.uniform(2.0, 6.0)
            prim[0][inside] *= ratio
            prim[D + 1][inside] *= rng.uniform(2.0, 6.0)
            for d in range(D):
                prim[1 + d][inside] += rng.uniform(-0.5, 0.5)
    return prim
