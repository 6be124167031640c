"""CPU oracle of the TENO-M method (arXiv 2010.13289): ctypes front end.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import this module.  It shares no code with the CUDA library.

The arithmetic lives in tenom_oracle.hpp / exact_riemann.hpp (plain C++17, FP64,
IEEE semantics: built with -ffp-contract=off so every operation rounds once, on any
host).  Parity pinned by tests/test_oracle_*.py except where the header of
tenom_oracle.hpp says "parity unpinned".
"""
import ctypes
import os
import subprocess
import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")
SOURCES = ["oracle_capi.cpp"]
HEADERS = ["tenom_oracle.hpp", "exact_riemann.hpp", "beta_forms.h"]

LIM_MP, LIM_TVD5, LIM_VA = 0, 1, 2
CT_CONST, CT_ADAPTIVE = 0, 1
CURV_M4, CURV_MM = 0, 1
W_TENOM, W_TENO = 0, 1
BC_PERIODIC, BC_TRANSMISSIVE = 0, 1


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("dx", ctypes.c_double * 3),
                ("bc", ctypes.c_int * 3), ("gamma", ctypes.c_double)]


class Scheme(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("limiter", ctypes.c_int), ("ct_mode", ctypes.c_int),
                ("ct_const", ctypes.c_double), ("mp_alpha", ctypes.c_double), ("mp_beta", ctypes.c_double),
                ("mp_curv", ctypes.c_int), ("weights", ctypes.c_int), ("d", ctypes.c_double * 6),
                ("positivity", ctypes.c_int)]


def make_grid(shape, dx, bc, gamma=1.4):
    """shape/dx/bc given x-first (n_x, n_y, n_z)."""
    g = Grid()
    g.dim = len(shape)
    for a in range(3):
        g.n[a] = shape[a] if a < len(shape) else 1
        g.dx[a] = dx[a] if a < len(shape) else 1.0
        g.bc[a] = bc[a] if a < len(shape) else BC_PERIODIC
    g.gamma = gamma
    return g


def make_scheme(K=6, limiter=LIM_MP, ct_mode=None, ct_const=1e-5, mp_alpha=1.25, mp_beta=4.0,
                mp_curv=CURV_M4, weights=W_TENOM, d=None, positivity=0):
    """Defaults: K = 6 uses constant C_T = 1e-5, K = 8 the adaptive C_T of TENO8A.
    positivity=1: the positivity-preserving flux limiter (Section 4.4) in every RK stage."""
    s = Scheme()
    s.K = K
    s.limiter = limiter
    s.ct_mode = (CT_CONST if K == 6 else CT_ADAPTIVE) if ct_mode is None else ct_mode
    s.ct_const = ct_const
    s.mp_alpha = mp_alpha
    s.mp_beta = mp_beta
    s.mp_curv = mp_curv
    s.weights = weights
    s.positivity = positivity
    for k in range(6):
        s.d[k] = 0.0 if d is None else (d[k] if k < len(d) else 0.0)
    return s


def build(force=False):
    """Compile liboracle.so with g++ (plain C++17, no FMA contraction)."""
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, h) for h in HEADERS]
    if not force and os.path.exists(LIB_PATH):
        t = os.path.getmtime(LIB_PATH)
        if all(os.path.getmtime(d) <= t for d in deps):
            return LIB_PATH
    tmp = LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp] + srcs
    subprocess.check_call(cmd, cwd=HERE)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


_lib = None


def lib():
    """The oracle library.  TENOM_ORACLE_LIB, when set, names a prebuilt copy to load instead
    (the mutation tests load copies of the oracle with one mistake planted in them)."""
    global _lib
    if _lib is None:
        path = os.environ.get("TENOM_ORACLE_LIB")
        if not path:
            build()
            path = LIB_PATH
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        dp, ip, u8p = P(ctypes.c_double), P(ctypes.c_int), P(ctypes.c_uint8)
        gp, sp = P(Grid), P(Scheme)
        c_int, c_double = ctypes.c_int, ctypes.c_double
        L.orc_recon.argtypes = [sp, dp, c_int, dp, ip, ip, dp, dp]
        L.orc_recon_parts.argtypes = [sp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
        L.orc_init_state.argtypes = [gp, dp, dp]
        L.orc_faces.argtypes = [gp, sp, dp, c_int, dp, u8p, dp, dp, dp]
        L.orc_faces.restype = c_int
        L.orc_faces_at.argtypes = [gp, sp, dp, c_int, ip, c_int, dp, u8p, dp, dp, dp]
        L.orc_faces_at.restype = c_int
        L.orc_faces_limited.argtypes = [gp, sp, dp, c_int, c_double, dp]
        L.orc_faces_limited.restype = c_int
        L.orc_positivity_limit.argtypes = [gp, dp, c_int, c_double, dp]
        L.orc_rhs.argtypes = [gp, sp, dp, dp]
        L.orc_rhs.restype = c_int
        L.orc_max_dt.argtypes = [gp, dp, c_double]
        L.orc_max_dt.restype = c_double
        L.orc_rk3_step.argtypes = [gp, sp, dp, c_double]
        L.orc_rk3_step.restype = c_int
        L.orc_advance.argtypes = [gp, sp, dp, c_double, c_double, c_int, dp, ip]
        L.orc_advance.restype = c_int
        L.orc_rhs_jvp.argtypes = [gp, sp, dp, dp, dp, dp]
        L.orc_rhs_jvp.restype = c_int
        L.orc_rk3_step_jvp.argtypes = [gp, sp, dp, dp, c_double]
        L.orc_rk3_step_jvp.restype = c_int
        L.orc_face_flops.argtypes = [gp, sp, dp, c_int]
        L.orc_face_flops.restype = ctypes.c_longlong
        L.orc_face_flops_at.argtypes = [gp, sp, dp, c_int, ip, c_int]
        L.orc_face_flops_at.restype = ctypes.c_longlong
        L.orc_roe_eigen.argtypes = [gp, dp, dp, c_int, dp, dp]
        L.orc_phys_flux.argtypes = [gp, dp, c_int, dp]
        L.orc_scalar_rhs.argtypes = [sp, c_int, c_double, dp, dp]
        L.orc_scalar_advance.argtypes = [sp, c_int, c_double, dp, c_double, c_int]
        L.orc_exact_riemann.argtypes = [c_double] * 7 + [dp, c_int, dp, dp, dp, dp]
        L.orc_exact_riemann.restype = c_int
        L.orc_default_weights.argtypes = [c_int, dp]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def default_weights(K):
    d = np.zeros(6)
    lib().orc_default_weights(K, _d(d))
    return d[:K - 2]


def recon(scheme, v):
    """Scalar TENO-M reconstructions of rows v[n, K]; returns (fhat, delta_bits, ct_exp, cut_rel, beta_ct)."""
    v = _c(v)
    n = v.shape[0]
    out = np.zeros(n)
    bits = np.zeros(n, dtype=np.int32)
    cte = np.zeros(n, dtype=np.int32)
    cut = np.zeros((n, 6))
    bct = np.zeros(n)
    lib().orc_recon(ctypes.byref(scheme), _d(v), n, _d(out), bits.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                    cte.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _d(cut), _d(bct))
    return out, bits, cte, cut, bct


def recon_parts(scheme, f):
    f = _c(f)
    K = scheme.K
    cand = np.zeros(6)
    beta = np.zeros(6)
    bK, tau, mn, mx, tv, va = (np.zeros(1) for _ in range(6))
    lib().orc_recon_parts(ctypes.byref(scheme), _d(f), _d(cand), _d(beta), _d(bK), _d(tau), _d(mn), _d(mx),
                          _d(tv), _d(va))
    return dict(cand=cand[:K - 2], beta=beta[:K - 2], betaK=bK[0], tau=tau[0], mpmin=mn[0], mpmax=mx[0],
                tvd5=tv[0], va=va[0])


def nvar(grid):
    return grid.dim + 2


def init_state(grid, prim):
    prim = _c(prim)
    U = np.zeros_like(prim)
    lib().orc_init_state(ctypes.byref(grid), _d(prim), _d(U))
    return U


def face_shape(grid, axis):
    """numpy shape (z, y, x) of the face array of an axis."""
    n = [grid.n[a] for a in range(grid.dim)]
    n[axis] += 1
    return tuple(reversed(n))


def faces(grid, scheme, U, axis, with_scale=False):
    """All face fluxes of one axis: (Fhat[nv, *face_shape], flags[*face_shape, nv, 2],
    cut[*face_shape, nv, 2], noise[*face_shape, nv, 2], bad).  flags = delta bits | ct code << 6;
    cut = distance of the cutoff decision from its threshold (relative); noise = rounding-noise
    ratio of the reconstructed sequence; scale[nv, *face_shape] (with_scale=True) = magnitude of
    the terms of the back-projection sum sum_s r_s (f+_s + f-_s)."""
    U = _c(U)
    fs = face_shape(grid, axis)
    nv = nvar(grid)
    F = np.zeros((nv,) + fs)
    fl = np.zeros(fs + (nv, 2), dtype=np.uint8)
    cut = np.zeros(fs + (nv, 2))
    noise = np.zeros(fs + (nv, 2))
    scale = np.zeros((nv,) + fs)
    bad = lib().orc_faces(ctypes.byref(grid), ctypes.byref(scheme), _d(U), axis, _d(F),
                          fl.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), _d(cut), _d(noise), _d(scale))
    if with_scale:
        return F, fl, cut, noise, bad, scale
    return F, fl, cut, noise, bad


def faces_at(grid, scheme, U, axis, idx, with_scale=False):
    """Face fluxes at selected faces; idx[n, 3] = (x, y, z) with the face index on `axis`."""
    U = _c(U)
    idx = _c(idx, np.int32)
    n = idx.shape[0]
    nv = nvar(grid)
    F = np.zeros((n, nv))
    fl = np.zeros((n, nv, 2), dtype=np.uint8)
    cut = np.zeros((n, nv, 2))
    noise = np.zeros((n, nv, 2))
    scale = np.zeros((n, nv))
    bad = lib().orc_faces_at(ctypes.byref(grid), ctypes.byref(scheme), _d(U), axis,
                             idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), n, _d(F),
                             fl.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), _d(cut), _d(noise), _d(scale))
    if with_scale:
        return F, fl, cut, noise, bad, scale
    return F, fl, cut, noise, bad


def faces_limited(grid, scheme, U, axis, dt):
    """Face fluxes [nv, *face_shape] of one axis after the positivity limiter of a
    forward-Euler stage of length dt (Section 4.4)."""
    U = _c(U)
    F = np.zeros((nvar(grid),) + face_shape(grid, axis))
    bad = lib().orc_faces_limited(ctypes.byref(grid), ctypes.byref(scheme), _d(U), axis, dt, _d(F))
    return F, bad


def positivity_limit(grid, U, axis, dt, F):
    """The positivity limiter (Section 4.4) applied to given face fluxes F[nv, *face_shape]
    of one axis; returns the limited copy."""
    F = _c(F).copy()
    lib().orc_positivity_limit(ctypes.byref(grid), _d(_c(U)), axis, dt, _d(F))
    return F


def rhs(grid, scheme, U):
    U = _c(U)
    out = np.zeros_like(U)
    bad = lib().orc_rhs(ctypes.byref(grid), ctypes.byref(scheme), _d(U), _d(out))
    return out, bad


def max_dt(grid, U, cfl):
    return lib().orc_max_dt(ctypes.byref(grid), _d(_c(U)), cfl)


def rk3_step(grid, scheme, U, dt):
    U = _c(U).copy()
    bad = lib().orc_rk3_step(ctypes.byref(grid), ctypes.byref(scheme), _d(U), dt)
    return U, bad


def advance(grid, scheme, U, t_end, cfl=0.4, max_steps=1 << 30):
    U = _c(U).copy()
    t = np.zeros(1)
    st = np.zeros(1, dtype=np.int32)
    bad = lib().orc_advance(ctypes.byref(grid), ctypes.byref(scheme), _d(U), t_end, cfl, max_steps, _d(t),
                            st.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return U, float(t[0]), int(st[0]), bad


def rk3_step_jvp(grid, scheme, U, dU, dt):
    U = _c(U).copy()
    dU = _c(dU).copy()
    bad = lib().orc_rk3_step_jvp(ctypes.byref(grid), ctypes.byref(scheme), _d(U), _d(dU), dt)
    return U, dU, bad


def rhs_jvp(grid, scheme, U, dU):
    """(L(U), L'(U) dU) with every branch frozen at U (dual numbers)."""
    U = _c(U)
    dU = _c(dU)
    Lv = np.zeros_like(U)
    dL = np.zeros_like(U)
    bad = lib().orc_rhs_jvp(ctypes.byref(grid), ctypes.byref(scheme), _d(U), _d(dU), _d(Lv), _d(dL))
    return Lv, dL, bad


def face_flops(grid, scheme, U, axis):
    return int(lib().orc_face_flops(ctypes.byref(grid), ctypes.byref(scheme), _d(_c(U)), axis))


def face_flops_at(grid, scheme, U, axis, idx):
    """Counted FP64 operations summed over the faces idx[n, 3]."""
    idx = _c(idx, np.int32)
    return int(lib().orc_face_flops_at(ctypes.byref(grid), ctypes.byref(scheme), _d(_c(U)), axis,
                                       idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), idx.shape[0]))


def roe_eigen(grid, UL, UR, axis):
    nv = nvar(grid)
    R = np.zeros((nv, nv))
    L = np.zeros((nv, nv))
    lib().orc_roe_eigen(ctypes.byref(grid), _d(_c(UL)), _d(_c(UR)), axis, _d(R), _d(L))
    return R, L


def phys_flux(grid, U, axis):
    F = np.zeros(nvar(grid))
    lib().orc_phys_flux(ctypes.byref(grid), _d(_c(U)), axis, _d(F))
    return F


def scalar_rhs(scheme, u, dx):
    u = _c(u)
    out = np.zeros_like(u)
    lib().orc_scalar_rhs(ctypes.byref(scheme), u.size, dx, _d(u), _d(out))
    return out


def scalar_advance(scheme, u, dx, dt, nsteps):
    u = _c(u).copy()
    lib().orc_scalar_advance(ctypes.byref(scheme), u.size, dx, _d(u), dt, nsteps)
    return u


def exact_riemann(left, right, gamma, xi):
    xi = _c(xi)
    n = xi.size
    rho, u, p = np.zeros(n), np.zeros(n), np.zeros(n)
    star = np.zeros(2)
    bad = lib().orc_exact_riemann(left[0], left[1], left[2], right[0], right[1], right[2], gamma, _d(xi), n,
                                  _d(rho), _d(u), _d(p), _d(star))
    if bad:
        raise ValueError("vacuum generated")
    return rho, u, p, star
