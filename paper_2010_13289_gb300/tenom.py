"""Python binding of the C ABI in include/tenom.h (argument marshalling only).

Every step of the method runs in libtenom.so's CUDA kernels; this module only converts
torch tensors to device pointers and streams.  If the library is missing it raises:
there is no CPU fallback.  PyTorch provides device memory and streams.
"""
import ctypes
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtenom.so")

TENOM_OK, TENOM_E_INVALID, TENOM_E_CUDA, TENOM_E_NONPHYSICAL, TENOM_E_TIMEOUT, TENOM_E_UNSUPPORTED = range(6)
BC_PERIODIC, BC_TRANSMISSIVE = 0, 1
LIM_MP, LIM_TVD5, LIM_VA = 0, 1, 2
PP_OFF, PP_ON = 0, 1
CT_CONST, CT_ADAPTIVE = 0, 1
CURV_M4, CURV_MM = 0, 1
W_TENOM, W_TENO = 0, 1
ST_RHO, ST_P, ST_ROE, ST_NONFINITE = 1, 2, 4, 8
NSTATS = 20  # tenom_decision_stats counters
STATS_FIELDS = ("sides", "certified", "certified_disagree", "all_smooth", "nonsmooth_k0", "nonsmooth_k1",
                "nonsmooth_k2", "nonsmooth_k3", "nonsmooth_k4", "nonsmooth_k5", "limited_sides",
                "limiter_changed", "near_cutoff", "near_cutoff_sides", "ct_exp_7", "ct_exp_8", "ct_exp_9",
                "ct_exp_10", "near_integer_beta", "nonfinite")


def stats_dict(counters, K):
    """The counters of tenom_decision_stats as a dict (nonsmooth_k for k < K - 2 only)."""
    vals = [int(x) for x in counters]
    d = dict(zip(STATS_FIELDS, vals))
    for k in range(K - 2, 6):
        d.pop("nonsmooth_k%d" % k)
    return d


class tenom_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("dx", ctypes.c_double * 3),
                ("bc", ctypes.c_int * 3), ("gamma", ctypes.c_double)]


class tenom_scheme(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("limiter", ctypes.c_int), ("ct_mode", ctypes.c_int),
                ("ct_const", ctypes.c_double), ("mp_alpha", ctypes.c_double), ("mp_beta", ctypes.c_double),
                ("mp_curv", ctypes.c_int), ("weights", ctypes.c_int), ("d", ctypes.c_double * 6),
                ("decisions", ctypes.c_int), ("positivity", ctypes.c_int)]


DECIDE_FILTERED, DECIDE_FP64 = 0, 1


class TenomError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("tenom status %d: %s" % (status, msg))
        self.status = status


_lib = None
VP = ctypes.c_void_p


def lib():
    """Load libtenom.so (build it first with __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libtenom.so not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        c_int, c_double, P = ctypes.c_int, ctypes.c_double, ctypes.POINTER
        L.tenom_scheme_default.argtypes = [P(tenom_scheme), c_int]
        L.tenom_create.argtypes = [P(VP), P(tenom_grid), P(tenom_scheme), VP]
        L.tenom_destroy.argtypes = [VP]
        L.tenom_init_state.argtypes = [VP, VP, VP]
        L.tenom_rhs.argtypes = [VP, VP, VP]
        L.tenom_max_dt.argtypes = [VP, VP, c_double, VP]
        L.tenom_rk3_step.argtypes = [VP, VP, VP]
        L.tenom_advance.argtypes = [VP, VP, VP, c_double, c_double, c_int]
        L.tenom_advance_host.argtypes = [VP, VP, VP, P(c_double), c_double, c_double, c_int]
        L.tenom_face_dump.argtypes = [VP, VP, c_int, VP, VP]
        L.tenom_decision_stats.argtypes = [VP, VP, c_int, VP]
        L.tenom_positivity_limit.argtypes = [VP, VP, c_int, VP, VP]
        L.tenom_status_word.argtypes = [VP, P(c_int), c_int]
        L.tenom_last_error.argtypes = [VP]
        L.tenom_last_error.restype = ctypes.c_char_p
        L.tenom_kernel_timing.argtypes = [VP, c_int, P(c_double), P(ctypes.c_longlong)]
        L.tenom_fp64_peak.argtypes = [VP, c_int, c_int, P(c_double)]
        L.tenom_flags_bytes.argtypes = [VP]
        L.tenom_flags_bytes.restype = ctypes.c_size_t
        L.tenom_rhs_vjp.argtypes = [VP, VP, VP, VP]
        L.tenom_rk3_step_record.argtypes = [VP, VP, VP, VP, VP]
        L.tenom_rk3_step_adjoint_tape.argtypes = [VP, VP, VP, VP, VP, VP, VP]
        L.tenom_rk3_step_adjoint.argtypes = [VP, VP, VP, VP, VP]
        L.tenom_lin_tape_bytes.argtypes = [VP]
        L.tenom_lin_tape_bytes.restype = ctypes.c_size_t
        L.tenom_rhs_record.argtypes = [VP, VP, VP, VP]
        L.tenom_rhs_vjp_lin.argtypes = [VP, VP, VP, VP, VP]
        L.tenom_rk3_step_record_lin.argtypes = [VP, VP, VP, VP, VP]
        L.tenom_rk3_step_adjoint_lin.argtypes = [VP, VP, VP, VP, VP, VP, VP]
        for name in ("tenom_rhs_vjp", "tenom_rk3_step_record", "tenom_rk3_step_adjoint_tape",
                     "tenom_rk3_step_adjoint", "tenom_rhs_record", "tenom_rhs_vjp_lin",
                     "tenom_rk3_step_record_lin", "tenom_rk3_step_adjoint_lin"):
            getattr(L, name).restype = c_int
        L.tenom_check_fastmath.argtypes = [VP, VP, ctypes.c_longlong, VP]
        L.tenom_check_fastmath.restype = c_int
        L.tenom_rhs_noalloc.argtypes = [P(tenom_grid), P(tenom_scheme), VP, VP, VP, VP]
        L.tenom_batch_create.argtypes = [P(VP), c_int, VP, VP, VP, c_double, P(tenom_scheme), VP]
        L.tenom_batch_destroy.argtypes = [VP]
        L.tenom_batch_layout.argtypes = [VP, VP, P(ctypes.c_longlong)]
        L.tenom_batch_init_state.argtypes = [VP, VP, VP]
        L.tenom_batch_set_time.argtypes = [VP, VP, VP]
        L.tenom_batch_get_time.argtypes = [VP, VP]
        L.tenom_batch_status_word.argtypes = [VP, P(c_int), c_int]
        L.tenom_batch_step.argtypes = [VP, VP, c_double, c_int]
        L.tenom_batch_step_direct.argtypes = [VP, VP, c_double, c_int]
        L.tenom_batch_stage.argtypes = [VP, c_int, VP]
        L.tenom_batch_autotune.argtypes = [VP, VP, P(c_int), P(c_int)]
        L.tenom_batch_set_tiling.argtypes = [VP, c_int, c_int]
        for name in ("tenom_batch_create", "tenom_batch_destroy", "tenom_batch_layout", "tenom_batch_init_state",
                     "tenom_batch_set_time", "tenom_batch_get_time", "tenom_batch_status_word", "tenom_batch_step",
                     "tenom_batch_step_direct", "tenom_batch_stage", "tenom_batch_autotune",
                     "tenom_batch_set_tiling"):
            getattr(L, name).restype = c_int
        L.tenom_rhs_noalloc.restype = c_int
        for name in ("tenom_scheme_default", "tenom_create", "tenom_destroy", "tenom_init_state", "tenom_rhs",
                     "tenom_max_dt", "tenom_rk3_step", "tenom_advance", "tenom_advance_host", "tenom_face_dump",
                     "tenom_positivity_limit", "tenom_status_word", "tenom_kernel_timing", "tenom_fp64_peak",
                     "tenom_decision_stats"):
            getattr(L, name).restype = c_int
        _lib = L
    return _lib


def make_grid(shape, dx, bc, gamma=1.4):
    """shape, dx, bc listed x-first."""
    g = tenom_grid()
    g.dim = len(shape)
    for a in range(3):
        g.n[a] = int(shape[a]) if a < len(shape) else 1
        g.dx[a] = float(dx[a]) if a < len(shape) else 1.0
        g.bc[a] = int(bc[a]) if a < len(shape) else BC_PERIODIC
    g.gamma = gamma
    return g


def make_scheme(K=6, limiter=LIM_MP, ct_mode=None, ct_const=1e-5, mp_alpha=1.25, mp_beta=4.0, mp_curv=CURV_M4,
                weights=W_TENOM, d=None, decisions=DECIDE_FILTERED, positivity=PP_OFF):
    s = tenom_scheme()
    st = lib().tenom_scheme_default(ctypes.byref(s), K)
    if st != TENOM_OK:
        raise TenomError(st, "tenom_scheme_default(K=%d)" % K)
    s.limiter = limiter
    if ct_mode is not None:
        s.ct_mode = ct_mode
    s.ct_const = ct_const
    s.mp_alpha = mp_alpha
    s.mp_beta = mp_beta
    s.mp_curv = mp_curv
    s.weights = weights
    s.decisions = decisions
    s.positivity = positivity
    if d is not None:
        for k in range(6):
            s.d[k] = d[k] if k < len(d) else 0.0
    return s


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Tape:
    """Device tape of one recorded SSP-RK3 step (see Solver.new_tape)."""

    def __init__(self, states, data, linear):
        self.states, self.data, self.linear = states, data, linear


class Solver:
    """One grid + scheme bound to the current torch CUDA stream.

    State tensors are torch float64 CUDA tensors of shape (nvar, nz, ny, nx) with the
    leading singleton spatial axes dropped (1D: (3, nx); 2D: (4, ny, nx))."""

    def __init__(self, shape, dx, bc, scheme=None, gamma=1.4, stream=None):
        import torch
        self.shape = tuple(int(n) for n in shape)
        self.dim = len(self.shape)
        self.nv = self.dim + 2
        self.grid = make_grid(self.shape, dx, bc, gamma)
        self.scheme = scheme if scheme is not None else make_scheme(6)
        self._ctx = ctypes.c_void_p()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        st = lib().tenom_create(ctypes.byref(self._ctx), ctypes.byref(self.grid), ctypes.byref(self.scheme),
                                ctypes.c_void_p(self.stream.cuda_stream))
        if st != TENOM_OK:
            raise TenomError(st, "tenom_create")
        self.dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        self.t = torch.zeros(1, dtype=torch.float64, device="cuda")

    # numpy-style (z, y, x) shape of the state
    @property
    def state_shape(self):
        return (self.nv,) + tuple(reversed(self.shape))

    def face_shape(self, axis):
        n = list(self.shape)
        n[axis] += 1
        return tuple(reversed(n))

    def _check(self, st, what):
        if st != TENOM_OK:
            msg = lib().tenom_last_error(self._ctx)
            raise TenomError(st, "%s: %s" % (what, msg.decode() if msg else ""))

    def close(self):
        if self._ctx:
            lib().tenom_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tensor(self):
        import torch
        return torch.empty(self.state_shape, dtype=torch.float64, device="cuda")

    def init_state(self, prim):
        """prim: float64 CUDA tensor (rho, u.., p) -> conserved state tensor."""
        U = self.tensor()
        self._check(lib().tenom_init_state(self._ctx, _ptr(prim), _ptr(U)), "tenom_init_state")
        return U

    def rhs(self, U, out=None):
        out = self.tensor() if out is None else out
        self._check(lib().tenom_rhs(self._ctx, _ptr(U), _ptr(out)), "tenom_rhs")
        return out

    def max_dt(self, U, cfl=0.4, out=None):
        out = self.dt if out is None else out
        self._check(lib().tenom_max_dt(self._ctx, _ptr(U), cfl, _ptr(out)), "tenom_max_dt")
        return out

    def rk3_step(self, U, dt_dev):
        self._check(lib().tenom_rk3_step(self._ctx, _ptr(U), _ptr(dt_dev)), "tenom_rk3_step")
        return U

    def advance(self, U, nsteps, t_end=math.inf, cfl=0.4, t_dev=None):
        t_dev = self.t if t_dev is None else t_dev
        self._check(lib().tenom_advance(self._ctx, _ptr(U), _ptr(t_dev), t_end, cfl, nsteps), "tenom_advance")
        return U

    def advance_host(self, U_host_in, U_host_out, t=0.0, t_end=math.inf, cfl=0.4, nsteps=1):
        """Host buffers (numpy float64, C-contiguous, or pinned torch CPU tensors)."""
        tt = ctypes.c_double(t)

        def hp(a):
            if isinstance(a, np.ndarray):
                assert a.dtype == np.float64 and a.flags.c_contiguous
                return ctypes.c_void_p(a.ctypes.data)
            return ctypes.c_void_p(a.data_ptr())
        self._check(lib().tenom_advance_host(self._ctx, hp(U_host_in), hp(U_host_out), ctypes.byref(tt), t_end, cfl,
                                             nsteps), "tenom_advance_host")
        return tt.value

    def face_dump(self, U, axis, flags=True):
        import torch
        if not 0 <= axis < self.dim:  # let the library reject it
            dummy = torch.empty(1, dtype=torch.float64, device="cuda")
            self._check(lib().tenom_face_dump(self._ctx, _ptr(U), axis, _ptr(dummy), None), "tenom_face_dump")
        F = torch.empty((self.nv,) + self.face_shape(axis), dtype=torch.float64, device="cuda")
        fl = torch.zeros(self.face_shape(axis) + (self.nv, 2), dtype=torch.uint8, device="cuda") if flags else None
        self._check(lib().tenom_face_dump(self._ctx, _ptr(U), axis, _ptr(F), _ptr(fl) if fl is not None else None),
                    "tenom_face_dump")
        return F, fl

    def positivity_limit(self, U, axis, dt_dev, F):
        """The positivity limiter of a stage of length dt_dev applied in place to face
        fluxes F (as face_dump returns them) of one axis at the state U."""
        self._check(lib().tenom_positivity_limit(self._ctx, _ptr(U), axis, _ptr(dt_dev), _ptr(F)),
                    "tenom_positivity_limit")
        return F

    # ---- frozen-branch adjoint ----
    def flags_bytes(self):
        return int(lib().tenom_flags_bytes(self._ctx))

    def rhs_vjp(self, U, w, out=None):
        """L'(U)^T w."""
        out = self.tensor() if out is None else out
        self._check(lib().tenom_rhs_vjp(self._ctx, _ptr(U), _ptr(w), _ptr(out)), "tenom_rhs_vjp")
        return out

    def lin_tape_bytes(self):
        """Bytes of the linearisation one operator evaluation records."""
        return int(lib().tenom_lin_tape_bytes(self._ctx))

    def rhs_record(self, U, lin, out=None):
        """L(U), also recording its linearisation into `lin` (lin_tape_bytes() bytes)."""
        out = self.tensor() if out is None else out
        self._check(lib().tenom_rhs_record(self._ctx, _ptr(U), _ptr(out), _ptr(lin)), "tenom_rhs_record")
        return out

    def rhs_vjp_lin(self, U, lin, w, out=None):
        """L'(U)^T w from the linearisation rhs_record wrote at U."""
        out = self.tensor() if out is None else out
        self._check(lib().tenom_rhs_vjp_lin(self._ctx, _ptr(U), _ptr(lin), _ptr(w), _ptr(out)), "tenom_rhs_vjp_lin")
        return out

    def new_lin(self):
        import torch
        return torch.empty(self.lin_tape_bytes() // 8, dtype=torch.float64, device="cuda")

    def tape_bytes(self, linear=False):
        """Device bytes of one step's tape (stage states + flags or linearisation)."""
        per_stage = self.lin_tape_bytes() if linear else self.flags_bytes()
        return 2 * 8 * self.nv * int(math.prod(self.shape)) + 3 * per_stage

    def new_tape(self, linear=False):
        """Tape of one SSP-RK3 step: the stage states U1, U2 and, per stage, the cutoff flags
        (compact; the reverse rebuilds the frozen reconstructions) or the linearisation
        (linear=True: larger; the reverse reads it)."""
        import torch
        states = torch.empty((2,) + self.state_shape, dtype=torch.float64, device="cuda")
        if linear:
            return Tape(states, torch.empty(3 * self.lin_tape_bytes() // 8, dtype=torch.float64, device="cuda"), True)
        return Tape(states, torch.empty(3 * self.flags_bytes(), dtype=torch.uint8, device="cuda"), False)

    def rk3_step_record(self, U, dt_dev, tape):
        if tape.linear:
            st = lib().tenom_rk3_step_record_lin(self._ctx, _ptr(U), _ptr(dt_dev), _ptr(tape.states), _ptr(tape.data))
        else:
            st = lib().tenom_rk3_step_record(self._ctx, _ptr(U), _ptr(dt_dev), _ptr(tape.states), _ptr(tape.data))
        self._check(st, "tenom_rk3_step_record")
        return U

    def rk3_step_adjoint(self, U_n, dt_dev, Ubar_np1, tape=None, out=None):
        out = self.tensor() if out is None else out
        if tape is None:
            st = lib().tenom_rk3_step_adjoint(self._ctx, _ptr(U_n), _ptr(dt_dev), _ptr(Ubar_np1), _ptr(out))
        elif tape.linear:
            st = lib().tenom_rk3_step_adjoint_lin(self._ctx, _ptr(U_n), _ptr(tape.states), _ptr(tape.data),
                                                  _ptr(dt_dev), _ptr(Ubar_np1), _ptr(out))
        else:
            st = lib().tenom_rk3_step_adjoint_tape(self._ctx, _ptr(U_n), _ptr(tape.states), _ptr(tape.data),
                                                   _ptr(dt_dev), _ptr(Ubar_np1), _ptr(out))
        self._check(st, "tenom_rk3_step_adjoint")
        return out

    def decision_stats(self, U, axis, counters=None):
        """Decision statistics of the reconstruction at U on the faces of one axis: adds
        the NSTATS counters (tenom_decision_stats) to `counters` (int64 CUDA tensor, made
        zero if None) and returns it."""
        import torch
        if counters is None:
            counters = torch.zeros(NSTATS, dtype=torch.int64, device="cuda")
        self._check(lib().tenom_decision_stats(self._ctx, _ptr(U), axis, _ptr(counters)), "tenom_decision_stats")
        return counters

    def status(self, reset=False):
        v = ctypes.c_int(0)
        st = lib().tenom_status_word(self._ctx, ctypes.byref(v), 1 if reset else 0)
        if st not in (TENOM_OK, TENOM_E_NONPHYSICAL):
            self._check(st, "tenom_status_word")
        return v.value

    def kernel_timing(self, enable):
        ms = ctypes.c_double(0)
        n = ctypes.c_longlong(0)
        self._check(lib().tenom_kernel_timing(self._ctx, 1 if enable else 0, ctypes.byref(ms), ctypes.byref(n)),
                    "tenom_kernel_timing")
        return ms.value, n.value


def fp64_peak(nblocks=152 * 8, iters=4096):
    f = ctypes.c_double(0)
    st = lib().tenom_fp64_peak(_stream(), nblocks, iters, ctypes.byref(f))
    if st != TENOM_OK:
        raise TenomError(st, "tenom_fp64_peak")
    return f.value


class Batch:
    """Independent 1D problems of uneven size advanced together (tenom_batch_*).

    State tensors are float64 CUDA tensors of shape (3, total): problem j owns columns
    off[j]:off[j+1]."""

    def __init__(self, n, dx, scheme=None, bc=None, gamma=1.4, stream=None):
        import torch
        self.n = np.ascontiguousarray(n, dtype=np.int32)
        self.dx = np.ascontiguousarray(dx, dtype=np.float64)
        self.P = int(self.n.size)
        self.scheme = scheme if scheme is not None else make_scheme(6)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._b = ctypes.c_void_p()
        bca = None if bc is None else np.ascontiguousarray(bc, dtype=np.int32)
        st = lib().tenom_batch_create(ctypes.byref(self._b), self.P, ctypes.c_void_p(self.n.ctypes.data),
                                      ctypes.c_void_p(self.dx.ctypes.data),
                                      None if bca is None else ctypes.c_void_p(bca.ctypes.data), gamma,
                                      ctypes.byref(self.scheme), ctypes.c_void_p(self.stream.cuda_stream))
        if st != TENOM_OK:
            raise TenomError(st, "tenom_batch_create")
        self._bc_keep = bca
        self.off = np.zeros(self.P + 1, dtype=np.int64)
        tot = ctypes.c_longlong(0)
        self._check(lib().tenom_batch_layout(self._b, ctypes.c_void_p(self.off.ctypes.data), ctypes.byref(tot)),
                    "layout")
        self.total = int(tot.value)

    def _check(self, st, what):
        if st != TENOM_OK:
            raise TenomError(st, "tenom_batch " + what)

    def close(self):
        if self._b:
            lib().tenom_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_state(self, prim):
        import torch
        U = torch.empty((3, self.total), dtype=torch.float64, device="cuda")
        self._check(lib().tenom_batch_init_state(self._b, _ptr(prim), _ptr(U)), "init_state")
        return U

    def set_time(self, t=None, t_end=None):
        ta = None if t is None else np.ascontiguousarray(np.broadcast_to(t, (self.P,)), dtype=np.float64)
        te = None if t_end is None else np.ascontiguousarray(np.broadcast_to(t_end, (self.P,)), dtype=np.float64)
        self._check(lib().tenom_batch_set_time(self._b, None if ta is None else ctypes.c_void_p(ta.ctypes.data),
                                               None if te is None else ctypes.c_void_p(te.ctypes.data)),
                    "set_time")

    def times(self):
        t = np.zeros(self.P)
        self._check(lib().tenom_batch_get_time(self._b, ctypes.c_void_p(t.ctypes.data)), "get_time")
        return t

    def step(self, U, nsteps=1, cfl=0.4, graph=True):
        fn = lib().tenom_batch_step if graph else lib().tenom_batch_step_direct
        self._check(fn(self._b, _ptr(U), cfl, nsteps), "step")
        return U

    def autotune(self, U):
        t, c = ctypes.c_int(0), ctypes.c_int(0)
        self._check(lib().tenom_batch_autotune(self._b, _ptr(U), ctypes.byref(t), ctypes.byref(c)), "autotune")
        return t.value, c.value

    def set_tiling(self, tile, ctas_per_sm):
        self._check(lib().tenom_batch_set_tiling(self._b, tile, ctas_per_sm), "set_tiling")

    def decision_stats(self, U, axis, counters=None):
        """Decision statistics of the reconstruction at U on the faces of one axis: adds
        the NSTATS counters (tenom_decision_stats) to `counters` (int64 CUDA tensor, made
        zero if None) and returns it."""
        import torch
        if counters is None:
            counters = torch.zeros(NSTATS, dtype=torch.int64, device="cuda")
        self._check(lib().tenom_decision_stats(self._ctx, _ptr(U), axis, _ptr(counters)), "tenom_decision_stats")
        return counters

    def status(self, reset=False):
        v = ctypes.c_int(0)
        st = lib().tenom_batch_status_word(self._b, ctypes.byref(v), 1 if reset else 0)
        if st not in (TENOM_OK, TENOM_E_NONPHYSICAL):
            self._check(st, "status_word")
        return v.value

