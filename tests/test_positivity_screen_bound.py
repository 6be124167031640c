"""The positivity kernel's FP32 early-exit screen (screen_fp32 in csrc/tenom_positivity.cuh) claims a
proof: when it returns true, the exact one-sided state W = U + m F has density >= 2e-13 and
pressure >= 2e-13.  Its error bound is restated here in numpy float32 with the kernel's
operations (truncating FP64 -> FP32 conversion, fused multiply-adds, the 1e-5 headroom) and
checked against exact rational arithmetic on random states near both thresholds.  CPU only;
the kernel itself is checked against the oracle by tests/test_gpu_positivity.py."""
from fractions import Fraction

import numpy as np

f32 = np.float32


def rz(x):
    """FP64 -> FP32 toward zero; below the normal range a signed zero, above it infinity."""
    f = f32(x)
    if not np.isfinite(f):
        return f32(np.copysign(np.inf, x))
    if abs(float(f)) > abs(x):
        f = np.nextafter(f, f32(0))
    if abs(float(f)) < 1.17549435e-38:
        return f32(np.copysign(0.0, x))
    return f


def fmaf(a, b, c):
    return f32(float(a) * float(b) + float(c))


def screen(U, F, m, gm1f):
    nv = len(U)
    w, M = [], []
    for v in range(nv):
        a, f = rz(U[v]), rz(F[v])
        w.append(fmaf(m, f, a))
        M.append(f32(f32(abs(a)) + f32(abs(f32(m * f)))) + f32(1e-30))
    m2, Bm = f32(0), f32(0)
    for d in range(1, nv - 1):
        m2 = fmaf(w[d], w[d], m2)
        Bm = fmaf(M[d], f32(abs(w[d]) + M[d]), Bm)
    pe = f32(w[0] * w[-1])
    rp = f32(gm1f * f32(pe - f32(0.5) * m2))
    B = f32(gm1f * f32(M[0] * f32(abs(w[-1]) + M[-1]) + M[-1] * f32(abs(w[0]) + M[0]) + Bm + abs(pe)
                       + f32(0.5) * m2))
    return (bool(f32(w[0] - f32(1e-5) * M[0]) >= f32(2.0001e-13))
            and bool(f32(rp - f32(1e-5) * B) >= f32(f32(2.0001e-13) * f32(w[0] + f32(1e-5) * M[0]))))


def test_fp32_screen_never_proves_a_false_exit():
    rng = np.random.default_rng(0)
    gm1 = 0.4
    gm1f = rz(gm1)
    proven = 0
    for _ in range(6000):
        nv = int(rng.integers(3, 6))
        rho = 10 ** rng.uniform(-14, 0)
        vel = rng.uniform(-1, 1, nv - 2) * 10 ** rng.uniform(-3, 1)
        p = 10 ** rng.uniform(-14, -1)
        U = [rho] + list(rho * vel) + [p / gm1 + 0.5 * rho * float((vel ** 2).sum())]
        mu = 10 ** rng.uniform(-3, 3)
        F = [x * rng.uniform(-1, 1) * 10 ** rng.uniform(-3, 0) / mu for x in U]
        m = -mu if rng.random() < 0.5 else mu
        if screen(U, F, rz(m), gm1f):
            proven += 1
            W = [Fraction(U[v]) + Fraction(m) * Fraction(F[v]) for v in range(nv)]
            m2 = sum(W[d] * W[d] for d in range(1, nv - 1))
            assert W[0] >= Fraction(2e-13)
            assert Fraction(gm1) * (W[0] * W[-1] - m2 / 2) >= Fraction(2e-13) * W[0]
    assert proven > 3000  # the screen does prove most of these states
