"""The kernels' Newton-Raphson reciprocal and reciprocal square root against CUDA's
correctly rounded 1.0/x and sqrt(x), over the exponent range the method meets; the
integer-pipe FP64 -> FP32 truncation used by the certified cutoff filter."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_newton_reciprocal_and_sqrt_within_two_ulp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2010_13289_gb300 import tenom as T
    rng = np.random.default_rng(0)
    x = np.concatenate([10.0 ** rng.uniform(-300, 300, 200000), 1e-40 + 10.0 ** rng.uniform(-60, -30, 20000),
                        rng.uniform(0.5, 2.0, 20000), [1.0, 2.0, 0.1, 1e-40, 3.0]])
    xd = torch.from_numpy(x).cuda()
    out = torch.empty(6 * x.size, dtype=torch.float64, device="cuda")
    st = T.lib().tenom_check_fastmath(ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(out.data_ptr()), x.size,
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == T.TENOM_OK
    o = out.cpu().numpy().reshape(-1, 6)
    ulp_r = np.abs(o[:, 0] - o[:, 1]) / np.spacing(np.abs(o[:, 1]))
    ulp_s = np.abs(o[:, 2] - o[:, 3]) / np.spacing(np.abs(o[:, 3]))
    assert np.all(np.isfinite(o[:, :5]))
    assert ulp_r.max() <= 2.0, ulp_r.max()
    assert ulp_s.max() <= 2.0, ulp_s.max()
    # one Newton step (used only where a comparison follows): relative error <= 1e-12
    rel1 = np.abs(o[:, 4] - o[:, 1]) / np.abs(o[:, 1])
    assert rel1.max() <= 1e-12, rel1.max()
    # CUDA's 1/x and sqrt are correctly rounded: the host agrees with them exactly
    np.testing.assert_array_equal(o[:, 1], 1.0 / x)
    np.testing.assert_array_equal(o[:, 3], np.sqrt(x))

    # FP32 truncation toward zero: the largest-magnitude float not above |x| in the float
    # range, a signed zero below it, infinity above it
    xs = np.where(np.arange(x.size) % 2 == 1, -x, x)
    y = o[:, 5]
    f32max, f32tiny = float(np.finfo(np.float32).max), float(np.finfo(np.float32).tiny)
    big, small = np.abs(xs) >= 2.0 ** 128, np.abs(xs) < f32tiny
    mid = ~big & ~small
    assert np.all(np.isinf(y[big])) and np.all(np.sign(y[big]) == np.sign(xs[big]))
    assert np.all(y[small] == 0.0) and np.all(np.signbit(y[small]) == np.signbit(xs[small]))
    y32 = y[mid].astype(np.float32)
    np.testing.assert_array_equal(y32.astype(np.float64), y[mid])  # exactly representable
    assert np.all(np.abs(y[mid]) <= np.abs(xs[mid])) and np.all(np.sign(y[mid]) == np.sign(xs[mid]))
    up = np.nextafter(y32, (np.sign(xs[mid]) * np.inf).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(up) > np.abs(xs[mid]))
