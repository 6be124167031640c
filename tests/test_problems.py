"""The seeded input generators (CPU): shapes, ranges and determinism of the initial states
that both the CUDA path and the oracle are fed from."""
import numpy as np

from paper_2010_13289_gb300 import problems as PB


def test_le_blanc_initial_state():
    """Eq. Leblanc: (1, 0, 2/3 1e-1) on x < 3 and (1e-3, 0, 2/3 1e-10) on x >= 3 of [0, 9]."""
    prim, dx = PB.le_blanc_1d(900)
    assert prim.shape == (3, 900) and dx == 9.0 / 900
    x = (np.arange(900) + 0.5) * dx
    left = x < 3.0
    assert np.all(prim[0][left] == 1.0) and np.all(prim[0][~left] == 1e-3)
    assert np.all(prim[1] == 0.0)
    assert np.all(prim[2][left] == 2.0 / 3.0 * 1e-1) and np.all(prim[2][~left] == 2.0 / 3.0 * 1e-10)
    assert left.sum() == 300


def test_near_vacuum_ranges_blocks_and_seed():
    for shape in ((128,), (24, 20), (10, 12, 8)):
        D = len(shape)
        a, b = PB.near_vacuum(shape, 3), PB.near_vacuum(shape, 3)
        assert a.shape == (D + 2,) + shape and np.array_equal(a, b)
        assert not np.array_equal(a, PB.near_vacuum(shape, 4))
        assert 1e-3 <= a[0].min() and a[0].max() <= 1.0
        assert 1e-10 <= a[-1].min() and a[-1].max() <= 1e-1
        assert np.abs(a[1:1 + D]).max() <= 1.0
        # piecewise constant on 4-cell blocks along the fastest axis
        x = a[0].reshape(-1, shape[-1])
        for c in range(0, shape[-1] - 1):
            if (c + 1) % 4:
                assert np.array_equal(x[:, c], x[:, c + 1])


def test_taylor_green_initial_state():
    """Eq. TGV at cell centres of [0, 2 pi]^3: rho = 1, w = 0, divergence-free velocity."""
    prim, dx = PB.taylor_green_3d(16)
    assert prim.shape == (5, 16, 16, 16) and np.isclose(dx, 2 * np.pi / 16)
    assert np.all(prim[0] == 1.0) and np.all(prim[3] == 0.0)
    # spectral divergence of (u, v) is zero to rounding
    k = np.fft.fftfreq(16, d=1.0 / 16)
    Kz, Ky, Kx = np.meshgrid(k, k, k, indexing="ij")
    div = Kx * np.fft.fftn(prim[1]) + Ky * np.fft.fftn(prim[2])
    assert np.abs(div).max() < 1e-10 * np.abs(np.fft.fftn(prim[1])).max()
    assert abs(prim[4].mean() - (100.0 - 2.0 / 16)) < 1e-12  # the cosines average to zero
