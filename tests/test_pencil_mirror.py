"""Index arithmetic of the pencil pass's mirror pairing, checked on the host.

For even Nx the pencil kernel (csrc/rism3d_kernels.cuh, k_pencil) gives one thread a
frequency index xx and its mirror xp and contracts both with one interpolation of the
Eq. 13 table, which is exact only if the two have the same |k|. The kernel computes
kx = ks0 (signed(xx) + hs) in the working precision (hs = 1/2 on the half-integer grid of
the numerical-procedure section), so the pairing needs kx(xp) == -kx(xx) bit for bit; then
kx^2 (with or without a fused multiply-add) and everything after it agree. These tests
walk the same item range and mirror rule over every even Nx up to 512, in FP32 and FP64,
and check that every x index is contracted exactly once."""
import numpy as np
import pytest


def _signed(i, n):
    return i if 2 * i < n else i - n


def _items(nx, half):
    """(xx, xp) per item, as the kernel forms them for even Nx."""
    nxh = nx // 2 if half else nx // 2 + 1
    for xx in range(nxh):
        xp = nx - 1 - xx if half else (0 if xx == 0 else nx - xx)
        yield xx, xp


@pytest.mark.parametrize("half", [False, True])
def test_every_x_contracted_once(half):
    for nx in range(2, 513, 2):
        seen = np.zeros(nx, dtype=int)
        for xx, xp in _items(nx, half):
            assert 0 <= xp < nx
            seen[xx] += 1
            if xp != xx:
                seen[xp] += 1
        assert np.all(seen == 1), (nx, half, np.flatnonzero(seen != 1))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("half", [False, True])
def test_mirror_has_the_opposite_kx_exactly(dtype, half):
    hs = dtype(0.5) if half else dtype(0.0)
    for nx in range(2, 513, 2):
        for spacing in (0.375, 0.5, 0.55):
            ks0 = dtype(2.0 * np.pi / (nx * spacing))
            for xx, xp in _items(nx, half):
                if xp == xx:          # xx = 0 and Nx/2 on the integer grid: one point
                    continue
                kx = ks0 * (dtype(_signed(xx, nx)) + hs)
                kp = ks0 * (dtype(_signed(xp, nx)) + hs)
                assert kp.dtype == dtype and kp == -kx, (nx, spacing, xx, xp, kx, kp)
