"""Pins of the oracle's breathing-motion resampling (Sec. "Consideration of
Breathing Motion", Eq. breathing: T(x) = T_ref(x + u_inv(x)), trilinear, clamped
to the grid) against identities and an independent library routine."""
import numpy as np
import pytest
from scipy import ndimage

import oracle
import phantoms as ph


def _theta(shape, seed=0):
    return np.random.default_rng(seed).normal(0.0, 10.0, size=shape)


def test_zero_field_is_identity():
    th = _theta((7, 9, 11))
    u = np.zeros((3,) + th.shape, np.float32)
    assert np.array_equal(oracle.warp_temperature(th, u, 1e-3, 37.0), th + 37.0)


@pytest.mark.parametrize("axis,k", [(0, 3), (1, -2), (2, 4)])
def test_integer_shift_with_clamp(axis, k):
    th = _theta((8, 9, 10), 1)
    h = 2.0 ** -11                               # k h is exact in float32
    u = np.zeros((3,) + th.shape, np.float32)
    u[axis] = k * h
    out = oracle.warp_temperature(th, u, h, 0.0)
    arr_axis = 2 - axis                          # u component x/y/z -> array axis 2/1/0
    n = th.shape[arr_axis]
    idx = np.clip(np.arange(n) + k, 0, n - 1)
    assert np.allclose(out, np.take(th, idx, axis=arr_axis), rtol=0, atol=1e-12)


def test_affine_field_reproduced_exactly():
    nz, ny, nx = 12, 10, 14
    h = 1e-3
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    a = np.array([0.7, -1.3, 2.1, 5.0])
    th = a[0] * x + a[1] * y + a[2] * z + a[3]
    rng = np.random.default_rng(2)
    d = rng.uniform(-2.0, 2.0, size=(3, nz, ny, nx))
    # keep every sample inside the grid (a margin covers the float32 rounding of u)
    for c, n, dd in ((x, nx, d[0]), (y, ny, d[1]), (z, nz, d[2])):
        np.clip(dd, -c + 0.01, n - 1.01 - c, out=dd)
    u = (d * h).astype(np.float32)
    dd = u.astype(np.float64) / h
    expect = a[0] * (x + dd[0]) + a[1] * (y + dd[1]) + a[2] * (z + dd[2]) + a[3]
    assert np.allclose(oracle.warp_temperature(th, u, h, 0.0), expect, rtol=0, atol=1e-12)


def test_matches_scipy_map_coordinates():
    nz, ny, nx = 9, 13, 11
    h = 0.75e-3
    th = _theta((nz, ny, nx), 3)
    rng = np.random.default_rng(4)
    u = (rng.uniform(-4.0, 4.0, size=(3, nz, ny, nx)) * h).astype(np.float32)  # some samples leave the grid
    u[0, 0, 0, 0] = np.nan                                                       # non-finite: low face
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    d = u.astype(np.float64) / h
    d[0, 0, 0, 0] = -(nx + 1.0)
    coords = np.stack([z + d[2], y + d[1], x + d[0]])
    ref = ndimage.map_coordinates(th, coords, order=1, mode="nearest")
    assert np.allclose(oracle.warp_temperature(th, u, h, 0.0), ref, rtol=0, atol=1e-12)


def test_breathing_field_is_a_diffeomorphism():
    case = ph.single_needle_case(seed=0, n=48, nsteps=1)
    for t in (0.0, 1.0, 2.0):
        u = ph.breathing_field(case, t).astype(np.float64) / case.h
        # Jacobian of x -> x + d(x) by central differences (voxel units)
        J = np.zeros((3, 3) + u.shape[1:])
        for comp in range(3):
            gz, gy, gx = np.gradient(u[comp])
            J[comp, 0], J[comp, 1], J[comp, 2] = gx, gy, gz
        for k in range(3):
            J[k, k] += 1.0
        det = np.linalg.det(np.moveaxis(J, (0, 1), (-2, -1)))
        assert det.min() > 0.5
        if t == 0.0:
            assert np.abs(u).max() == 0.0
