"""Pins of the morphing-transform oracle (oracle/morph.py, Sec. 2.2) to facts outside it: integer
shifts against np.roll, the bilinear interpolation against SciPy's map_coordinates, the inverse
mapping by its defining equation, and the special cases of the inverse transform."""

import numpy as np
import pytest

from oracle import morph
from synth import fields


def _const_T(K, ny, nx, cx, cy):
    T = np.zeros((2, K, ny, nx))
    T[0] += cx
    T[1] += cy
    return T


def test_compose_integer_shift_is_roll():
    # f o (I + c) at p is f(p + c): np.roll by -c.  Non-square grid, cx != cy: catches a transposed
    # axis or a sign error.
    rng = np.random.default_rng(1)
    f = rng.standard_normal((6, 10))
    T = _const_T(1, 6, 10, 3, -2)[:, 0]
    got = morph.compose(f, T)
    np.testing.assert_array_equal(got, np.roll(f, shift=(2, -3), axis=(0, 1)))


def test_forward_integer_shift_is_roll():
    # (I + c)^-1 is p - c, so r = u(p - c) - u_ref(p) = roll(u, +c) - u_ref, for any n_iter >= 1.
    rng = np.random.default_rng(2)
    M, K, ny, nx = 2, 3, 8, 12
    u = rng.standard_normal((M, K, ny, nx))
    u_ref = rng.standard_normal((M, ny, nx))
    T = _const_T(K, ny, nx, -5, 3)
    for n_iter in (1, 4):
        r = morph.morph_forward(u, u_ref, T, n_iter)
        want = np.roll(u, shift=(3, -5), axis=(2, 3)) - u_ref[:, None]
        np.testing.assert_allclose(r, want, rtol=0, atol=1e-14)


def test_interpolation_matches_scipy_grid_wrap():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(3)
    f = rng.standard_normal((9, 14))
    qy = rng.uniform(-20, 30, size=50)
    qx = rng.uniform(-20, 30, size=50)
    got = morph.interp_periodic(f, qy, qx)
    want = ndimage.map_coordinates(f, [qy, qx], order=1, mode="grid-wrap")
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_compose_random_displacement_matches_scipy():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(4)
    ny, nx = 16, 24
    f = rng.standard_normal((ny, nx))
    T = rng.uniform(-3, 3, size=(2, ny, nx))
    py, px = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    want = ndimage.map_coordinates(f, [py + T[1], px + T[0]], order=1, mode="grid-wrap")
    np.testing.assert_allclose(morph.compose(f, T), want, rtol=0, atol=1e-12)


def test_inverse_points_solve_defining_equation():
    # q + T(q) = p at every node for a smooth contraction (max |grad T| well below 1).
    ndimage = pytest.importorskip("scipy.ndimage")
    ny, nx = 32, 48
    T = fields.smooth_mappings(5, 1, ny, nx, amp=2.0, ell=8.0)[:, 0].astype(np.float64)
    qy, qx = morph.inverse_points(T, 60)
    ty = ndimage.map_coordinates(T[1], [qy, qx], order=1, mode="grid-wrap")
    tx = ndimage.map_coordinates(T[0], [qy, qx], order=1, mode="grid-wrap")
    py, px = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    assert np.abs(qy + ty - py).max() < 1e-10
    assert np.abs(qx + tx - px).max() < 1e-10
    # zero iterations leave the nodes in place
    qy0, qx0 = morph.inverse_points(T, 0)
    np.testing.assert_array_equal(qy0, py)
    np.testing.assert_array_equal(qx0, px)


def test_inverse_with_zero_mapping_adds_residual():
    rng = np.random.default_rng(6)
    M, K, ny, nx = 2, 3, 6, 8
    ext = rng.standard_normal((M + 2, K, ny, nx))
    ext[:2] = 0.0
    u_ref = rng.standard_normal((M, ny, nx))
    np.testing.assert_allclose(morph.morph_inverse(ext, u_ref), u_ref[:, None] + ext[2:], rtol=0, atol=1e-15)


def test_round_trip_integer_shift_is_exact():
    rng = np.random.default_rng(7)
    M, K, ny, nx = 3, 2, 10, 6
    u = rng.standard_normal((M, K, ny, nx))
    u_ref = rng.standard_normal((M, ny, nx))
    T = _const_T(K, ny, nx, 2, -7)
    ext = np.concatenate([T, morph.morph_forward(u, u_ref, T, 2)])
    np.testing.assert_allclose(morph.morph_inverse(ext, u_ref), u, rtol=0, atol=1e-13)


def test_round_trip_smooth_mapping_is_close():
    # Smooth fields and mappings: forward then inverse returns the members up to the bilinear
    # interpolation error, which is small against the fields' unit scale.
    M, K, ny, nx = 1, 2, 64, 64
    u = fields.smooth_members(8, M, K, ny, nx, ell=12.0).astype(np.float64)
    u_ref = fields.smooth_members(9, M, 1, ny, nx, ell=12.0)[:, 0].astype(np.float64)
    T = fields.smooth_mappings(10, K, ny, nx, amp=1.5, ell=10.0).astype(np.float64)
    ext = np.concatenate([T, morph.morph_forward(u, u_ref, T, 40)])
    err = np.abs(morph.morph_inverse(ext, u_ref) - u).max()
    assert err < 0.05 * np.abs(u).max()


def test_reference_is_member_mean():
    rng = np.random.default_rng(11)
    one = rng.standard_normal((5, 1, 4, 6))
    np.testing.assert_allclose(morph.morph_reference(np.repeat(one, 7, axis=1)), one, rtol=0, atol=1e-15)
    ext = rng.standard_normal((5, 3, 4, 6))
    np.testing.assert_allclose(morph.morph_reference(ext)[:, 0], (ext[:, 0] + ext[:, 1] + ext[:, 2]) / 3,
                               rtol=0, atol=1e-15)


def test_tolerance_stop():
    # tol beyond any step: every point stops after the first step, as with n_iter = 1; a small tol
    # still solves the defining equation closely.
    ndimage = pytest.importorskip("scipy.ndimage")
    ny, nx = 32, 40
    rng = np.random.default_rng(12)
    u = rng.standard_normal((1, 2, ny, nx))
    u_ref = rng.standard_normal((1, ny, nx))
    T = fields.smooth_mappings(13, 2, ny, nx, amp=2.0, ell=8.0).astype(np.float64)
    np.testing.assert_array_equal(morph.morph_forward(u, u_ref, T, 20, tol=1e9), morph.morph_forward(u, u_ref, T, 1))
    np.testing.assert_array_equal(morph.morph_forward(u, u_ref, T, 20, tol=0.0), morph.morph_forward(u, u_ref, T, 20))
    qy, qx = morph.inverse_points(T[:, 0], 60, tol=1e-9)
    ty = ndimage.map_coordinates(T[1, 0], [qy, qx], order=1, mode="grid-wrap")
    tx = ndimage.map_coordinates(T[0, 0], [qy, qx], order=1, mode="grid-wrap")
    py, px = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    assert np.abs(qy + ty - py).max() < 1e-8 and np.abs(qx + tx - px).max() < 1e-8
