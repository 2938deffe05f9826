"""Pins of the oracle's Gaussian-splatting render (3DGS forward equations):
closed forms for one isotropic Gaussian on the optical axis, front-to-back
compositing of two, the transmittance cut-off, culling behind the camera and
the quaternion's rotation of the scale axes."""
import numpy as np

import oracle

I3 = np.eye(3)
Z3 = np.zeros(3)


def render(mu, quat, scale, opac, color, W=32, H=32, f=40.0, bg=(0.1, 0.2, 0.3)):
    return oracle.gs_render(np.array(mu, float), np.array(quat, float), np.array(scale, float),
                            np.array(opac, float), np.array(color, float), I3, Z3, f, f, W / 2, H / 2,
                            W, H, 0.01, bg)


def test_one_isotropic_gaussian_closed_form():
    W = H = 32
    f, z0, s, o = 40.0, 2.0, 0.2, 0.8
    c, bg = np.array([0.9, 0.5, 0.1]), np.array([0.1, 0.2, 0.3])
    img, T = render([[0, 0, z0]], [[1, 0, 0, 0]], [[s, s, s]], [o], [c], W, H, f, bg)
    var = (f * s / z0) ** 2 + 0.3
    r = int(np.ceil(3 * np.sqrt(var)))
    assert int((16 - r) / 16) == 0 and int((16 + r + 15) / 16) >= 2   # both tile rows / columns covered
    py, px = np.mgrid[0:H, 0:W]
    a = np.minimum(0.99, o * np.exp(-0.5 * ((px - W / 2) ** 2 + (py - H / 2) ** 2) / var))
    a = np.where(a >= 1 / 255, a, 0.0)
    np.testing.assert_allclose(img, a[..., None] * c + (1 - a[..., None]) * bg, atol=1e-12)
    np.testing.assert_allclose(T, 1 - a, atol=1e-12)


def test_two_layers_front_to_back_and_input_order():
    red, green = [1.0, 0, 0], [0, 1.0, 0]
    args = dict(quat=[[1, 0, 0, 0]] * 2, scale=[[0.3, 0.3, 0.3]] * 2)
    img, _ = render([[0, 0, 3.0], [0, 0, 2.0]], args["quat"], args["scale"], [0.6, 0.5], [green, red])
    img2, _ = render([[0, 0, 2.0], [0, 0, 3.0]], args["quat"], args["scale"], [0.5, 0.6], [red, green])
    np.testing.assert_allclose(img, img2, atol=1e-15)
    a1, a2 = 0.5, 0.6                                      # at the centre pixel the exponent is 0
    expect = a1 * np.array(red) + (1 - a1) * a2 * np.array(green) + (1 - a1) * (1 - a2) * np.array([0.1, 0.2, 0.3])
    np.testing.assert_allclose(img[16, 16], expect, atol=1e-12)


def test_transmittance_cut_off():
    """alpha 0.95 per layer: T after 3 layers is 1.25e-4, a 4th would go below 1e-4, so the
    pixel stops there."""
    n = 6
    img, T = render([[0, 0, 2.0 + 0.1 * k] for k in range(n)], [[1, 0, 0, 0]] * n, [[0.3] * 3] * n,
                    [0.95] * n, [[1.0, 1.0, 1.0]] * n)
    np.testing.assert_allclose(T[16, 16], 0.05 ** 3, rtol=1e-12)
    np.testing.assert_allclose(img[16, 16], 0.95 * (1 + 0.05 + 0.05 ** 2) + 0.05 ** 3 * np.array([0.1, 0.2, 0.3]),
                               rtol=1e-12)


def test_behind_the_camera_is_culled():
    img, T = render([[0, 0, -1.0], [0, 0, 0.005]], [[1, 0, 0, 0]] * 2, [[0.3] * 3] * 2, [0.9, 0.9], [[1, 1, 1]] * 2)
    np.testing.assert_allclose(img, np.broadcast_to([0.1, 0.2, 0.3], img.shape), atol=0)
    assert (T == 1).all()


def test_quaternion_rotates_the_scale_axes():
    """90 degrees about the optical axis swaps the x and y extents."""
    q90 = [np.cos(np.pi / 4), 0, 0, np.sin(np.pi / 4)]
    a, _ = render([[0.1, -0.05, 2.5]], [q90], [[0.4, 0.1, 0.05]], [0.7], [[0.2, 0.8, 0.4]])
    b, _ = render([[0.1, -0.05, 2.5]], [[1, 0, 0, 0]], [[0.1, 0.4, 0.05]], [0.7], [[0.2, 0.8, 0.4]])
    np.testing.assert_allclose(a, b, atol=1e-12)


def render_flags(mu, quat, scale, opac, color, W=32, H=32, f=40.0, bg=(0.1, 0.2, 0.3)):
    return oracle.gs_render(np.array(mu, float), np.array(quat, float), np.array(scale, float),
                            np.array(opac, float), np.array(color, float), I3, Z3, f, f, W / 2, H / 2,
                            W, H, 0.01, bg, flags=True)


def test_parity_flags_leave_the_image_and_mark_the_alpha_floor():
    """The flagged render returns the plain render's image and transmittance bit for
    bit; a pixel is flagged exactly where the closed-form alpha is within the relative
    margin of the 1/255 floor (one isotropic Gaussian: no other decision is near a
    threshold for this placement)."""
    W = H = 32
    f, z0, s, o = 40.0, 2.0, 0.2, 0.8
    args = ([[0, 0, z0]], [[1, 0, 0, 0]], [[s, s, s]], [o], [[0.9, 0.5, 0.1]])
    img, T = render(*args)
    img2, T2, frag = render_flags(*args)
    assert np.array_equal(img, img2) and np.array_equal(T, T2)
    var = (f * s / z0) ** 2 + 0.3
    py, px = np.mgrid[0:H, 0:W]
    a = np.minimum(0.99, o * np.exp(-0.5 * ((px - W / 2) ** 2 + (py - H / 2) ** 2) / var))
    near_floor = np.abs(a - 1 / 255) <= 2e-3 / 255
    np.testing.assert_array_equal(frag, near_floor)


def test_parity_flags_mark_depth_ties_where_both_reach():
    """Two Gaussians at the same depth (their order decided by the index alone, which
    float32 depths need not reproduce): flagged are exactly the pixels both reach and
    the pixels where either alpha is within the margin of the 1/255 floor."""
    W, H = 48, 32
    mu = [[-0.15, 0, 2.0], [0.15, 0, 2.0]]
    img, T, frag = render_flags(mu, [[1, 0, 0, 0]] * 2, [[0.1] * 3] * 2, [0.7, 0.7],
                                [[1, 0, 0], [0, 0, 1]], W, H)
    f, var = 40.0, (40.0 * 0.1 / 2.0) ** 2 + 0.3
    py, px = np.mgrid[0:H, 0:W]
    a = [np.minimum(0.99, 0.7 * np.exp(-0.5 * ((px - (W / 2 + f * x / 2.0)) ** 2 + (py - H / 2) ** 2) / var))
         for x in (-0.15, 0.15)]
    both = (a[0] >= 1 / 255) & (a[1] >= 1 / 255)
    floor = (np.abs(a[0] - 1 / 255) <= 2e-3 / 255) | (np.abs(a[1] - 1 / 255) <= 2e-3 / 255)
    assert both.any() and ((a[0] >= 1 / 255) & ~both).any()
    np.testing.assert_array_equal(frag, both | floor)


def test_parity_flags_mark_the_tile_column_a_radius_step_moves():
    """A Gaussian whose 3-sigma radius is an integer to float64 precision (where a
    float32 ceil may give the next one), placed so that the radius step moves its tile
    square's left edge by one tile column: the pixels of that column the Gaussian reaches
    are flagged, the centre and the far corners are not."""
    W = H = 128
    f, z0, o = 40.0, 2.0, 0.9
    # 3 sqrt(lam) = 30: lam = 100 = mid + sqrt(0.1) (the eigenvalue floor), mid = (f s / z0)^2 + 0.3
    s = np.sqrt(100.0 - np.sqrt(0.1) - 0.3) * z0 / f
    # on the optical axis with the principal point at u = 78.5: the left edge (u - r) / 16 is
    # 3.03 for r = 30 and 2.97 for r = 31
    img, T, frag = oracle.gs_render(np.array([[0, 0, z0]], float), np.array([[1, 0, 0, 0]], float),
                                    np.array([[s, s, s]]), np.array([o]), np.array([[0.2, 0.4, 0.6]]),
                                    I3, Z3, f, f, 78.5, 64.0, W, H, 0.01, (0.1, 0.2, 0.3), flags=True)
    var = 100.0 - np.sqrt(0.1)
    assert o * np.exp(-0.5 * 31.5 ** 2 / var) >= 1 / 255          # pixel 47 of column 2 is reached
    assert frag[64, 47]
    assert not frag[64, 70:88].any()                              # around the centre (u = 78.5)
    assert not frag[:16, :16].any() and not frag[112:, 112:].any()


def test_parity_flags_ignore_a_radius_step_that_moves_no_tile_edge():
    """The same radius at a centre where r -> r + 1 leaves every tile edge in place
    ((u - r) / 16 = 2.25 either way): no tile column is flagged, only the ring where
    alpha meets the 1/255 floor."""
    W = H = 96
    f, z0, o = 40.0, 2.0, 0.5
    s = np.sqrt(16.0 - np.sqrt(0.1) - 0.3) * z0 / f
    img, T, frag = render_flags([[0, 0, z0]], [[1, 0, 0, 0]], [[s, s, s]], [o], [[0.2, 0.4, 0.6]], W, H)
    var = 16.0 - np.sqrt(0.1)
    py, px = np.mgrid[0:H, 0:W]
    a = np.minimum(0.99, o * np.exp(-0.5 * ((px - 48) ** 2 + (py - 48) ** 2) / var))
    np.testing.assert_array_equal(frag, np.abs(a - 1 / 255) <= 2e-3 / 255)
