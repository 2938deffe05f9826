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
