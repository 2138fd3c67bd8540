"""Properties of the seeded input generators that the operators rely on (no GPU)."""
import numpy as np

import synthetic as syn


def _field(x, y, z):
    return np.array(syn.convection_field(x, y, z, 7, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), beta_max=1.0))


def test_convection_field_is_tangential_on_every_face():
    g = np.linspace(0.0, 1.0, 9)
    a, b = np.meshgrid(g, g, indexing="ij")
    a, b = a.ravel(), b.ravel()
    zero, one = np.zeros_like(a), np.ones_like(a)
    faces = [((zero, a, b), 0), ((one, a, b), 0), ((a, zero, b), 1), ((a, one, b), 1), ((a, b, zero), 2),
             ((a, b, one), 2)]
    scale = np.abs(_field(*np.random.default_rng(0).random((3, 200)))).max()
    for (x, y, z), normal in faces:
        beta = _field(x, y, z)
        assert np.abs(beta[normal]).max() <= 1e-13 * scale
        # the tangential flow along a face is not identically zero
        assert np.abs(np.delete(beta, normal, axis=0)).max() > 1e-3 * scale


def test_convection_field_is_divergence_free():
    rng = np.random.default_rng(1)
    x, y, z = rng.uniform(0.05, 0.95, (3, 64))
    h = 1e-5
    div = ((_field(x + h, y, z)[0] - _field(x - h, y, z)[0]) + (_field(x, y + h, z)[1] - _field(x, y - h, z)[1])
           + (_field(x, y, z + h)[2] - _field(x, y, z - h)[2])) / (2 * h)
    grad_scale = np.abs(_field(x + h, y, z)[0] - _field(x - h, y, z)[0]).max() / (2 * h)
    assert np.abs(div).max() <= 1e-6 * max(grad_scale, 1.0)


def test_convection_field_scaled_to_unit_maximum():
    g = np.linspace(0.0, 1.0, 11)
    x, y, z = (v.ravel() for v in np.meshgrid(g, g, g, indexing="ij"))
    beta = np.array(syn.convection_field(x, y, z, 3, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)))
    assert abs(np.sqrt((beta ** 2).sum(0)).max() - 1.0) <= 1e-15
