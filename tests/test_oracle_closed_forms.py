"""The closed forms used by the physics tests, checked against independent
limits (no GPU)."""
import math

import pytest

from tests import _physics as P


def test_lens_volume_limits():
    assert P.lens_volume(3.0, 2.0, 5.0) == 0.0
    assert P.lens_volume(3.0, 1.0, 0.5) == pytest.approx(4 / 3 * math.pi)
    # two equal balls of radius R at distance R share 5 pi R^3 / 12
    assert P.lens_volume(2.0, 2.0, 2.0) == pytest.approx(5 * math.pi * 8 / 12)


def test_sessile_on_sphere_reduces_to_flat_cap():
    """For a huge solid ball the drop is a spherical cap on a plane: height
    h = r (1 - cos theta), V = pi h^2 (3 r - h) / 3."""
    Rs = 1e6
    for theta in (30.0, 90.0, 150.0):
        r = 10.0
        h = r * (1 - math.cos(math.radians(theta)))
        V = math.pi * h * h * (3 * r - h) / 3
        top, rr, d = P.sessile_top_on_sphere(Rs, theta, V)
        assert rr == pytest.approx(r, rel=1e-4)
        assert top - Rs == pytest.approx(h, abs=2e-3)


def test_sessile_on_sphere_neutral_wetting():
    """theta = 90: the drop meets the solid at right angles, d^2 = Rs^2 + r^2."""
    top, r, d = P.sessile_top_on_sphere(15.0, 90.0, 5000.0)
    assert d * d == pytest.approx(15.0 ** 2 + r * r)


def test_washburn_quadratic_solves_the_ode():
    """The integrated position satisfies the speed law (finite difference)
    and reduces to z^2 - z0^2 = sigma cos(theta) H t / (3 mu) for mu2 = 0."""
    args = (0.01, 45.0, 16.0, 1 / 6, 1e-3 / 3, 768.0)
    z1 = P.washburn_z(10000.0, 0.0, 20.0, *args)
    z2 = P.washburn_z(10001.0, 0.0, 20.0, *args)
    assert z2 - z1 == pytest.approx(P.washburn_speed(0.5 * (z1 + z2), *args), rel=1e-6)
    z = P.washburn_z(5000.0, 0.0, 10.0, 0.01, 0.0, 16.0, 0.2, 0.0, 768.0)
    assert z * z - 100.0 == pytest.approx(0.01 * 16.0 * 5000.0 / (3 * 0.2), rel=1e-9)
