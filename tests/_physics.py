"""Closed forms the GPU physics tests compare against (textbook geometry
and the paper's Lucas-Washburn law); no simulation code."""
import math


def lens_volume(R, r, d):
    """Volume common to two balls of radii R and r whose centres are d apart."""
    if d >= R + r:
        return 0.0
    if d <= abs(R - r):
        return 4.0 / 3.0 * math.pi * min(R, r) ** 3
    return (math.pi * (R + r - d) ** 2 *
            (d * d + 2 * d * r - 3 * r * r + 2 * d * R + 6 * r * R - 3 * R * R) / (12.0 * d))


def sessile_top_on_sphere(Rs, theta_deg, V):
    """Drop of volume V resting on top of a solid ball of radius Rs with
    contact angle theta (measured inside the drop): the drop is a ball of
    radius r whose centre lies d = sqrt(Rs^2 + r^2 - 2 Rs r cos theta) from
    the solid's centre (law of cosines at the contact line, where the two
    outward normals make the angle theta), and its volume outside the solid
    is V.  Returns (height of the drop's top above the solid's centre, r, d)."""
    c = math.cos(math.radians(theta_deg))

    def vol(r):
        d = math.sqrt(Rs * Rs + r * r - 2 * Rs * r * c)
        return 4.0 / 3.0 * math.pi * r ** 3 - lens_volume(Rs, r, d)

    lo, hi = 1e-9, Rs + 10.0 * V ** (1.0 / 3.0)
    for _ in range(200):  # vol(r) increases with r
        m = 0.5 * (lo + hi)
        lo, hi = (lo, m) if vol(m) > V else (m, hi)
    r = 0.5 * (lo + hi)
    d = math.sqrt(Rs * Rs + r * r - 2 * Rs * r * c)
    return d + r, r, d


def washburn_speed(z, sigma, theta_deg, H, mu1, mu2, L):
    """Front speed of the viscous capillary filling of a slit of height H
    and length L (the paper's Sec. IV B balance, no applied pressure):
    [mu1 z + mu2 (L - z)] dz/dt = sigma cos(theta) H / 6."""
    return sigma * math.cos(math.radians(theta_deg)) * H / 6.0 / (mu1 * z + mu2 * (L - z))


def washburn_z(t, t0, z0, sigma, theta_deg, H, mu1, mu2, L):
    """Front position at time t >= t0 from the integrated (quadratic) form
    of the same balance, starting at z0 at t0."""
    a = 0.5 * (mu1 - mu2)
    b = mu2 * L
    c = -sigma * math.cos(math.radians(theta_deg)) * H * (t - t0) / 6.0 - a * z0 * z0 - b * z0
    if abs(a) < 1e-300:
        return -c / b
    return (-b + math.sqrt(b * b - 4 * a * c)) / (2 * a)
