"""Input fields evaluated at caller-supplied coordinates (no FE arithmetic here)."""
import numpy as np

from .rng import uniform_pm1, uniform_01


def sphere_distance(x, y, z, centre=(0.5, 0.5, 0.5), radius=0.3):
    """Signed distance to a sphere, positive inside (the dense/liquid side)."""
    return radius - np.sqrt((x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2)


def wavy_plane_phases(seed):
    """Two seeded phases in [0, 2*pi) for the perturbed planar interface."""
    u = uniform_01(seed, 2)
    return 2.0 * np.pi * u[0], 2.0 * np.pi * u[1]


def wavy_plane_distance(x, y, z, theta1, theta2, z0=0.5, amplitude=0.05):
    """Vertical distance to z = z0 + A sin(2 pi x + t1) sin(2 pi y + t2), positive below."""
    zg = z0 + amplitude * np.sin(2.0 * np.pi * x + theta1) * np.sin(2.0 * np.pi * y + theta2)
    return zg - z


def _assoc_legendre(lmax, t):
    """Schmidt-scaled associated Legendre functions P_l^m(t), 0 <= m <= l <= lmax."""
    from math import factorial, sqrt
    s = np.sqrt(np.maximum(0.0, 1.0 - t * t))
    P = {}
    for m in range(lmax + 1):
        pmm = np.ones_like(t)
        for k in range(1, m + 1):
            pmm = pmm * (2 * k - 1) * s
        P[(m, m)] = pmm
        if m + 1 <= lmax:
            P[(m + 1, m)] = t * (2 * m + 1) * pmm
        for l in range(m + 2, lmax + 1):
            P[(l, m)] = ((2 * l - 1) * t * P[(l - 1, m)] - (l + m - 1) * P[(l - 2, m)]) / (l - m)
    for (l, m) in list(P):
        P[(l, m)] = P[(l, m)] * sqrt(factorial(l - m) / factorial(l + m))
    return P


def _harmonic_sum(theta, varphi, coeffs, lmax):
    t = np.cos(theta)
    P = _assoc_legendre(lmax, t)
    S = np.zeros_like(theta)
    idx = 0
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            ang = np.cos(m * varphi) if m >= 0 else np.sin(-m * varphi)
            S = S + coeffs[idx] * P[(l, abs(m))] * ang
            idx += 1
    return S


def deformed_sphere_distance(x, y, z, seed, lmax=6, amplitude=0.05, radius=0.3,
                             centre=(0.5, 0.5, 0.5)):
    """Radial pseudo-distance r(theta, varphi) - |x - c| to a sphere deformed by a seeded
    real spherical-harmonic series of degree <= lmax, normalised so that the relative
    deformation is at most ``amplitude`` (max taken on a fixed 256 x 512 angular grid)."""
    ncoef = (lmax + 1) ** 2
    coeffs = uniform_pm1(seed, ncoef)
    tg = (np.arange(256) + 0.5) * (np.pi / 256)
    pg = np.arange(512) * (2.0 * np.pi / 512)
    TG, PG = np.meshgrid(tg, pg, indexing="ij")
    smax = np.max(np.abs(_harmonic_sum(TG, PG, coeffs, lmax)))
    dx, dy, dz = x - centre[0], y - centre[1], z - centre[2]
    rr = np.sqrt(dx * dx + dy * dy + dz * dz)
    theta = np.arccos(np.clip(dz / np.maximum(rr, 1e-300), -1.0, 1.0))
    varphi = np.arctan2(dy, dx)
    S = _harmonic_sum(theta, varphi, coeffs, lmax)
    return radius * (1.0 + amplitude * S / smax) - rr


def initial_level_set(d, eps):
    """Regularised level set phi = tanh(d / (2 eps)) of Section 2.2, eq. (initial_phi)."""
    return np.tanh(d / (2.0 * eps))


_WAVES = np.array([[1, 1, 1], [1, 2, 1], [2, 1, 1], [1, 1, 2]], dtype=np.float64)


def convection_field(x, y, z, seed, lo, hi, beta_max=None):
    """Divergence-free field beta = curl(b A) of a seeded trigonometric vector potential
    A_c = sum_m a_cm sin(2 pi k_m . xi + t_cm), xi = (x - lo)/(hi - lo), times the bubble
    b = sin(pi xi_x) sin(pi xi_y) sin(pi xi_z). The bubble vanishes on every face of the box, so
    beta . n = 0 there: no flow enters or leaves through any boundary, in particular not through
    a natural (open) one, where inflow would make the convection form indefinite. The field is
    scaled so that the largest |beta| over the given points equals one (or over ``beta_max``)."""
    a = uniform_pm1(seed, 12).reshape(3, 4)
    t = 2.0 * np.pi * uniform_01(seed + 1000, 12).reshape(3, 4)
    xi = [(x - lo[0]) / (hi[0] - lo[0]), (y - lo[1]) / (hi[1] - lo[1]), (z - lo[2]) / (hi[2] - lo[2])]
    s = [np.sin(np.pi * v) for v in xi]
    c = [np.cos(np.pi * v) for v in xi]
    b = s[0] * s[1] * s[2]
    db = [np.pi * c[0] * s[1] * s[2], np.pi * s[0] * c[1] * s[2], np.pi * s[0] * s[1] * c[2]]
    A = np.zeros((3,) + np.shape(x))
    dA = np.zeros((3, 3) + np.shape(x))  # dA[c][d] = d A_c / d xi_d
    for m in range(4):
        k = _WAVES[m]
        arg = 2.0 * np.pi * (k[0] * xi[0] + k[1] * xi[1] + k[2] * xi[2])
        for cc in range(3):
            A[cc] = A[cc] + a[cc, m] * np.sin(arg + t[cc, m])
            g = a[cc, m] * np.cos(arg + t[cc, m]) * 2.0 * np.pi
            for d in range(3):
                dA[cc, d] = dA[cc, d] + g * k[d]
    # d(b A_c)/d xi_d = b dA_c/dxi_d + A_c db/dxi_d
    dbA = [[b * dA[cc, d] + A[cc] * db[d] for d in range(3)] for cc in range(3)]
    bx = dbA[2][1] - dbA[1][2]
    by = dbA[0][2] - dbA[2][0]
    bz = dbA[1][0] - dbA[0][1]
    if beta_max is None:
        beta_max = np.max(np.sqrt(bx * bx + by * by + bz * bz))
    return bx / beta_max, by / beta_max, bz / beta_max


def heat_initial_temperature(x, y, z, r_laser, z_top, t_base=500.0, t_peak_rise=2633.0):
    """Previous-step temperature: T0 + dT exp(-2 (x^2+y^2)/r^2 - 2 ((z - z_top)/r)^2)."""
    return t_base + t_peak_rise * np.exp(-2.0 * (x * x + y * y) / r_laser ** 2
                                         - 2.0 * ((z - z_top) / r_laser) ** 2)


def heat_target_temperature(x, y, z, z_top, seed, t_base=500.0, rise=2000.0,
                            r=55e-6, x0=5e-6, y0=-5e-6, noise=1.0):
    """Seeded target field of the adjoint objective: a shifted Gaussian plus U[-1,1) noise
    (one draw per point, in the caller's order)."""
    g = np.exp(-2.0 * ((x - x0) ** 2 + (y - y0) ** 2) / r ** 2 - 2.0 * ((z - z_top) / r) ** 2)
    return t_base + rise * g + noise * uniform_pm1(seed, np.size(x)).reshape(np.shape(x))


def kq_field(n_values, seed, k0):
    """Per-quadrature-point conductivity k0 * (1 + 0.25 (1 + U[-1,1))), values in [k0, 1.5 k0)."""
    return k0 * (1.0 + 0.25 * (1.0 + uniform_pm1(seed, n_values)))


def interface_temperature(x, y, z, t_base=2000.0, t_peak=3600.0, centre=(0.5, 0.5, 0.5), radius=0.2):
    """A hot spot across the interface region of the unit-cube workloads:
    T = t_base + (t_peak - t_base) exp(-2 |x - c|^2 / r^2), above the boiling point near c."""
    r2 = (x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2
    return t_base + (t_peak - t_base) * np.exp(-2.0 * r2 / radius ** 2)


def meltpool_state(x, y, z, seed, lo, hi, eps, u_max=1.0, r_hot=50e-6, t_base=500.0, t_peak=3600.0,
                   surface=0.6, amplitude=0.03):
    """Two time levels (n and n-1) of the fields of one melt-pool step on the box [lo, hi]:
    a wavy melt surface z_s = lo_z + L_z (surface + amplitude sin(2 pi xi_x + t1) sin(2 pi xi_y + t2))
    with the dense phase below (phi = tanh(d / (2 eps)), d = z_s - z; one step earlier the surface
    stood eps/4 higher), a hot spot T = t_base + (t_peak - t_base) exp(-2 rho^2/r^2 - 2 (z - z_s)^2/r^2)
    under the box centre (3 % cooler one step earlier), and the divergence-free, wall-tangential
    convection field scaled to u_max (10 % slower one step earlier)."""
    t1, t2 = wavy_plane_phases(seed)
    L = [hi[i] - lo[i] for i in range(3)]
    xi, eta = (x - lo[0]) / L[0], (y - lo[1]) / L[1]
    zs = lo[2] + L[2] * (surface + amplitude * np.sin(2.0 * np.pi * xi + t1) * np.sin(2.0 * np.pi * eta + t2))
    d = zs - z
    xc, yc = 0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1])
    g = np.exp(-2.0 * ((x - xc) ** 2 + (y - yc) ** 2) / r_hot ** 2 - 2.0 * ((z - zs) / r_hot) ** 2)
    T = t_base + (t_peak - t_base) * g
    u = u_max * np.array(convection_field(x, y, z, seed, lo, hi))
    return dict(u=u, u_prev=0.9 * u, T=T, T_prev=t_base + 0.97 * (T - t_base),
                phi=initial_level_set(d, eps), phi_prev=initial_level_set(d + 0.25 * eps, eps))
