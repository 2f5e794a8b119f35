"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no part of the method: it draws particle sets, cameras,
transfer functions and pixel samples.  Both the CUDA path and the oracle are
fed from here.  The paper's only rendered data set (an unnamed SPH temperature
field) is not available, so these sets stand in for it:

* ``uniform_cube``     -- N particles uniform in [0,1]^3, constant h, value U[0,1],
                          mass 1/N, density 1 (the small parity case).
* ``halo_mixture``     -- Plummer-profile halos plus a uniform background; h is the
                          expected distance to the 32nd nearest neighbour from the
                          analytic number density, the value is the analytic mass
                          density (what an SPH density estimate converges to).
* ``halo_mixture_knn`` -- the same positions, prepared the way an SPH code would:
                          h = the distance to the 32nd nearest neighbour (a k-d
                          tree query), value = density = the SPH density
                          estimate over those neighbours (mass 1/N).
* ``dam_break_slab``   -- a dense, floor-graded lower layer plus a sparse splash,
                          h clamped to [1e-4, 1e-2].

Every generator takes an explicit seed and uses numpy's PCG64.
"""
import math

import numpy as np

BASE_SEED = 2401028960


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def uniform_cube(n=1000, h=0.08, seed=BASE_SEED + 0):
    r = _rng(seed)
    pos = r.random((n, 3), dtype=np.float64).astype(np.float32)
    val = r.random(n, dtype=np.float64).astype(np.float32)
    return dict(
        pos=pos,
        h=np.full(n, h, np.float32),
        mass=np.full(n, 1.0 / n, np.float32),
        density=np.ones(n, np.float32),
        value=val,
    )


def _plummer_radius(r, a, n, trunc=10.0):
    """Plummer-profile radii (cumulative mass fraction X = r^3/(r^2+a^2)^(3/2)), truncated at trunc*a."""
    xmax = trunc ** 3 / (trunc ** 2 + 1.0) ** 1.5
    x = r.random(n) * xmax
    x = np.clip(x, 1e-12, None)
    return a / np.sqrt(x ** (-2.0 / 3.0) - 1.0)


def halo_mixture(n=1_000_000, n_halos=64, bg_frac=0.2, a_range=(0.005, 0.05), seed=BASE_SEED + 1,
                 neighbours=32, chunk=1 << 20, device=None):
    """Plummer halos + uniform background in the unit cube.

    Halo centres U[0.1,0.9]^3, scale a log-uniform in ``a_range``, halo weights
    log-normal (sigma 1); radii from the Plummer inverse CDF truncated at 10 a.
    h_i = (neighbours / (4/3 pi n(x_i)))^(1/3) with n the analytic number
    density of the mixture; value_i = mass * n(x_i) (mass density); mass 1/N.
    """
    pos32, cen, a, counts, n_bg = _halo_positions(n, n_halos, bg_frac, a_range, seed)
    # analytic number density of the mixture at each particle
    xmax = 10.0 ** 3 / (10.0 ** 2 + 1.0) ** 1.5
    if device is not None:
        nd = _halo_density_torch(pos32, cen, a, counts, xmax, float(n_bg), device)
    else:
        nd = _halo_density_np(pos32, cen, a, counts, xmax, float(n_bg), chunk)
    h = (neighbours / (4.0 / 3.0 * math.pi * nd)) ** (1.0 / 3.0)
    mass = np.full(n, 1.0 / n, np.float32)
    dens = (nd / n).astype(np.float32)
    return dict(pos=pos32, h=h.astype(np.float32), mass=mass, density=dens, value=dens.copy())


def halo_mixture_knn(n=1_000_000, n_halos=64, bg_frac=0.2, a_range=(0.005, 0.05), seed=BASE_SEED + 1,
                     neighbours=32, chunk=1 << 20, workers=-1):
    """The positions of ``halo_mixture`` (same arguments, same seed), with h and the value computed from
    the particles themselves, as an SPH code prepares its output:

    * h_i = the distance from particle i to its 32nd nearest neighbour (scipy k-d tree, FP64);
    * rho_i = sum over i and those neighbours j of m_j W(|x_i - x_j|; h_i), W the normalised cubic
      spline with support radius h_i (the common "N_ngb neighbours inside the kernel" convention of SPH
      density estimates); value_i = density_i = rho_i, mass 1/N.

    This is input preparation (the SPH simulation's job), not part of the rendering method: the renderer
    and the oracle receive the resulting arrays.  Cost: a k-d tree over N points and one query of
    neighbours + 1 per point (about 20 s for 16.8M points on 8 cores).
    """
    from scipy.spatial import cKDTree

    pos32, _, _, _, _ = _halo_positions(n, n_halos, bg_frac, a_range, seed)
    p64 = pos32.astype(np.float64)
    tree = cKDTree(p64, leafsize=16, balanced_tree=False, compact_nodes=False)
    h = np.empty(n, np.float64)
    rho = np.empty(n, np.float64)
    m = 1.0 / n
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        d, _ = tree.query(p64[s:e], k=neighbours + 1, workers=workers)  # column 0: the particle itself
        H = d[:, neighbours]
        u = d / H[:, None]
        wq = np.where(u < 0.5, 1.0 - 6.0 * u ** 2 + 6.0 * u ** 3, np.where(u < 1.0, 2.0 * (1.0 - u) ** 3, 0.0))
        h[s:e] = H
        rho[s:e] = m * 8.0 / (math.pi * H ** 3) * wq.sum(axis=1)
    dens = rho.astype(np.float32)
    return dict(pos=pos32, h=h.astype(np.float32), mass=np.full(n, m, np.float32), density=dens, value=dens.copy())


def _halo_positions(n, n_halos, bg_frac, a_range, seed):
    """Positions of the halo mixture (FP32) and its parameters (centres, scales, counts, background)."""
    r = _rng(seed)
    n_bg = int(round(bg_frac * n))
    n_h = n - n_bg
    cen = 0.1 + 0.8 * r.random((n_halos, 3))
    la, lb = math.log(a_range[0]), math.log(a_range[1])
    a = np.exp(la + (lb - la) * r.random(n_halos))
    w = np.exp(r.normal(0.0, 1.0, n_halos))
    counts = r.multinomial(n_h, w / w.sum())
    pos = np.empty((n, 3), np.float64)
    o = 0
    for k in range(n_halos):
        c = counts[k]
        if c == 0:
            continue
        rad = _plummer_radius(r, a[k], c)
        d = r.normal(size=(c, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        pos[o:o + c] = cen[k] + rad[:, None] * d
        o += c
    pos[o:] = r.random((n - o, 3))
    return pos.astype(np.float32), cen, a, counts, n_bg


def _halo_density_np(pos32, cen, a, counts, xmax, n_bg, chunk):
    n = pos32.shape[0]
    nd = np.full(n, n_bg, np.float64)  # background: n_bg per unit volume
    p64 = pos32.astype(np.float64)
    n_halos = len(a)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        acc = nd[s:e]
        for k in range(n_halos):
            if counts[k] == 0:
                continue
            r2 = ((p64[s:e] - cen[k]) ** 2).sum(axis=1)
            inside = r2 < (10.0 * a[k]) ** 2
            rho = 3.0 / (4.0 * math.pi * a[k] ** 3) * (1.0 + r2 / a[k] ** 2) ** -2.5
            acc += np.where(inside, counts[k] / xmax * rho, 0.0)
        nd[s:e] = acc
    return nd


def _halo_density_torch(pos32, cen, a, counts, xmax, n_bg, device, chunk=1 << 22):
    """Same analytic density as _halo_density_np, evaluated in float64 with torch."""
    import torch

    n = pos32.shape[0]
    out = np.empty(n, np.float64)
    cen_t = torch.tensor(cen, dtype=torch.float64, device=device)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        p = torch.from_numpy(pos32[s:e]).to(device=device, dtype=torch.float64)
        acc = torch.full((e - s,), n_bg, dtype=torch.float64, device=device)
        for k in range(len(a)):
            if counts[k] == 0:
                continue
            r2 = ((p - cen_t[k]) ** 2).sum(dim=1)
            rho = 3.0 / (4.0 * math.pi * a[k] ** 3) * (1.0 + r2 / a[k] ** 2) ** -2.5
            acc += torch.where(r2 < (10.0 * a[k]) ** 2, counts[k] / xmax * rho, torch.zeros_like(rho))
        out[s:e] = acc.cpu().numpy()
    return out


def dam_break_slab(n=64_000_000, seed=BASE_SEED + 4, neighbours=32, chunk=1 << 22):
    """Dam-break-like slab in a [0,1]x[0,0.5]x[0,1] tank.

    95% of the particles in a lower layer z in [0, 0.25] whose density grows
    linearly toward the floor (pdf of z proportional to 2 - z/0.25), 5% in a
    sparse splash z in [0.25, 1] with density falling off as exp(-(z-0.25)/0.15).
    h from the analytic number density (``neighbours`` neighbours), clamped to
    [1e-4, 1e-2]; value = a hydrostatic-pressure-like 1 - z (in [0,1]); mass
    1/N; density = analytic mass density.
    """
    r = _rng(seed)
    n_low = int(round(0.95 * n))
    n_up = n - n_low
    pos = np.empty((n, 3), np.float32)
    vol_xy = 0.5
    # lower layer: pdf(z) ~ (2 - z/0.25) on [0, 0.25]
    u = r.random(n_low)
    # inverse CDF of f(z) = (2 - 4z) / (0.25*1.5) normalised on [0,0.25]
    # F(z) = (2 z - 2 z^2) / 0.375 -> solve 2z^2 - 2z + 0.375 u = 0
    zl = (2.0 - np.sqrt(4.0 - 8.0 * 0.375 * u)) / 4.0
    pos[:n_low, 0] = r.random(n_low)
    pos[:n_low, 1] = 0.5 * r.random(n_low)
    pos[:n_low, 2] = zl
    lam = 0.15
    zmax = 0.75
    uu = r.random(n_up) * (1 - math.exp(-zmax / lam))
    zu = 0.25 - lam * np.log1p(-uu)
    pos[n_low:, 0] = r.random(n_up)
    pos[n_low:, 1] = 0.5 * r.random(n_up)
    pos[n_low:, 2] = zu
    z = pos[:, 2].astype(np.float64)
    nd = np.where(
        z <= 0.25,
        n_low * (2.0 - 4.0 * z) / 0.375 / vol_xy,
        n_up * np.exp(-(z - 0.25) / lam) / (lam * (1 - math.exp(-zmax / lam))) / vol_xy,
    )
    h = np.clip((neighbours / (4.0 / 3.0 * math.pi * nd)) ** (1.0 / 3.0), 1e-4, 1e-2)
    mass = np.full(n, 1.0 / n, np.float32)
    dens = (nd / n).astype(np.float32)
    val = (1.0 - z).astype(np.float32)
    return dict(pos=pos, h=h.astype(np.float32), mass=mass, density=dens, value=val)


# --------------------------------------------------------------------------
# cameras
# --------------------------------------------------------------------------

def ortho_camera_z(width=64, height=64, lo=(0.0, 0.0), hi=(1.0, 1.0), z0=-1.0):
    """Orthographic rays along +z through the pixel centres of [lo,hi] in x,y."""
    cx, cy = 0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1])
    return dict(projection="orthographic", eye=(cx, cy, z0), target=(cx, cy, z0 + 1.0), up=(0.0, -1.0, 0.0),
                half_w=0.5 * (hi[0] - lo[0]), half_h=0.5 * (hi[1] - lo[1]), t_near=0.0, width=width, height=height)


def orbit_camera(width, height, azimuth_deg=30.0, elevation_deg=20.0, distance=2.0, fovy_deg=40.0,
                 center=(0.5, 0.5, 0.5), t_near=0.0):
    """Perspective camera on a sphere around ``center`` looking at it."""
    az, el = math.radians(azimuth_deg), math.radians(elevation_deg)
    eye = (center[0] + distance * math.cos(el) * math.cos(az),
           center[1] + distance * math.cos(el) * math.sin(az),
           center[2] + distance * math.sin(el))
    return dict(projection="perspective", eye=eye, target=tuple(center), up=(0.0, 0.0, 1.0), fovy_deg=fovy_deg,
                t_near=t_near, width=width, height=height)


def random_orbit_cameras(count, seed, resolutions=(256, 512, 1024, 2048), center=(0.5, 0.5, 0.5)):
    r = _rng(seed)
    cams = []
    for _ in range(count):
        res = int(resolutions[r.integers(len(resolutions))])
        cams.append(orbit_camera(res, res, azimuth_deg=360.0 * r.random(), elevation_deg=-60 + 120 * r.random(),
                                 distance=2.0, fovy_deg=40.0, center=center))
    return cams


# --------------------------------------------------------------------------
# transfer functions
# --------------------------------------------------------------------------

def tf_bumps(n=256, lo=0.0, hi=2.0, centres=(0.5, 1.0, 1.5), width=0.05, base=0.05, scale=2.0, sigma_scale=1.0):
    """Piecewise-linear RGBA table: RGB a smooth ramp, A = scale*(base + sum of Gaussian bumps)."""
    v = np.linspace(lo, hi, n)
    s = (v - lo) / (hi - lo)
    rgba = np.zeros((n, 4))
    rgba[:, 0] = s
    rgba[:, 1] = 0.5 + 0.5 * np.sin(math.pi * s)
    rgba[:, 2] = 1.0 - s
    bumps = sum(np.exp(-0.5 * ((v - c) / width) ** 2) for c in centres)
    rgba[:, 3] = scale * (base + bumps)
    return dict(rgba=rgba.astype(np.float32), lo=float(lo), hi=float(hi), sigma_scale=float(sigma_scale))


def tf_density(values, n=256, quantile=0.999, sigma_scale=1.0, opacity=1.0):
    """Transfer function over [0, quantile(values)] with a log-like opacity ramp and three bands."""
    hi = float(np.quantile(np.asarray(values, np.float64), quantile))
    v = np.linspace(0.0, hi, n)
    s = v / hi
    rgba = np.zeros((n, 4))
    rgba[:, 0] = np.sqrt(s)
    rgba[:, 1] = s ** 2
    rgba[:, 2] = 0.3 + 0.7 * (1 - s)
    bands = sum(np.exp(-0.5 * ((s - c) / 0.03) ** 2) for c in (0.1, 0.35, 0.7))
    rgba[:, 3] = opacity * (0.05 + 1.5 * s + 3.0 * bands)
    return dict(rgba=rgba.astype(np.float32), lo=0.0, hi=hi, sigma_scale=float(sigma_scale))


def pixel_sample(width, height, count, seed):
    r = _rng(seed)
    count = min(count, width * height)
    return np.sort(r.choice(width * height, size=count, replace=False)).astype(np.int32)
