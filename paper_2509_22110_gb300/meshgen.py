"""Seeded synthetic closed triangle meshes (inputs only).

This module builds vertex arrays ``V`` (float64, [nv, 3]) and face arrays ``F``
(int32, [nt, 3], counter-clockwise seen from outside) for the workloads the
library is measured on.  It holds none of the tangent-point arithmetic: no
centroid, normal, area or energy is computed here, only positions and
connectivity.  Both the CUDA path and the CPU oracle consume these arrays.

The shapes stand in for the paper's sphere-topology meshes (a dumbbell in
Fig. 3, the discocyte-to-stomatocyte transition of Sec. 4.2 and the confined
sphere inversion of Sec. 4.3); none of the paper's meshes is available, so
every mesh here is a subdivided icosahedron mapped to a seeded shape:

* ``icosphere(level)`` - 10*4^L+2 vertices, 20*4^L faces on the unit sphere.
* ``perturbed_sphere`` - radial noise r = 1 + eps, eps ~ N(0, sigma^2).
* ``stomatocyte_dish`` - a double-walled spherical cap (outer radius 1, inner
  radius 1-gap, polar half-angle 60 degrees, half-torus rim) with seeded
  jitter along the profile normal; the two sheets face each other across
  the gap, the near-contact situation of the paper's stomatocyte shapes.
* ``sh_deformed_sphere`` - r = 1 + sum_{l=1..lmax} sum_m a_lm Y_lm with
  a_lm ~ N(0, (amp/l)^2) and real orthonormal spherical harmonics.
* ``folded_sphere`` - radial Gaussian grooves along random great-circle arcs
  (a wrinkled, epithelium-like surface).
* ``smooth_displacement`` - a seeded smooth vector field (random Fourier
  modes) used to move a mesh over successive evaluations.
"""

from __future__ import annotations

import hashlib

import numpy as np

__all__ = [
    "icosahedron",
    "octahedron",
    "icosphere",
    "perturbed_sphere",
    "stomatocyte_dish",
    "sh_deformed_sphere",
    "folded_sphere",
    "smooth_displacement",
    "nested_spheres",
    "mesh_hash",
    "workload",
]


def octahedron():
    """Unit octahedron with vertices +-e_i and outward counter-clockwise faces."""
    V = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], dtype=np.float64)
    F = []
    for sx, ix in ((1, 0), (-1, 1)):
        for sy, iy in ((1, 2), (-1, 3)):
            for sz, iz in ((1, 4), (-1, 5)):
                tri = [ix, iy, iz]
                # orientation: (v1-v0)x(v2-v0) must point along (sx, sy, sz)
                if sx * sy * sz < 0:
                    tri = [ix, iz, iy]
                F.append(tri)
    return V, np.asarray(F, dtype=np.int32)


def icosahedron():
    """Regular icosahedron inscribed in the unit sphere, outward faces."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    V = np.array(
        [
            [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
            [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
            [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
        ],
        dtype=np.float64,
    )
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    F = np.array(
        [
            [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
            [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
            [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
            [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
        ],
        dtype=np.int32,
    )
    return V, F


def _subdivide(V, F):
    """One 1-to-4 split; edge midpoints are projected to the unit sphere."""
    nv = V.shape[0]
    a, b, c = F[:, 0].astype(np.int64), F[:, 1].astype(np.int64), F[:, 2].astype(np.int64)
    e = np.stack([np.stack([a, b], 1), np.stack([b, c], 1), np.stack([c, a], 1)], 1)  # [m,3,2]
    lo = e.min(axis=2)
    hi = e.max(axis=2)
    key = lo * nv + hi
    ukey, inv = np.unique(key.ravel(), return_inverse=True)
    inv = inv.reshape(-1, 3)
    ua = ukey // nv
    ub = ukey % nv
    mid = V[ua] + V[ub]
    mid /= np.linalg.norm(mid, axis=1, keepdims=True)
    Vn = np.concatenate([V, mid], 0)
    m_ab = nv + inv[:, 0]
    m_bc = nv + inv[:, 1]
    m_ca = nv + inv[:, 2]
    Fn = np.concatenate(
        [
            np.stack([a, m_ab, m_ca], 1),
            np.stack([b, m_bc, m_ab], 1),
            np.stack([c, m_ca, m_bc], 1),
            np.stack([m_ab, m_bc, m_ca], 1),
        ],
        0,
    )
    return Vn, Fn.astype(np.int32)


def icosphere(level: int):
    """Subdivided icosahedron on the unit sphere (V = 10*4^L + 2, F = 20*4^L)."""
    V, F = icosahedron()
    for _ in range(int(level)):
        V, F = _subdivide(V, F)
    return V, F


def perturbed_sphere(level: int, sigma: float = 0.01, seed: int = 0, radius: float = 1.0):
    """Icosphere with radii r_v = radius * (1 + eps_v), eps_v ~ N(0, sigma^2)."""
    V, F = icosphere(level)
    rng = np.random.default_rng(seed)
    r = 1.0 + sigma * rng.standard_normal(V.shape[0])
    return V * (radius * r)[:, None], F


def _dish_profile(s, gap, cap_deg):
    """Point (rho, z) and outward unit normal of the dish profile at arc length s."""
    psi_c = np.deg2rad(cap_deg)
    r_out, r_in = 1.0, 1.0 - gap
    tube = 0.5 * gap
    r_mid = 0.5 * (r_out + r_in)
    l_out = r_out * psi_c
    l_rim = np.pi * tube
    rho = np.empty_like(s)
    z = np.empty_like(s)
    nr = np.empty_like(s)
    nz = np.empty_like(s)
    m0 = s <= l_out
    psi = s[m0] / r_out
    rho[m0], z[m0] = r_out * np.sin(psi), -r_out * np.cos(psi)
    nr[m0], nz[m0] = np.sin(psi), -np.cos(psi)
    m1 = (s > l_out) & (s <= l_out + l_rim)
    beta = (s[m1] - l_out) / tube
    ur = np.array([np.sin(psi_c), -np.cos(psi_c)])
    ut = np.array([np.cos(psi_c), np.sin(psi_c)])
    cx, cz = r_mid * ur
    dr = np.cos(beta) * ur[0] + np.sin(beta) * ut[0]
    dz = np.cos(beta) * ur[1] + np.sin(beta) * ut[1]
    rho[m1], z[m1] = cx + tube * dr, cz + tube * dz
    nr[m1], nz[m1] = dr, dz
    m2 = s > l_out + l_rim
    psi = psi_c - (s[m2] - l_out - l_rim) / r_in
    psi = np.maximum(psi, 0.0)
    rho[m2], z[m2] = r_in * np.sin(psi), -r_in * np.cos(psi)
    # the inner sheet faces the outer one: its outward normal points to the centre
    nr[m2], nz[m2] = -np.sin(psi), np.cos(psi)
    return rho, z, nr, nz, l_out + l_rim + r_in * psi_c


def stomatocyte_dish(level: int = 5, gap: float = 0.02, cap_deg: float = 60.0, jitter: float = 0.002, seed: int = 1):
    """Double-walled spherical dish: two sheets a distance ``gap`` apart.

    The icosphere's polar angle from the south pole is mapped linearly to arc
    length along a closed meridian profile (outer cap of radius 1 over polar
    half-angle ``cap_deg``, a half-torus rim of tube radius gap/2, the inner
    cap of radius 1-gap back to the axis); the azimuth is kept.  Each vertex
    is then moved along the profile normal by N(0, jitter^2).
    """
    V, F = icosphere(level)
    rng = np.random.default_rng(seed)
    theta0 = np.arccos(np.clip(-V[:, 2], -1.0, 1.0))
    phi = np.arctan2(V[:, 1], V[:, 0])
    _, _, _, _, total = _dish_profile(np.zeros(1), gap, cap_deg)
    s = theta0 / np.pi * total
    rho, z, nr, nz, _ = _dish_profile(s, gap, cap_deg)
    eps = jitter * rng.standard_normal(V.shape[0])
    rho = rho + eps * nr
    z = z + eps * nz
    rho = np.maximum(rho, 0.0)
    W = np.stack([rho * np.cos(phi), rho * np.sin(phi), z], 1)
    # put the two poles exactly on the axis
    W[np.abs(V[:, 2]) == 1.0, :2] = 0.0
    return W, F


def _real_sph_harm(lmax: int, theta, phi):
    """Real orthonormal spherical harmonics Y_lm, l=0..lmax, as dict (l,m)->array.

    Associated Legendre functions by the standard stable three-term
    recurrence (normalised form), no Condon-Shortley phase ambiguity matters
    because the coefficients are random.
    """
    x = np.cos(theta)
    sx = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    out = {}
    # normalised P_l^m with sqrt((2l+1)/(4pi) (l-m)!/(l+m)!)
    pmm = np.full_like(x, np.sqrt(1.0 / (4.0 * np.pi)))
    for m in range(lmax + 1):
        if m > 0:
            pmm = pmm * (-np.sqrt((2.0 * m + 1.0) / (2.0 * m)) * sx)
        plm2 = pmm
        vals = {m: pmm}
        if m + 1 <= lmax:
            plm1 = np.sqrt(2.0 * m + 3.0) * x * pmm
            vals[m + 1] = plm1
            for l in range(m + 2, lmax + 1):
                a = np.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
                b = np.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
                pl = a * (x * plm1 - b * plm2)
                vals[l] = pl
                plm2, plm1 = plm1, pl
        for l, p in vals.items():
            if m == 0:
                out[(l, 0)] = p
            else:
                out[(l, m)] = np.sqrt(2.0) * p * np.cos(m * phi)
                out[(l, -m)] = np.sqrt(2.0) * p * np.sin(m * phi)
    return out


def sh_deformed_sphere(level: int = 7, lmax: int = 12, amp: float = 0.05, seed: int = 2):
    """Icosphere with r(x) = 1 + sum_{l=1..lmax} sum_m a_lm Y_lm(x), a_lm ~ N(0, (amp/l)^2)."""
    V, F = icosphere(level)
    rng = np.random.default_rng(seed)
    theta = np.arccos(np.clip(V[:, 2], -1.0, 1.0))
    phi = np.arctan2(V[:, 1], V[:, 0])
    Y = _real_sph_harm(lmax, theta, phi)
    r = np.ones(V.shape[0])
    for l in range(1, lmax + 1):
        for m in range(-l, l + 1):
            r += rng.normal(0.0, amp / l) * Y[(l, m)]
    return V * r[:, None], F


def folded_sphere(level: int = 8, n_folds: int = 40, depth: float = 0.1, arc_len: float = 0.6,
                  width: float = 0.04, seed: int = 3):
    """Sphere with ``n_folds`` Gaussian radial grooves along random great-circle arcs.

    r(x) = 1 - depth * max_k exp(-dist_k(x)^2 / (2 width^2)), dist_k the angular
    distance from x to arc k (length ``arc_len`` radians, random centre and
    direction).  Using the max keeps overlapping grooves at depth ``depth``.
    """
    V, F = icosphere(level)
    rng = np.random.default_rng(seed)
    g = np.zeros(V.shape[0])
    for _ in range(n_folds):
        c = rng.standard_normal(3)
        c /= np.linalg.norm(c)
        t = rng.standard_normal(3)
        t -= c * (t @ c)
        t /= np.linalg.norm(t)
        nrm = np.cross(c, t)  # pole of the great circle through c along t
        # angular coordinate along the circle and distance off it
        s_along = np.arctan2(V @ t, V @ c)
        off = np.arcsin(np.clip(V @ nrm, -1.0, 1.0))
        beyond = np.maximum(np.abs(s_along) - 0.5 * arc_len, 0.0)
        dist2 = off * off + beyond * beyond
        g = np.maximum(g, np.exp(-dist2 / (2.0 * width * width)))
    return V * (1.0 - depth * g)[:, None], F


def smooth_displacement(X, n_modes: int = 8, kmax: int = 3, seed: int = 4):
    """Seeded smooth field u(X) = sum of ``n_modes`` random Fourier modes, max |u| = 1."""
    rng = np.random.default_rng(seed)
    u = np.zeros_like(X)
    for _ in range(n_modes):
        k = rng.integers(-kmax, kmax + 1, size=3)
        if not k.any():
            k[0] = 1
        a = rng.standard_normal(3)
        ph = rng.uniform(0.0, 2.0 * np.pi)
        u += np.sin(X @ k.astype(np.float64) + ph)[:, None] * a[None, :]
    u /= np.max(np.linalg.norm(u, axis=1))
    return u


def nested_spheres(level: int, gap: float):
    """Two disjoint concentric icospheres of radii 1 and 1-gap; the inner one faces inwards."""
    V, F = icosphere(level)
    nv = V.shape[0]
    V2 = np.concatenate([V, (1.0 - gap) * V], 0)
    F2 = np.concatenate([F, F[:, ::-1] + nv], 0).astype(np.int32)
    return V2, F2


def sphere_in_sphere(level: int = 7, radius: float = 1.1, sigma: float = 0.005, seed: int = 13):
    """Evolving sphere of radius 1 (radial jitter N(0, sigma^2)) and the concentric
    confining icosphere of the given radius, both at the same subdivision level:
    the setting of the sphere inversion in a spherical confinement (radius 1.1)."""
    V, F = perturbed_sphere(level, sigma, seed)
    Vc, Fc = icosphere(level)
    return V, F, radius * Vc, Fc


def mesh_hash(V, F) -> str:
    """SHA-256 over the little-endian bytes of V (float64) and F (int32)."""
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(V, dtype="<f8").tobytes())
    h.update(np.ascontiguousarray(F, dtype="<i4").tobytes())
    return h.hexdigest()


def workload(name: str):
    """The named synthetic workloads, returned as (V, F).

    ``sphere_l3``   - level 3 (1,280 faces), radial N(0, 0.01^2) noise, seed 0.
    ``dish_l5``     - level 5 (20,480 faces) stomatocyte-like dish, gap 0.02, seed 1.
    ``sh_l7``       - level 7 (327,680 faces) SH-deformed sphere, l<=12, seed 2.
    ``folds_l8``    - level 8 (1,310,720 faces), 40 folds of depth 0.1, seed 3.
    """
    if name == "sphere_l3":
        return perturbed_sphere(3, 0.01, 0)
    if name == "dish_l5":
        return stomatocyte_dish(5, 0.02, 60.0, 0.002, 1)
    if name == "sh_l7":
        return sh_deformed_sphere(7, 12, 0.05, 2)
    if name == "folds_l8":
        return folded_sphere(8, 40, 0.1, 0.6, 0.04, 3)
    if name.startswith("sh_l") and "_s" in name:
        lev, seed = name[4:].split("_s")
        return sh_deformed_sphere(int(lev), 12, 0.05, int(seed))
    raise KeyError(name)
