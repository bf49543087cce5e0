"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test ties the oracle to something fixed independently of its code:
closed forms (octahedron, sphere), an independent brute-force evaluation
(complex-step derivatives of a separately written energy), the refinement
limit pi^2/(4 R^2) of the sphere, the scaling law Phi(lambda X) =
lambda^(4+q-p) Phi(X), translation/rotation invariance, Euler's relation for
homogeneous functions, central finite differences and the embedding property
(Eq. TP is finite iff the surface does not self-intersect, Sec. 2.2.2).
"""

import math

import numpy as np
import pytest

from paper_2509_22110_gb300 import meshgen

Q, P = 6.0, 12.0


# --------------------------------------------------------------- independent brute force
def brute_energy(V, F, q=6, p=12, exclude="vertex"):
    """Separately written Eq. (TP) sum; works for complex V (analytic in V for even q)."""
    V = np.asarray(V)
    F = np.asarray(F)
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    cen = (a + b + c) / 3.0
    nrm = np.stack(
        [
            (b[:, 1] - a[:, 1]) * (c[:, 2] - a[:, 2]) - (b[:, 2] - a[:, 2]) * (c[:, 1] - a[:, 1]),
            (b[:, 2] - a[:, 2]) * (c[:, 0] - a[:, 0]) - (b[:, 0] - a[:, 0]) * (c[:, 2] - a[:, 2]),
            (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0]),
        ],
        1,
    )
    length = np.sqrt(np.sum(nrm * nrm, axis=1))  # analytic sqrt (no abs)
    area = length / 2
    unit = nrm / length[:, None]
    nt = F.shape[0]
    sets = [set(int(v) for v in f) for f in F]
    total = 0
    for T in range(nt):
        keep = []
        for S in range(nt):
            k = len(sets[T] & sets[S])
            if S == T or (k >= 1 if exclude == "vertex" else k >= 2):
                continue
            keep.append(S)
        keep = np.array(keep, dtype=np.int64)
        d = cen[T][None, :] - cen[keep]
        n = d @ unit[T]
        r2 = np.sum(d * d, axis=1)
        total = total + area[T] * np.sum(area[keep] * n**q / r2 ** (p // 2))
    return total


def complex_step_grad(V, F, h=1e-30):
    g = np.zeros_like(V)
    for i in range(V.shape[0]):
        for k in range(3):
            Vc = V.astype(np.complex128)
            Vc[i, k] += 1j * h
            g[i, k] = brute_energy(Vc, F).imag / h
    return g


# --------------------------------------------------------------- closed forms
def test_octahedron_closed_form(oracle_mod):
    """Each face of the unit octahedron admits only the opposite face:
    w = sqrt(3)/2, |d| = <nu,d> = 2/sqrt(3), Phi = 8 * (3/4) / (2/sqrt3)^6 = 81/32;
    Euler (degree 4+q-p = -2) and the octahedral symmetry give dPhi/dv = -(81/96) v."""
    V, F = meshgen.octahedron()
    E, g = oracle_mod.gradient(V, F, Q, P, 1.0)
    assert abs(E - 81.0 / 32.0) < 1e-14
    np.testing.assert_allclose(g, -(81.0 / 96.0) * V, atol=1e-14)


def test_octahedron_scale_factor(oracle_mod):
    V, F = meshgen.octahedron()
    c = 1e-4 / 6.0  # the paper's rho/alpha
    E, g = oracle_mod.gradient(V, F, Q, P, c)
    assert abs(E - c * 81.0 / 32.0) < 1e-18
    np.testing.assert_allclose(g, -c * (81.0 / 96.0) * V, atol=1e-18)


def test_sphere_points_radial_normals_exact(oracle_mod):
    """On a sphere <nu(x), x-y> = |x-y|^2 / (2R) (the tangent-point geometry of
    Sec. 2.2.2), so with centroids on the sphere and radial normals every pair
    term is (2R)^-6 w_T w_S: Phi = (2R)^-6 * sum over admitted ordered pairs of w_T w_S."""
    rng = np.random.default_rng(5)
    V, F = meshgen.icosphere(2)
    R = 1.7
    x = rng.standard_normal((F.shape[0], 3))
    x = R * x / np.linalg.norm(x, axis=1, keepdims=True)
    nu = x / R
    w = rng.uniform(0.5, 2.0, F.shape[0])
    E = oracle_mod.energy_soa(x, nu, w, F, Q, P, 1.0)
    sets = [set(f) for f in F.tolist()]
    tot = w.sum() ** 2
    for T in range(F.shape[0]):
        for S in range(F.shape[0]):
            if T == S or sets[T] & sets[S]:
                tot -= w[T] * w[S]
    expect = tot / (2 * R) ** 6
    assert abs(E - expect) < 1e-13 * expect


def test_sphere_refinement_limit(oracle_mod):
    """The continuum value on the unit sphere is (4 pi)^2 / 2^6 = pi^2/4; the
    one-point flat discretisation converges to it at about second order."""
    vals = []
    for L in (2, 3, 4, 5):
        V, F = meshgen.icosphere(L)
        vals.append(oracle_mod.energy(V, F, Q, P, 1.0))
    exact = math.pi**2 / 4.0
    err = [v - exact for v in vals]
    assert all(e > 0 for e in err)
    ratios = [err[i] / err[i + 1] for i in range(3)]
    assert all(3.0 < r < 4.5 for r in ratios), ratios
    rich = vals[-1] + (vals[-1] - vals[-2]) / (ratios[-1] - 1.0)
    assert abs(rich - exact) / exact < 2e-4, (rich, exact)


# --------------------------------------------------------------- independent brute force
@pytest.mark.parametrize("mesh", ["icosahedron", "ico1_noisy", "ico2_noisy"])
def test_bruteforce_energy(oracle_mod, mesh):
    if mesh == "icosahedron":
        V, F = meshgen.icosahedron()
    elif mesh == "ico1_noisy":
        V, F = meshgen.perturbed_sphere(1, 0.05, 7)
    else:
        V, F = meshgen.perturbed_sphere(2, 0.02, 8)
    E = oracle_mod.energy(V, F, Q, P, 1.0)
    B = brute_energy(V, F)
    assert abs(E - B) < 1e-13 * abs(B)
    Ee = oracle_mod.energy(V, F, Q, P, 1.0, adj=1)
    Be = brute_energy(V, F, exclude="edge")
    assert abs(Ee - Be) < 1e-13 * abs(Be)
    assert Ee > E


def test_icosahedron_pair_count(oracle_mod):
    """Each icosahedron face shares a vertex with 9 others: 10 partners, 200 ordered pairs.
    With unit weights and radial normals the SoA energy counts them."""
    V, F = meshgen.icosahedron()
    x = V[F].mean(axis=1)
    R = np.linalg.norm(x, axis=1)
    x = x / R[:, None]
    E = oracle_mod.energy_soa(x, x, np.ones(20), F, Q, P, 1.0)
    assert abs(E - 200.0 / 2.0**6) < 1e-13


def test_complex_step_gradient(oracle_mod):
    """The oracle's hand-written chain rule against complex-step derivatives of
    the independent brute-force energy (exact to rounding, no step error)."""
    V, F = meshgen.perturbed_sphere(1, 0.05, 9)
    _, g = oracle_mod.gradient(V, F, Q, P, 1.0)
    gc = complex_step_grad(V, F)
    np.testing.assert_allclose(g, gc, rtol=1e-11, atol=1e-12 * np.abs(gc).max())


# --------------------------------------------------------------- laws and invariants
@pytest.mark.parametrize("lam", [0.5, 2.0, 3.7])
def test_scaling_law(oracle_mod, lam):
    """Phi(lambda X) = lambda^(4+q-p) Phi(X) and grad(lambda X) = lambda^(3+q-p) grad(X)."""
    V, F = meshgen.workload("sphere_l3")
    E0, g0 = oracle_mod.gradient(V, F, Q, P, 1.0)
    E1, g1 = oracle_mod.gradient(lam * V, F, Q, P, 1.0)
    assert abs(E1 - lam ** (4 + Q - P) * E0) < 1e-12 * abs(E1)
    np.testing.assert_allclose(g1, lam ** (3 + Q - P) * g0, rtol=1e-10, atol=1e-12 * np.abs(g1).max())


@pytest.mark.parametrize("name", ["sphere_l3", "dish_l3"])
def test_invariants(oracle_mod, name):
    """Translation: sum dPhi/dv = 0; rotation: sum v x dPhi/dv = 0;
    homogeneity of degree 4+q-p: sum v . dPhi/dv = (4+q-p) Phi."""
    if name == "dish_l3":
        V, F = meshgen.stomatocyte_dish(3, 0.1, 60.0, 0.005, 1)
    else:
        V, F = meshgen.workload(name)
    E, g = oracle_mod.gradient(V, F, Q, P, 1.0)
    scale = np.abs(g).sum()
    assert np.abs(g.sum(0)).max() < 1e-12 * scale
    assert np.abs(np.cross(V, g).sum(0)).max() < 1e-12 * scale
    assert abs(np.sum(V * g) - (4 + Q - P) * E) < 1e-11 * abs(E)


def test_translation_rotation_energy(oracle_mod):
    V, F = meshgen.workload("sphere_l3")
    E = oracle_mod.energy(V, F)
    rng = np.random.default_rng(3)
    Qm, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    E2 = oracle_mod.energy(V @ Qm.T + np.array([0.3, -2.0, 5.0]), F)
    assert abs(E2 - E) < 1e-11 * E


def test_energy_touching_is_local_difference(oracle_mod):
    V, F = meshgen.workload("sphere_l3")
    v = 17
    tris = oracle_mod.incident_triangles(F, [v])
    V2 = V.copy()
    V2[v] += [1e-3, -2e-3, 5e-4]
    full = oracle_mod.energy(V2, F) - oracle_mod.energy(V, F)
    loc = oracle_mod.energy_touching(V2, F, tris) - oracle_mod.energy_touching(V, F, tris)
    assert abs(full - loc) < 1e-12 * abs(full) + 1e-14


@pytest.mark.parametrize("name,seed", [("sphere_l3", 10), ("dish_l5", 11)])
def test_central_fd(oracle_mod, name, seed):
    """Central differences (h = 1e-6) of the energy on 32 seeded vertex coordinates."""
    V, F = meshgen.workload(name)
    rng = np.random.default_rng(seed)
    verts = rng.choice(V.shape[0], 32, replace=False)
    axes = rng.integers(0, 3, 32)
    g = oracle_mod.vertex_gradient_sample(V, F, verts)
    h = 1e-6
    gmax = np.abs(g).max()
    for i, (v, k) in enumerate(zip(verts, axes)):
        tris = oracle_mod.incident_triangles(F, [v])
        Vp = V.copy()
        Vm = V.copy()
        Vp[v, k] += h
        Vm[v, k] -= h
        fd = (oracle_mod.energy_touching(Vp, F, tris) - oracle_mod.energy_touching(Vm, F, tris)) / (2 * h)
        assert abs(fd - g[i, k]) <= 1e-6 * max(abs(g[i, k]), 1e-3 * gmax), (v, k, fd, g[i, k])


def test_sampled_vertex_gradient_matches_full(oracle_mod):
    V, F = meshgen.workload("sphere_l3")
    _, g = oracle_mod.gradient(V, F)
    verts = np.array([0, 5, 100, 641])
    gs = oracle_mod.vertex_gradient_sample(V, F, verts)
    np.testing.assert_allclose(gs, g[verts], rtol=1e-12, atol=1e-14)


def test_embedding_growth(oracle_mod):
    """Two nested spheres: Phi stays finite for a positive gap and grows as the gap closes."""
    vals = []
    for gap in (0.5, 0.3, 0.2, 0.1, 0.05):
        V, F = meshgen.nested_spheres(2, gap)
        E = oracle_mod.energy(V, F)
        assert np.isfinite(E)
        vals.append(E)
    assert all(vals[i] < vals[i + 1] for i in range(len(vals) - 1)), vals


def test_coincident_centroids_infinite(oracle_mod):
    """A self-intersecting configuration (two admitted triangles with the same
    centroid) has no finite energy (Sec. 2.2.2: finite iff embedded)."""
    V, F = meshgen.icosahedron()
    x, nu, w = oracle_mod.tri_data(V, F)
    # move face 0's data onto a non-adjacent face's centroid, tilted normal
    sets = [set(f) for f in F.tolist()]
    S = next(s for s in range(20) if not (sets[0] & sets[s]))
    x[0] = x[S]
    nu[0] = np.array([1.0, 0.0, 0.0])
    with np.errstate(all="ignore"):
        E = oracle_mod.energy_soa(x, nu, w, F)
    assert not np.isfinite(E) or E > 1e300


# --------------------------------------------------------------- per-triangle fields
def brute_energy_soa(x, nu, w, F, q=6, p=12):
    """Separately written Eq. (TP) sum from per-triangle (x, nu, w) taken as free
    variables (vertex-sharing exclusion from F); analytic in x, nu, w."""
    sets = [set(int(v) for v in f) for f in np.asarray(F)]
    nt = len(sets)
    total = 0
    for T in range(nt):
        keep = np.array([S for S in range(nt) if S != T and not (sets[T] & sets[S])], dtype=np.int64)
        d = x[T][None, :] - x[keep]
        n = d @ nu[T]
        r2 = np.sum(d * d, axis=1)
        total = total + w[T] * np.sum(w[keep] * n**q / r2 ** (p // 2))
    return total


def test_triangle_fields_complex_step(oracle_mod):
    """dPhi/dw_T, dPhi/dnu_T and dPhi/dx_T of the oracle (the one-point counterparts
    of f_K, f_nu, f of Eq. (dTP_reordered)) against complex-step derivatives of an
    independently written sum, with w, nu and x as independent variables."""
    V, F = meshgen.sh_deformed_sphere(1, 12, 0.05, 7)
    x, nu, w = oracle_mod.tri_data(V, F)
    gw, gnu, gx = oracle_mod.tri_accum(V, F, soa=(x, nu, w))
    h = 1e-30
    for T in (0, 17, 43, 79):
        wc = w.astype(np.complex128)
        wc[T] += 1j * h
        assert abs(brute_energy_soa(x, nu, wc, F).imag / h - gw[T]) <= 1e-12 * abs(gw[T])
        for a in range(3):
            nc = nu.astype(np.complex128)
            nc[T, a] += 1j * h
            ref = brute_energy_soa(x, nc, w, F).imag / h
            assert abs(ref - gnu[T, a]) <= 1e-12 * np.linalg.norm(gnu[T]), (T, a, ref, gnu[T, a])
            xc = x.astype(np.complex128)
            xc[T, a] += 1j * h
            ref = brute_energy_soa(xc, nu, w, F).imag / h
            assert abs(ref - gx[T, a]) <= 1e-12 * np.linalg.norm(gx[T]), (T, a, ref, gx[T, a])
