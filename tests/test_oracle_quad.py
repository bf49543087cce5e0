"""Pins of the oracle's multi-point quadrature form (Sec. 3.1, 3.2: a rule per
element for both integrals) against facts that do not come from its code:
exactness of the rules on polynomials (a! b! / (a + b + 2)! over the unit
triangle), the centroid rule reproducing the one-point oracle, complex-step
derivatives of an independently written sum, the scaling law and Euler's
relation for the homogeneous energy, invariance under rigid motions, and
convergence to the sphere's continuum value pi^2 / (4 R^2)."""

import math

import numpy as np
import pytest

from paper_2509_22110_gb300 import meshgen


@pytest.mark.parametrize("k,degree", [(1, 1), (3, 2), (6, 4)])
def test_rule_exactness(oracle_mod, k, degree):
    bary, om = oracle_mod.quad_rule(k)
    assert abs(om.sum() - 1.0) <= 1e-15 and np.allclose(bary.sum(axis=1), 1.0, atol=1e-15)
    x, y = bary[:, 1], bary[:, 2]  # reference triangle (0,0), (1,0), (0,1)
    for a in range(degree + 1):
        for b in range(degree + 1 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(0.5 * np.sum(om * x**a * y**b) - exact) <= 1e-15, (a, b)
    if k > 1:  # not exact one degree higher (the rule's stated degree is sharp)
        errs = [abs(0.5 * np.sum(om * x**a * y**(degree + 1 - a)) -
                    math.factorial(a) * math.factorial(degree + 1 - a) / math.factorial(degree + 3))
                for a in range(degree + 2)]
        assert max(errs) > 1e-6


def test_centroid_rule_is_the_one_point_sum(oracle_mod):
    V, F = meshgen.perturbed_sphere(2, 0.01, 3)
    E1, g1 = oracle_mod.gradient(V, F)
    Eq, gq = oracle_mod.quad_gradient(V, F, 1)
    assert abs(Eq - E1) <= 1e-14 * E1
    assert np.linalg.norm(gq - g1) <= 1e-13 * np.linalg.norm(g1)


def brute_quad_energy(V, F, bary, om, q=6, p=12):
    """Separately written k-point sum (complex-safe: no abs)."""
    A, B, C = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    N = np.cross(B - A, C - A)
    length = np.sqrt(np.sum(N * N, axis=1))
    nu = N / length[:, None]
    area = length / 2
    pts = np.stack([l[0] * A + l[1] * B + l[2] * C for l in bary], axis=1)  # [nt, k, 3]
    sets = [set(int(v) for v in f) for f in F]
    total = 0
    nt = F.shape[0]
    for T in range(nt):
        keep = [S for S in range(nt) if S != T and not (sets[T] & sets[S])]
        for qa in range(len(om)):
            d = pts[T, qa][None, None, :] - pts[keep]  # [m, k, 3]
            n = d @ nu[T]
            r2 = np.sum(d * d, axis=2)
            total = total + om[qa] * area[T] * np.sum(om[None, :] * area[keep][:, None] * n**q / r2 ** (p // 2))
    return total


@pytest.mark.parametrize("k", [3, 6])
def test_quad_gradient_complex_step(oracle_mod, k):
    V, F = meshgen.perturbed_sphere(1, 0.02, 4)
    bary, om = oracle_mod.quad_rule(k)
    E, g = oracle_mod.quad_gradient(V, F, k)
    assert abs(E - brute_quad_energy(V, F, bary, om)) <= 1e-12 * E
    h = 1e-30
    for i in (0, 9, 27):
        for c in range(3):
            Vz = V.astype(np.complex128)
            Vz[i, c] += 1j * h
            ref = brute_quad_energy(Vz, F, bary, om).imag / h
            assert abs(ref - g[i, c]) <= 1e-11 * np.linalg.norm(g[i]), (i, c, ref, g[i, c])


@pytest.mark.parametrize("k", [3, 6])
def test_quad_scaling_euler_and_invariance(oracle_mod, k):
    V, F = meshgen.perturbed_sphere(2, 0.01, 5)
    E, g = oracle_mod.quad_gradient(V, F, k)
    for lam in (0.5, 2.0):
        assert abs(oracle_mod.quad_energy(lam * V, F, k) - lam**-2 * E) <= 1e-12 * E
    # Euler: sum_v v . dPhi/dv = (4 + q - p) Phi = -2 Phi; translation and rotation
    assert abs(np.sum(V * g) + 2 * E) <= 1e-11 * E
    scale = np.abs(g).sum()
    assert np.linalg.norm(g.sum(axis=0)) <= 1e-12 * scale
    assert np.linalg.norm(np.cross(V, g).sum(axis=0)) <= 1e-12 * scale


@pytest.mark.parametrize("k", [3, 6])
def test_quad_sphere_continuum(oracle_mod, k):
    exact = math.pi**2 / 4  # unit sphere: the kernel is (2R)^-6 for every pair
    errs = []
    for L in (2, 3, 4):
        V, F = meshgen.icosphere(L)
        errs.append(abs(oracle_mod.quad_energy(V, F, k) - exact) / exact)
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.03, errs
