"""Pins of the oracle's confinement energy, Eq. (TPConf), Sec. 2.2 (Confinement),
against facts that do not come from its code:

- the union identity: for two disjoint surfaces A and B (no shared vertex),
  Phi(A u B) = Phi(A) + Phi(B) + Phi_conf(A; B) + Phi_conf(B; A), with Phi the
  self-energy oracle (pinned in test_oracle_pins.py);
- complex-step derivatives of an independently written sum, per triangle
  (w, nu, x free) and per vertex;
- the continuum limit for concentric spheres, where the inner integral does
  not depend on the outer point and reduces to a one-dimensional integral
  (computed here with scipy's adaptive quadrature): second-order convergence
  of the flat one-point rule and its Richardson extrapolate.
"""

import numpy as np
import pytest

from paper_2509_22110_gb300 import meshgen


def rotation(seed):
    Q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((3, 3)))
    return Q if np.linalg.det(Q) > 0 else -Q


def brute_conf_soa(x, nu, w, y, a, q=6, p=12):
    """Separately written double sum over (T on S, K on S_conf); analytic in x, nu, w."""
    d = x[:, None, :] - y[None, :, :]
    n = np.einsum("ti,tki->tk", nu, d)
    r2 = np.einsum("tki,tki->tk", d, d)
    return np.sum(w[:, None] * a[None, :] * n**q / r2 ** (p // 2))


def brute_conf_vertices(V, F, y, a):
    """The same sum as a function of the vertices of S (complex-safe: no abs)."""
    A, B, C = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    x = (A + B + C) / 3.0
    N = np.cross(B - A, C - A)
    length = np.sqrt(np.sum(N * N, axis=1))
    return brute_conf_soa(x, N / length[:, None], length / 2, y, a)


def test_union_identity(oracle_mod):
    VA, FA = meshgen.perturbed_sphere(2, 0.01, 3)
    VB, FB = meshgen.icosphere(2)
    VB = 1.1 * VB @ rotation(1).T
    V = np.vstack([VA, VB])
    F = np.vstack([FA, FB + VA.shape[0]])
    c = 0.7
    lhs = oracle_mod.energy(V, F, c=c)
    rhs = (oracle_mod.energy(VA, FA, c=c) + oracle_mod.energy(VB, FB, c=c) +
           oracle_mod.conf_energy(VA, FA, VB, FB, c=c) + oracle_mod.conf_energy(VB, FB, VA, FA, c=c))
    assert abs(lhs - rhs) <= 1e-12 * lhs, (lhs, rhs)


def test_per_triangle_complex_step(oracle_mod):
    V, F = meshgen.perturbed_sphere(1, 0.02, 5)
    Vc, Fc = meshgen.icosphere(1)
    Vc = 1.2 * Vc @ rotation(2).T
    x, nu, w = oracle_mod.tri_data(V, F)
    y, a = oracle_mod.conf_data(Vc, Fc)
    gw, gnu, gx = oracle_mod.conf_accum(V, F, Vc, Fc)
    h = 1e-30
    for T in (0, 13, 41, 77):
        wc = w.astype(np.complex128)
        wc[T] += 1j * h
        assert abs(brute_conf_soa(x, nu, wc, y, a).imag / h - gw[T]) <= 1e-12 * abs(gw[T])
        for k in range(3):
            nc = nu.astype(np.complex128)
            nc[T, k] += 1j * h
            assert abs(brute_conf_soa(x, nc, w, y, a).imag / h - gnu[T, k]) <= 1e-12 * np.linalg.norm(gnu[T])
            xc = x.astype(np.complex128)
            xc[T, k] += 1j * h
            assert abs(brute_conf_soa(xc, nu, w, y, a).imag / h - gx[T, k]) <= 1e-12 * np.linalg.norm(gx[T])


def test_vertex_gradient_complex_step(oracle_mod):
    V, F = meshgen.perturbed_sphere(1, 0.02, 6)
    Vc, Fc = meshgen.perturbed_sphere(1, 0.02, 7, radius=1.3)
    y, a = oracle_mod.conf_data(Vc, Fc)
    c = 0.3
    E, g = oracle_mod.conf_gradient(V, F, Vc, Fc, c=c)
    assert abs(E - c * brute_conf_vertices(V, F, y, a)) <= 1e-12 * E
    h = 1e-30
    for i in (0, 5, 23, 41):
        for k in range(3):
            Vz = V.astype(np.complex128)
            Vz[i, k] += 1j * h
            ref = c * brute_conf_vertices(Vz, F, y, a).imag / h
            assert abs(ref - g[i, k]) <= 1e-11 * np.linalg.norm(g[i]), (i, k, ref, g[i, k])


@pytest.mark.parametrize("R1,R2", [(1.0, 2.0), (0.5, 0.75)])
def test_concentric_spheres_continuum(oracle_mod, R1, R2):
    """Evolving sphere R1 (outward normals) inside a confining sphere R2:
    Phi_conf -> 4 pi R1^2 * 2 pi R2^2 * int_{-1}^{1} (R1 - R2 u)^6 / (R1^2 + R2^2 - 2 R1 R2 u)^6 du."""
    from scipy.integrate import quad

    f = lambda u: (R1 - R2 * u) ** 6 / (R1 * R1 + R2 * R2 - 2 * R1 * R2 * u) ** 6
    exact = 4 * np.pi * R1**2 * 2 * np.pi * R2**2 * quad(f, -1, 1, epsabs=0, epsrel=1e-13, limit=200)[0]
    E = []
    for L in (3, 4):
        V, F = meshgen.icosphere(L)
        E.append(oracle_mod.conf_energy(R1 * V, F, R2 * V, F))
    ratio = (E[0] - exact) / (E[1] - exact)
    assert 3.8 < ratio < 4.3, ratio  # second order in the mesh size
    richardson = (4 * E[1] - E[0]) / 3
    assert abs(richardson - exact) <= 1e-4 * exact, (richardson, exact)
