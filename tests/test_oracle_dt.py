"""Pins of the oracle's cluster-cluster (dual-tree) Barnes-Hut form.

The scheme clusters both integrals: every unordered pair of triangles is
assigned to exactly one unordered pair of tree nodes, evaluated by the cluster
monopole of both orderings when the pair is admissible (vertex boxes apart,
max(diag_A, diag_B) < theta |X_A - X_B|) and exactly otherwise.  Pinned by:
the partition (near pairs plus represented far pairs equal the admitted pairs
counted by brute force), theta = 0 reproducing the direct sum, Euler's
relation for the homogeneous approximate energy, translation invariance, the
error falling with theta, and complex-step derivatives of an energy written
here in numpy (traversal decisions from real data, moments recomputed from
complex positions), which pins the chain rule through the cluster moments.
"""

import numpy as np
import pytest

from paper_2509_22110_gb300 import meshgen


def setup(oracle_mod, level, leaf, seed=2):
    V, F = meshgen.sh_deformed_sphere(level, 12, 0.05, seed)
    x, nu, w = oracle_mod.tri_data(V, F)
    t = oracle_mod.lbvh(x, 30, leaf)
    mom, box = oracle_mod.moments(V, F, t, soa=(x, nu, w))
    return V, F, (x, nu, w), t, mom, box


@pytest.mark.parametrize("theta", [0.0, 0.5, 1.0, 2.0])
def test_partition_of_the_pairs(oracle_mod, theta):
    V, F, soa, t, mom, box = setup(oracle_mod, 3, 8)
    E, gw, gnu, gx, info = oracle_mod.dt_accum(V, F, t, mom, box, theta, soa=soa)
    assert info["near_pairs"] + info["far_represented"] == oracle_mod.admitted_pairs(F)
    if theta == 0.0:
        assert info["far_pairs"] == 0
    else:
        assert info["far_pairs"] > 0


def test_theta_zero_is_direct(oracle_mod):
    V, F = meshgen.sh_deformed_sphere(3, 12, 0.05, 2)
    E, g = oracle_mod.gradient(V, F)
    Ed, gd, info = oracle_mod.dt_gradient(V, F, 0.0)
    assert info["far_pairs"] == 0
    assert abs(Ed - E) <= 1e-12 * E
    np.testing.assert_allclose(gd, g, rtol=1e-10, atol=1e-12 * np.abs(g).max())


@pytest.mark.parametrize("theta", [0.5, 1.5])
def test_euler_and_translation(oracle_mod, theta):
    V, F = meshgen.sh_deformed_sphere(4, 12, 0.05, 3)
    E, g, info = oracle_mod.dt_gradient(V, F, theta)
    assert info["far_pairs"] > 0
    assert abs(info["phi_from_weights"] - E) <= 1e-12 * E  # homogeneous of degree 2 in the weights
    assert abs(np.sum(V * g) + 2.0 * E) <= 1e-10 * E       # degree 4 + q - p = -2 in the positions
    assert np.abs(g.sum(0)).max() <= 1e-10 * np.abs(g).sum()
    E2, _, _ = oracle_mod.dt_gradient(V + np.array([0.25, -0.5, 1.0]), F, theta)
    assert abs(E2 - E) <= 1e-11 * E


def test_error_falls_with_theta(oracle_mod):
    V, F = meshgen.sh_deformed_sphere(4, 12, 0.05, 2)
    E, g = oracle_mod.gradient(V, F)
    errs = []
    for th in (2.0, 1.0, 0.5, 0.25):
        Ed, gd, info = oracle_mod.dt_gradient(V, F, th)
        errs.append((abs(Ed - E) / E, np.linalg.norm(gd - g) / np.linalg.norm(g)))
    assert all(errs[i][0] > errs[i + 1][0] for i in range(3)), errs
    assert all(errs[i][1] > errs[i + 1][1] for i in range(3)), errs


def _dt_lists(t, mom, box, theta, leaf):
    """The node-pair partition by a traversal written here (same rule as documented)."""
    n = t["n"]
    first, last, left, right = t["first"], t["last"], t["left"], t["right"]

    def small(N):
        return last[N] - first[N] + 1 <= leaf or N >= n - 1

    def adm(A, B):
        bA, bB = box[A], box[B]
        if not any(bA[3 + a] < bB[a] or bB[3 + a] < bA[a] for a in range(3)):
            return False
        dA = np.sqrt(np.sum((bA[3:] - bA[:3]) ** 2))
        dB = np.sqrt(np.sum((bB[3:] - bB[:3]) ** 2))
        XA, XB = mom[A, 1:4] / mom[A, 0], mom[B, 1:4] / mom[B, 0]
        return max(dA, dB) < theta * np.sqrt(np.sum((XA - XB) ** 2))

    far, near, stack = [], [], [(0, 0)]
    while stack:
        A, B = stack.pop()
        if A == B:
            if small(A):
                near.append((A, A))
            else:
                stack += [(left[A], left[A]), (right[A], right[A]), (left[A], right[A])]
        elif adm(A, B):
            far.append((A, B))
        elif small(A) and small(B):
            near.append((A, B))
        elif not small(A) and (last[A] - first[A] >= last[B] - first[B] or small(B)):
            stack += [(left[A], B), (right[A], B)]
        else:
            stack += [(A, left[B]), (A, right[B])]
    return far, near


def _dt_energy_complex(V, F, t, far, near, q=6, p=12):
    """The cluster-cluster energy from (possibly complex) positions, analytic for even q."""
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    x = (a + b + c) / 3.0
    N = np.cross(b - a, c - a)
    ln = np.sqrt(np.sum(N * N, axis=1))
    w = ln / 2
    nu = N / ln[:, None]
    perm, first, last = t["perm"], t["first"], t["last"]
    sets = [set(int(v) for v in f) for f in F]

    def members(Nd):
        return perm[first[Nd]: last[Nd] + 1]

    def mono(Nd):
        m = members(Nd)
        A = np.sum(w[m])
        return A, np.sum(w[m, None] * x[m], axis=0) / A, np.sum(w[m, None] * nu[m], axis=0) / A

    E = 0
    for A_, B_ in far:
        AA, XA, nA = mono(A_)
        AB, XB, nB = mono(B_)
        d = XA - XB
        r2 = np.sum(d * d)
        E = E + AA * AB * ((nA @ d) ** q + (nB @ (-d)) ** q) / r2 ** (p // 2)
    for A_, B_ in near:
        mA, mB = members(A_), members(B_)
        for i, T in enumerate(mA):
            for S in mB if A_ != B_ else mA[i + 1:]:
                if T == S or sets[T] & sets[S]:
                    continue
                d = x[T] - x[S]
                r2 = np.sum(d * d)
                E = E + w[T] * w[S] * ((nu[T] @ d) ** q + (nu[S] @ (-d)) ** q) / r2 ** (p // 2)
    return E


def test_complex_step_gradient(oracle_mod):
    leaf, theta = 4, 1.2
    V, F, soa, t, mom, box = setup(oracle_mod, 2, leaf, seed=7)
    E, gw, gnu, gx, info = oracle_mod.dt_accum(V, F, t, mom, box, theta, soa=soa)
    far, near = _dt_lists(t, mom, box, theta, leaf)
    assert len(far) == info["far_pairs"] and len(far) > 20
    E_np = _dt_energy_complex(V, F, t, far, near)
    assert abs(E_np - E) <= 1e-12 * E
    g = oracle_mod.adjoint(V, F, gw, gnu, gx, 1.0)
    rng = np.random.default_rng(3)
    for v in rng.choice(V.shape[0], 12, replace=False):
        for k in range(3):
            Vc = V.astype(np.complex128)
            Vc[v, k] += 1e-30j
            cs = _dt_energy_complex(Vc, F, t, far, near).imag / 1e-30
            assert abs(g[v, k] - cs) <= 1e-9 * np.abs(g).max(), (v, k, g[v, k], cs)
