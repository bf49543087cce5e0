"""Pins of the oracle's cluster tree, moments and Barnes-Hut form.

The tree is checked against the defining properties of a binary radix tree
over the sorted distinct keys (which fix it uniquely), the moments against
brute-force sums over each node's members, and the Barnes-Hut form against
the direct sum: theta = 0 admits no cluster and must reproduce it; the error
must fall as theta falls (Sec. 3.2: the separation parameter controls how
eagerly clusters are used).
"""

import numpy as np
import pytest

from paper_2509_22110_gb300 import meshgen


def decode(code, bits):
    qx = qy = qz = 0
    for i in range(bits):
        qz |= ((code >> (3 * i)) & 1) << i
        qy |= ((code >> (3 * i + 1)) & 1) << i
        qx |= ((code >> (3 * i + 2)) & 1) << i
    return qx, qy, qz


@pytest.fixture(scope="module")
def sh_mesh():
    return meshgen.sh_deformed_sphere(4, 12, 0.05, 2)


def test_morton_quantisation_properties(oracle_mod, sh_mesh):
    V, F = sh_mesh
    x, _, _ = oracle_mod.tri_data(V, F)
    t = oracle_mod.lbvh(x, 30, 16)
    q = np.array([decode(int(c), 10) for c in t["codes"]])
    assert q.min() >= 0 and q.max() <= 1023
    for a in range(3):
        # quantisation is monotone in the coordinate and spans the full range
        order = np.argsort(x[:, a], kind="stable")
        assert np.all(np.diff(q[order, a]) >= 0)
        assert q[np.argmin(x[:, a]), a] == 0
        assert q[np.argmax(x[:, a]), a] == 1023
        # cells have width (hi-lo)/1024
        lo, hi = x[:, a].min(), x[:, a].max()
        cell = (hi - lo) / 1024
        assert np.all(x[:, a] >= lo + q[:, a] * cell - 1e-12)
        assert np.all(x[:, a] <= lo + (q[:, a] + 1) * cell + 1e-12)


def test_sorted_permutation(oracle_mod, sh_mesh):
    V, F = sh_mesh
    x, _, _ = oracle_mod.tri_data(V, F)
    t = oracle_mod.lbvh(x, 30, 16)
    perm = t["perm"]
    assert np.array_equal(np.sort(perm), np.arange(F.shape[0]))
    keys = (t["codes"][perm].astype(np.uint64) << np.uint64(32)) | perm.astype(np.uint64)
    assert np.all(np.diff(keys.astype(np.float64)) >= 0) and np.all(keys[1:] > keys[:-1])


def test_radix_tree_properties(oracle_mod, sh_mesh):
    V, F = sh_mesh
    x, _, _ = oracle_mod.tri_data(V, F)
    t = oracle_mod.lbvh(x, 30, 16)
    n = t["n"]
    perm = t["perm"]
    keys = [(int(t["codes"][perm[k]]) << 32) | int(perm[k]) for k in range(n)]
    first, last, parent = t["first"], t["last"], t["parent"]
    assert first[0] == 0 and last[0] == n - 1 and parent[0] == -1
    seen = np.zeros(2 * n - 1, dtype=int)
    for i in range(n - 1):
        lc, rc = int(t["left"][i]), int(t["right"][i])
        seen[lc] += 1
        seen[rc] += 1
        assert parent[lc] == i and parent[rc] == i
        lo, hi = first[i], last[i]
        g = last[lc]
        assert first[lc] == lo and first[rc] == g + 1 and last[rc] == hi
        # node ids follow the split: left child is node g (or primitive), right is g+1
        assert lc == (g if g != lo else n - 1 + g)
        assert rc == (g + 1 if g + 1 != hi else n - 1 + hi)
        hb = (keys[lo] ^ keys[hi]).bit_length() - 1
        for k in range(lo, hi + 1):
            assert keys[k] >> (hb + 1) == keys[lo] >> (hb + 1)
            assert ((keys[k] >> hb) & 1) == (0 if k <= g else 1)
    assert seen[0] == 0 and np.all(seen[1:] == 1)


def test_cluster_leaves_partition(oracle_mod, sh_mesh):
    V, F = sh_mesh
    x, _, _ = oracle_mod.tri_data(V, F)
    t = oracle_mod.lbvh(x, 30, 16)
    n = t["n"]
    pos = 0
    for L in t["leaves"]:
        cnt = t["last"][L] - t["first"][L] + 1
        assert t["first"][L] == pos and cnt <= 16
        par = t["parent"][L]
        assert par < 0 or t["last"][par] - t["first"][par] + 1 > 16
        pos = t["last"][L] + 1
    assert pos == n


def test_moments_bruteforce(oracle_mod, sh_mesh):
    V, F = sh_mesh
    x, nu, w = oracle_mod.tri_data(V, F)
    t = oracle_mod.lbvh(x, 30, 16)
    mom, box = oracle_mod.moments(V, F, t)
    rng = np.random.default_rng(0)
    nodes = np.concatenate([[0], rng.choice(2 * t["n"] - 1, 300, replace=False)])
    iu = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    for v in nodes:
        mem = t["perm"][t["first"][v]: t["last"][v] + 1]
        A = w[mem].sum()
        ref = [A, *(w[mem, None] * x[mem]).sum(0), *(w[mem, None] * nu[mem]).sum(0)]
        ref += [(w[mem] * nu[mem, a] * nu[mem, b]).sum() for a, b in iu]
        np.testing.assert_allclose(mom[v], ref, rtol=1e-12, atol=1e-14)
        vv = V[F[mem].ravel()]
        np.testing.assert_array_equal(box[v], np.concatenate([vv.min(0), vv.max(0)]))


def test_bh_theta_zero_is_direct(oracle_mod):
    V, F = meshgen.sh_deformed_sphere(3, 12, 0.05, 2)
    E, g = oracle_mod.gradient(V, F)
    Eb, gb, info = oracle_mod.bh_gradient(V, F, 0.0)
    assert info["far_terms"] == 0
    assert abs(Eb - E) < 1e-12 * E
    np.testing.assert_allclose(gb, g, rtol=1e-10, atol=1e-12 * np.abs(g).max())


def test_bh_error_falls_with_theta(oracle_mod):
    V, F = meshgen.sh_deformed_sphere(4, 12, 0.05, 2)
    E, g = oracle_mod.gradient(V, F)
    errs = []
    for th in (1.0, 0.5, 0.25, 0.125):
        Eb, gb, info = oracle_mod.bh_gradient(V, F, th)
        assert info["far_terms"] > 0
        errs.append((abs(Eb - E) / E, np.linalg.norm(gb - g) / np.linalg.norm(g)))
    e_energy = [e[0] for e in errs]
    e_grad = [e[1] for e in errs]
    assert all(e_grad[i] > e_grad[i + 1] for i in range(3)), errs
    assert all(e_energy[i] > e_energy[i + 1] for i in range(3)), errs
    # the accuracy the cluster form is held to: relative error <= 1e-3 at theta = 0.125
    assert e_energy[3] < 1e-3 and e_grad[3] < 1e-3, errs


def test_bh_no_excluded_pair_is_far(oracle_mod):
    """Admissible clusters have vertex boxes disjoint from the target leaf's, so
    they contain no triangle sharing a vertex with any target."""
    V, F = meshgen.sh_deformed_sphere(3, 12, 0.05, 2)
    x, nu, w = oracle_mod.tri_data(V, F)
    t = oracle_mod.lbvh(x, 30, 16)
    mom, box = oracle_mod.moments(V, F, t, soa=(x, nu, w))
    # a box that touches another shares at least a point; boxes of adjacent triangles touch
    for T in range(0, F.shape[0], 97):
        for S in range(F.shape[0]):
            if set(F[T]) & set(F[S]):
                bt = box[t["n"] - 1 + np.where(t["perm"] == T)[0][0]]
                bs = box[t["n"] - 1 + np.where(t["perm"] == S)[0][0]]
                overlap = all(bt[a] <= bs[3 + a] and bs[a] <= bt[3 + a] for a in range(3))
                assert overlap


def _bh_target_energy(xT, nuT, wT, T, near, far, x, nu, w, mom, q=6, p=12):
    """The Barnes-Hut energy seen by target T as a function of its own (x, nu, w): exact
    pairs (both orderings) with its near triangles plus, for every admissible cluster C,
    the monopole of both orderings with C's moments held fixed (only the inner integral
    is clustered, Sec. 3.2; area-weighted centroid and unnormalised area-averaged normal).
    Analytic in xT, nuT for even q, so complex steps give its exact derivatives."""
    f = 0
    if len(near):
        d = xT[None, :] - x[near]
        r2 = np.sum(d * d, axis=1)
        a = d @ nuT
        b = np.sum(nu[near] * d, axis=1)
        f = f + wT * np.sum(w[near] * (a**q + b**q) / r2 ** (p // 2))
    for C in far:
        A = mom[C, 0]
        X = mom[C, 1:4] / A
        nb = mom[C, 4:7] / A
        d = xT - X
        r2 = np.sum(d * d)
        f = f + wT * A * ((d @ nuT) ** q + (nb @ (-d)) ** q) / r2 ** (p // 2)
    return f


def test_bh_far_term_complex_step(oracle_mod):
    """Every target's Barnes-Hut derivatives dPhi/dw, dPhi/dnu, dPhi/dx (or_bh_accum) equal
    the complex-step derivatives of the target's energy written above, with the near/far
    split found by a traversal written here from the admissibility rule (vertex boxes
    strictly apart on some axis and diag_C < theta (|X_C - c_L| - diag_L / 2))."""
    V, F = meshgen.sh_deformed_sphere(3, 12, 0.05, 2)
    x, nu, w = oracle_mod.tri_data(V, F)
    leaf = 4
    t = oracle_mod.lbvh(x, 30, leaf)
    mom, box = oracle_mod.moments(V, F, t, soa=(x, nu, w))
    theta = 0.5
    gw, gnu, gx, nn, nf = oracle_mod.bh_accum(V, F, t, mom, box, theta, soa=(x, nu, w))
    n = t["n"]
    left, right, first, last, perm = t["left"], t["right"], t["first"], t["last"], t["perm"]
    sets = [set(int(v) for v in f) for f in F]
    rng = np.random.default_rng(5)
    far_total = near_total = 0
    leaves = list(t["leaves"])
    checked = 0
    for L in rng.choice(leaves, 24, replace=False):
        bl = box[L]
        cl = 0.5 * (bl[:3] + bl[3:])
        dl = np.linalg.norm(bl[3:] - bl[:3])
        near, far = [], []
        stack = [0]
        while stack:
            C = stack.pop()
            bc = box[C]
            apart = any(bl[3 + a] < bc[a] or bc[3 + a] < bl[a] for a in range(3))
            X = mom[C, 1:4] / mom[C, 0]
            if apart and np.linalg.norm(bc[3:] - bc[:3]) < theta * (np.linalg.norm(X - cl) - 0.5 * dl):
                far.append(C)
            elif last[C] - first[C] + 1 <= leaf:
                near.extend(int(perm[m]) for m in range(first[C], last[C] + 1))
            else:
                stack += [right[C], left[C]]
        for k in range(first[L], last[L] + 1):
            T = int(perm[k])
            nearT = np.array([S for S in near if S != T and not (sets[T] & sets[S])], dtype=np.int64)
            far_total += len(far)
            near_total += len(nearT)
            h = 1e-30
            f0 = _bh_target_energy(x[T], nu[T], w[T], T, nearT, far, x, nu, w, mom)
            assert abs(gw[T] - f0 / w[T]) <= 1e-12 * abs(gw[T])
            for a in range(3):
                e = np.zeros(3, dtype=complex)
                e[a] = 1j * h
                dx = _bh_target_energy(x[T] + e, nu[T], w[T], T, nearT, far, x, nu, w, mom).imag / h
                dn = _bh_target_energy(x[T], nu[T] + e, w[T], T, nearT, far, x, nu, w, mom).imag / h
                assert abs(gx[T, a] - dx) <= 1e-11 * np.abs(gx[T]).max(), (T, a, gx[T, a], dx)
                assert abs(gnu[T, a] - dn) <= 1e-11 * np.abs(gnu[T]).max(), (T, a, gnu[T, a], dn)
            checked += 1
    assert checked > 50 and far_total > 10 * checked and near_total > 0
