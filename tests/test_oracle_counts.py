"""Pins of the oracle's admitted-pair count and of its energy on unperturbed icospheres.

The count of ordered pairs the sum of Eq. (TP) runs over is the numerator of
the benchmark's pair-interaction rate, so it is pinned to closed forms: on a
closed triangle mesh two distinct triangles share an edge or exactly one
vertex, an edge is shared by exactly two triangles, and a vertex of degree d
is shared by C(d, 2) pairs, so the unordered pairs sharing at least one
vertex number sum_v C(d_v, 2) - E (edge-sharing pairs are met at both
endpoints).  Open sub-meshes are checked against a count written here from
vertex stars.
"""

import json
import os
from itertools import combinations

import numpy as np
import pytest

from paper_2509_22110_gb300 import meshgen

HERE = os.path.dirname(os.path.abspath(__file__))


def closed_mesh_admitted(F, adj):
    nt = F.shape[0]
    edges = {tuple(sorted((int(f[i]), int(f[(i + 1) % 3])))) for f in F for i in range(3)}
    E = len(edges)
    assert 2 * E == 3 * nt  # closed: every edge in exactly two triangles
    if adj == 1:
        return nt * (nt - 1) - 2 * E
    deg = np.bincount(F.ravel())
    return nt * (nt - 1) - 2 * (int(np.sum(deg * (deg - 1) // 2)) - E)


def star_count(F, adj):
    """Ordered admitted pairs from the unordered vertex-sharing pairs found in vertex stars."""
    nt = F.shape[0]
    star = {}
    for t, f in enumerate(F):
        for v in f:
            star.setdefault(int(v), []).append(t)
    shared = {}
    for ts in star.values():
        for a, b in combinations(sorted(set(ts)), 2):
            shared[(a, b)] = shared.get((a, b), 0) + 1
    excl = sum(1 for k in shared.values() if (k >= 2 if adj == 1 else k >= 1))
    return nt * (nt - 1) - 2 * excl


@pytest.mark.parametrize("level", [0, 1, 2, 3])
@pytest.mark.parametrize("adj", [0, 1])
def test_admitted_pairs_closed_icosphere(oracle_mod, level, adj):
    V, F = meshgen.icosphere(level)
    assert oracle_mod.admitted_pairs(F, adj=adj) == closed_mesh_admitted(F, adj)


def test_admitted_pairs_small_polyhedra(oracle_mod):
    # octahedron: every face keeps only the opposite face; tetrahedron: all faces share an edge
    _, Fo = meshgen.octahedron()
    assert oracle_mod.admitted_pairs(Fo) == 8
    assert oracle_mod.admitted_pairs(Fo, adj=1) == 8 * 7 - 2 * 12
    Ft = np.array([[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]], dtype=np.int32)
    assert oracle_mod.admitted_pairs(Ft) == 0 and oracle_mod.admitted_pairs(Ft, adj=1) == 0


@pytest.mark.parametrize("nt_keep", [1, 2, 37, 1023, 1025])
def test_admitted_pairs_open_submeshes(oracle_mod, nt_keep):
    _, F = meshgen.perturbed_sphere(4, 0.01, 3)
    F = np.ascontiguousarray(F[:nt_keep])
    for adj in (0, 1):
        assert oracle_mod.admitted_pairs(F, adj=adj) == star_count(F, adj)


def test_dish_admitted_pairs(oracle_mod):
    _, F = meshgen.workload("dish_l5")
    for adj in (0, 1):
        assert oracle_mod.admitted_pairs(F, adj=adj) == closed_mesh_admitted(F, adj)


@pytest.mark.parametrize("level", [1, 2, 3, 4])
def test_unperturbed_icosphere_energy(oracle_mod, level):
    """Independent 10-digit values of Phi on the unperturbed unit icosphere."""
    with open(os.path.join(HERE, "golden", "icosphere_unperturbed.json")) as f:
        ref = json.load(f)["energy"][str(level)]
    V, F = meshgen.icosphere(level)
    E = oracle_mod.energy(V, F)
    assert abs(E - ref) <= 1e-9 * ref, (E, ref)
