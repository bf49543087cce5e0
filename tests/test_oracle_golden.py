"""The oracle against the values stored in tests/golden/oracle_values.json (written by
tests/golden/make_golden.py from the oracle itself): a change of the oracle's arithmetic
shows up here and must come with a regenerated file and the reason for the change.  The
octahedron entry is also checked against its closed form Phi = 81/32, dPhi/dv = -(81/96) v."""

import json
import os

import numpy as np

from paper_2509_22110_gb300 import meshgen

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_values.json")


def test_golden_values(oracle_mod):
    gold = json.load(open(GOLDEN))
    V, F = meshgen.workload("sphere_l3")
    for k in (1, 3, 6):
        ent = gold[f"sphere_l3_quad{k}"]
        E, g = oracle_mod.quad_gradient(V, F, k)
        assert abs(E - ent["energy"]) <= 1e-13 * ent["energy"]
        np.testing.assert_allclose(g[ent["verts"]], np.array(ent["grad"]), rtol=1e-12, atol=1e-15)
    Vc, Fc = meshgen.octahedron()
    ent = gold["octahedron"]
    assert abs(ent["energy"] - 81 / 32) <= 1e-14
    np.testing.assert_allclose(np.array(ent["grad"]), -(81 / 96) * Vc, atol=1e-13)
    V, F, Vc, Fc = meshgen.sphere_in_sphere(3, 1.1, 0.005, 13)
    ent = gold["conf_sphere_l3"]
    E, g = oracle_mod.conf_gradient(V, F, Vc, Fc)
    assert abs(E - ent["energy"]) <= 1e-13 * ent["energy"]
    np.testing.assert_allclose(g[ent["verts"]], np.array(ent["grad"]), rtol=1e-12, atol=1e-15)
