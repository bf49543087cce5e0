"""Write tests/golden/oracle_values.json: energies and sampled vertex gradients of the FP64
oracle on small seeded meshes (one-point, 3- and 6-point quadrature, confinement).  The
values come from oracle/ only; rerun this script (and say why in the commit) whenever the
oracle's arithmetic is deliberately changed.

    python tests/golden/make_golden.py
"""

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2509_22110_gb300 import meshgen  # noqa: E402

VERTS = [0, 1, 2, 7, 40, 101]


def main():
    out = {"_about": "FP64 oracle values (c = 1, q = 6, p = 12, vertex-sharing exclusion) written by make_golden.py"}
    V, F = meshgen.workload("sphere_l3")
    for k in (1, 3, 6):
        E, g = oracle.quad_gradient(V, F, k)
        out[f"sphere_l3_quad{k}"] = {"energy": E, "verts": VERTS, "grad": g[VERTS].tolist()}
    Vo, Fo = meshgen.octahedron()
    E, g = oracle.gradient(Vo, Fo)
    out["octahedron"] = {"energy": E, "verts": list(range(6)), "grad": g.tolist()}
    V, F, Vc, Fc = meshgen.sphere_in_sphere(3, 1.1, 0.005, 13)
    E, g = oracle.conf_gradient(V, F, Vc, Fc)
    out["conf_sphere_l3"] = {"energy": E, "verts": VERTS, "grad": g[VERTS].tolist()}
    with open(os.path.join(HERE, "oracle_values.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
