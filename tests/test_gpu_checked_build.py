"""The checked build (libtp_debug.so, -DTP_DEBUG=1: every index that a
list-driven kernel reads from a work list is bounds-checked on the device and a
failure is reported as a status) runs the direct, Barnes-Hut, learned and
cluster-cluster evaluations without a failed check and with the release
library's results (needs a GPU)."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu

# one evaluation of each form on a level-4 mesh; prints energies and gradient norms as JSON
SCRIPT = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import paper_2509_22110_gb300 as tp
from paper_2509_22110_gb300 import meshgen
out = {"lib": tp._tp.LIB_PATH}
V, F = meshgen.sh_deformed_sphere(4, 12, 0.05, 3)
ctx = tp.tp_create(0, torch.cuda.current_stream().cuda_stream)
tp.tp_far_model_load(ctx, sys.argv[1] + "/paper_2509_22110_gb300/far_model_l7.bin")
tp.tp_mesh_upload(ctx, V, F)
g = np.zeros_like(V)
out["direct"] = [tp.tp_gradient(ctx, g, tp.tp_params_default()), g.tolist()]
out["direct_energy"] = tp.tp_energy(ctx, tp.tp_params_default())
for leaf in (16, 32):
    tp.tp_tree_build(ctx, leaf, 30)
    for name, mode, th in (("bh", tp.TP_BH, 0.25), ("learned", tp.TP_LEARNED, 0.25), ("dual", tp.TP_BH_DUAL, 0.5)):
        g = np.zeros_like(V)
        out[f"{name}{leaf}"] = [tp.tp_gradient(ctx, g, tp.tp_params_default(mode=mode, theta=th)), g.tolist()]
tp.tp_destroy(ctx)
print(json.dumps(out))
"""


def run(lib):
    env = dict(os.environ)
    if lib:
        env["TP_LIB"] = lib
    else:
        env.pop("TP_LIB", None)
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_matches_release():
    pytest.importorskip("torch")
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_22110_gb300 import build

    rel_lib = build.build()
    dbg_lib = build.build(debug=True)
    a = run(None)
    b = run(dbg_lib)
    assert a["lib"] == rel_lib and b["lib"] == dbg_lib
    for key in a:
        if key == "lib":
            continue
        if key == "direct_energy":
            assert abs(a[key] - b[key]) <= 1e-12 * abs(a[key]), key
            continue
        ea, ga = a[key]
        eb, gb = b[key]
        ga, gb = np.asarray(ga), np.asarray(gb)
        # the same arithmetic; the order of FP64 atomic adds may differ between runs. The
        # cluster-cluster lists are appended with atomics, so their order, and with it the
        # order of the FP32 partial sums over a leaf's partners, differs between runs too
        tol = 1e-6 if key.startswith("dual") else 1e-12
        assert abs(ea - eb) <= tol * abs(ea), (key, ea, eb)
        assert np.linalg.norm(ga - gb) <= tol * np.linalg.norm(ga), key
