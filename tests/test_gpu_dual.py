"""Parity of the cluster-cluster (dual-tree) Barnes-Hut form with the oracle (needs a GPU).

Bars: the node-pair partition identical to the oracle's (far node pairs,
represented pairs and admitted near pairs counted exactly: the admissibility
decisions are FP64 with the same operations on both sides); energy within
1e-6 and gradient within 1e-5 (relative L2 and per vertex) of or_dt_accum at
the same theta, leaf size and exponents; theta = 0 reproduces the direct sum;
Euler's relation and translation invariance at full size.
"""

import numpy as np
import pytest

from paper_2509_22110_gb300 import meshgen

pytestmark = pytest.mark.gpu

E_TOL = 1e-6
G_TOL = 1e-5


@pytest.fixture(scope="module")
def tp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_22110_gb300 import build

    build.build()
    import paper_2509_22110_gb300 as tpm

    return tpm


@pytest.fixture()
def ctx(tp):
    import torch

    c = tp.tp_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    tp.tp_destroy(c)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def maxrel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def oracle_dt(oracle_mod, V, F, theta, leaf, q=6.0, p=12.0, adj=0):
    x, nu, w = oracle_mod.tri_data(V, F)
    t = oracle_mod.lbvh(x, 30, leaf)
    mom, box = oracle_mod.moments(V, F, t, soa=(x, nu, w))
    E, gw, gnu, gx, info = oracle_mod.dt_accum(V, F, t, mom, box, theta, q, p, adj, soa=(x, nu, w))
    return E, oracle_mod.adjoint(V, F, gw, gnu, gx, 1.0), (gw, gnu, gx), info


@pytest.mark.parametrize("theta,leaf,q,adj", [(0.5, 16, 6, 0), (1.0, 8, 6, 0), (2.0, 16, 8, 0), (1.0, 32, 6, 1),
                                              (0.7, 4, 6, 0), (1.5, 1, 6, 0)])
def test_dual_parity_with_oracle(tp, ctx, oracle_mod, theta, leaf, q, adj):
    V, F = meshgen.sh_deformed_sphere(4, 12, 0.05, 2)
    E, g, (ow, onu, ox), info = oracle_dt(oracle_mod, V, F, theta, leaf, q, 2.0 * q, adj)
    assert info["far_pairs"] > 0
    tp.tp_mesh_upload(ctx, V, F)
    tp.tp_tree_build(ctx, leaf, 30)
    grad = np.zeros_like(V)
    flags = tp._tp.TP_EXCLUDE_EDGE if adj else 0
    e = tp.tp_gradient(ctx, grad, tp.tp_params_default(mode=tp.TP_BH_DUAL, theta=theta, q=q, p=2 * q, flags=flags))
    st = tp.tp_get_stats(ctx)
    assert st["far_terms"] == info["far_pairs"]
    assert st["far_pairs"] == info["far_represented"]
    assert st["pairs_exact"] == info["near_pairs"]
    assert abs(e - E) <= E_TOL * E, (e, E)
    assert rel(grad, g) <= G_TOL and maxrel(grad, g) <= G_TOL, (rel(grad, g), maxrel(grad, g))
    gw, gnu, gx = tp.tp_debug_accum(ctx, F.shape[0])
    assert rel(gw, ow) <= E_TOL and rel(gnu, onu) <= G_TOL and rel(gx, ox) <= G_TOL
    assert abs(tp.tp_energy(ctx, tp.tp_params_default(mode=tp.TP_BH_DUAL, theta=theta, q=q, p=2 * q,
                                                       flags=flags)) - E) <= E_TOL * E


def test_dual_theta_zero_is_direct(tp, ctx, oracle_mod):
    V, F = meshgen.workload("sphere_l3")
    E, g = oracle_mod.gradient(V, F)
    tp.tp_mesh_upload(ctx, V, F)
    tp.tp_tree_build(ctx, 16, 30)
    grad = np.zeros_like(V)
    e = tp.tp_gradient(ctx, grad, tp.tp_params_default(mode=tp.TP_BH_DUAL, theta=0.0))
    assert tp.tp_get_stats(ctx)["far_terms"] == 0
    assert tp.tp_get_stats(ctx)["pairs_exact"] == oracle_mod.admitted_pairs(F)
    assert abs(e - E) <= E_TOL * E and rel(grad, g) <= G_TOL


@pytest.mark.parametrize("nt_keep", [1, 2, 37, 2000])
def test_dual_ragged_sizes(tp, ctx, oracle_mod, nt_keep):
    V, F = meshgen.perturbed_sphere(4, 0.01, 3)
    F = np.ascontiguousarray(F[:nt_keep])
    E, g, _, info = oracle_dt(oracle_mod, V, F, 1.0, 16)
    tp.tp_mesh_upload(ctx, V, F)
    tp.tp_tree_build(ctx, 16, 30)
    grad = np.zeros_like(V)
    e = tp.tp_gradient(ctx, grad, tp.tp_params_default(mode=tp.TP_BH_DUAL, theta=1.0))
    assert tp.tp_get_stats(ctx)["far_terms"] == info["far_pairs"]
    if E == 0.0:
        assert e == 0.0 and not grad.any()
        return
    assert abs(e - E) <= E_TOL * E and rel(grad, g) <= G_TOL


def test_dual_full_size_properties(tp, ctx):
    """327,680 triangles: Euler's relation (degree -2), translation invariance, the
    error against the direct sum falling with theta."""
    V, F = meshgen.workload("sh_l7")
    tp.tp_mesh_upload(ctx, V, F)
    gd = np.zeros_like(V)
    ed = tp.tp_gradient(ctx, gd, tp.tp_params_default())
    tp.tp_tree_build(ctx, 16, 30)
    errs = []
    for th in (1.0, 0.5, 0.25):
        g = np.zeros_like(V)
        e = tp.tp_gradient(ctx, g, tp.tp_params_default(mode=tp.TP_BH_DUAL, theta=th))
        scale = np.abs(g).sum()
        assert np.abs(g.sum(0)).max() <= 1e-6 * scale
        assert abs(np.sum(V * g) + 2 * e) <= 1e-5 * e
        errs.append((abs(e - ed) / ed, rel(g, gd)))
    assert errs[0][0] > errs[1][0] > errs[2][0] and errs[0][1] > errs[1][1] > errs[2][1], errs
