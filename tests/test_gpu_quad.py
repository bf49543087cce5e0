"""Parity of the multi-point quadrature form (tp_set_quadrature; Sec. 3.1, 3.2)
with the FP64 oracle (needs a GPU).  Same bars as the one-point form: energy
1e-6, gradient 1e-5 relative L2 in FP32; 1e-11 in the FP64 form."""

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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


@pytest.mark.parametrize("k", [3, 6])
def test_quad_parity(tp, ctx, oracle_mod, k):
    """1,280 triangles x k points: 3,840 or 7,680 elements, several super-tiles with a ragged tail."""
    V, F = meshgen.perturbed_sphere(3, 0.01, 21)
    c = 0.5
    E, g = oracle_mod.quad_gradient(V, F, k, c=c)
    tp.tp_set_quadrature(ctx, k)
    tp.tp_mesh_upload(ctx, V, F)
    assert tp.tp_get_stats(ctx)["nt"] == k * F.shape[0]
    grad = np.zeros_like(V)
    e = tp.tp_gradient(ctx, grad, tp.tp_params_default(scale=c))
    assert abs(e - E) <= E_TOL * E, (e, E)
    assert rel(grad, g) <= G_TOL, rel(grad, g)
    e64 = tp.tp_gradient(ctx, grad, tp.tp_params_default(scale=c, prec=tp._tp.TP_F64))
    assert abs(e64 - E) <= 1e-11 * E and rel(grad, g) <= 1e-11
    assert abs(tp.tp_energy(ctx, tp.tp_params_default(scale=c)) - E) <= E_TOL * E
    # positions-only re-upload keeps the rule
    V2 = V * 1.01
    E2, g2 = oracle_mod.quad_gradient(V2, F, k, c=c)
    tp.tp_mesh_upload(ctx, V2, None, flags=tp._tp.TP_POSITIONS_ONLY)
    e2 = tp.tp_gradient(ctx, grad, tp.tp_params_default(scale=c))
    assert abs(e2 - E2) <= E_TOL * E2 and rel(grad, g2) <= G_TOL
    # per-element fields: k per triangle, in the caller's triangle order
    e3, fw, fnu, fx = tp.tp_fields(ctx, k * F.shape[0], tp.tp_params_default(scale=c))
    x, nu, w, Fq = oracle_mod.quad_points(V2, F, k)
    ow, onu, ox = oracle_mod.tri_accum(V2, Fq, soa=(x, nu, w))
    assert rel(fw, c * ow) <= G_TOL and rel(fnu, c * onu) <= G_TOL and rel(fx, c * ox) <= G_TOL


def test_quad_bh_theta_zero_and_reset(tp, ctx, oracle_mod):
    V, F = meshgen.perturbed_sphere(3, 0.01, 22)
    tp.tp_set_quadrature(ctx, 3)
    tp.tp_mesh_upload(ctx, V, F)
    gd = np.zeros_like(V)
    ed = tp.tp_gradient(ctx, gd, tp.tp_params_default())
    tp.tp_tree_build(ctx, 16, 30)
    gb = np.zeros_like(V)
    eb = tp.tp_gradient(ctx, gb, tp.tp_params_default(mode=tp.TP_BH, theta=0.0))
    assert abs(eb - ed) <= 1e-6 * ed and rel(gb, gd) <= 1e-5
    # back to the centroid rule
    tp.tp_set_quadrature(ctx, 1)
    tp.tp_mesh_upload(ctx, V, F)
    E1, g1 = oracle_mod.gradient(V, F)
    g = np.zeros_like(V)
    assert abs(tp.tp_gradient(ctx, g, tp.tp_params_default()) - E1) <= E_TOL * E1 and rel(g, g1) <= G_TOL
    with pytest.raises(tp.TPError) as ei:
        tp.tp_set_quadrature(ctx, 4)
    assert ei.value.status == tp._tp.TP_E_ARG
