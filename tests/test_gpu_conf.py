"""Parity of the CUDA confinement energy (Eq. TPConf, Sec. 2.2, Confinement)
with the FP64 oracle (needs a GPU).

Bars as for the direct self-energy: energy within 1e-6 relative, vertex
gradient within 1e-5 relative L2 in the FP32 form; 1e-11 in the FP64 form.
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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def rotation(seed):
    Q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((3, 3)))
    return Q if np.linalg.det(Q) > 0 else -Q


@pytest.mark.parametrize("level,radius", [(3, 1.1), (4, 1.1), (4, 1.02)])
def test_conf_parity(tp, ctx, oracle_mod, level, radius):
    """Evolving perturbed sphere inside a rotated confining sphere (the paper's
    sphere-in-sphere setting, Sec. 4.3, radius 1.1; and a near-contact gap 0.02);
    level 4 spans several super-tiles with ragged tails on both surfaces."""
    V, F = meshgen.perturbed_sphere(level, 0.005, 11)
    Vc, Fc = meshgen.icosphere(level)
    Vc = radius * Vc @ rotation(level).T
    c = 1e-4 / 6
    E, g = oracle_mod.conf_gradient(V, F, Vc, Fc, c=c)
    tp.tp_mesh_upload(ctx, V, F)
    tp.tp_conf_upload(ctx, Vc, Fc)
    grad = np.zeros_like(V)
    e = tp.tp_conf_gradient(ctx, grad, tp.tp_params_default(scale=c))
    assert abs(e - E) <= E_TOL * E, (e, E)
    assert rel(grad, g) <= G_TOL, rel(grad, g)
    st = tp.tp_get_stats(ctx)
    assert st["pairs_exact"] == F.shape[0] * Fc.shape[0]
    e64 = tp.tp_conf_gradient(ctx, grad, tp.tp_params_default(scale=c, prec=tp._tp.TP_F64))
    assert abs(e64 - E) <= 1e-11 * E and rel(grad, g) <= 1e-11
    assert abs(tp.tp_conf_gradient(ctx, None, tp.tp_params_default(scale=c)) - E) <= E_TOL * E


def test_conf_device_and_f32_inputs(tp, ctx, oracle_mod):
    import torch

    V, F = meshgen.perturbed_sphere(3, 0.005, 12)
    Vc, Fc = meshgen.icosphere(3)
    Vc = 1.1 * Vc
    tp.tp_mesh_upload(ctx, V, F)
    tp.tp_conf_upload(ctx, torch.tensor(Vc, dtype=torch.float32, device="cuda"),
                      torch.tensor(Fc, device="cuda"))
    # the library widens f32 positions exactly, so the reference uses the rounded ones
    E32, g32 = oracle_mod.conf_gradient(V, F, Vc.astype(np.float32).astype(np.float64), Fc)
    gd = torch.zeros((V.shape[0], 3), dtype=torch.float32, device="cuda")
    e = tp.tp_conf_gradient(ctx, gd)
    assert abs(e - E32) <= E_TOL * E32
    assert rel(gd.cpu().numpy().astype(np.float64), g32) <= G_TOL


def test_conf_errors(tp, ctx):
    V, F = meshgen.icosphere(2)
    tp.tp_mesh_upload(ctx, V, F)
    with pytest.raises(tp.TPError) as ei:
        tp.tp_conf_gradient(ctx, np.zeros_like(V))
    assert ei.value.status == tp._tp.TP_E_STATE
    tp.tp_conf_upload(ctx, 1.1 * V, F)
    tp.tp_tree_build(ctx, 16, 30)
    with pytest.raises(tp.TPError) as ei:
        tp.tp_conf_gradient(ctx, np.zeros_like(V), tp.tp_params_default(mode=tp.TP_BH, theta=0.5))
    assert ei.value.status == tp._tp.TP_E_ARG
    with pytest.raises(tp.TPError) as ei:  # compensated FP32 sums exist for the direct self-energy only
        tp.tp_conf_gradient(ctx, np.zeros_like(V), tp.tp_params_default(prec=tp._tp.TP_F32_KAHAN))
    assert ei.value.status == tp._tp.TP_E_ARG
    bad = F.copy()
    bad[3, 1] = V.shape[0] + 5
    with pytest.raises(tp.TPError) as ei:
        tp.tp_conf_upload(ctx, V, bad)
    assert ei.value.status == tp._tp.TP_E_ARG
    # touching surfaces (the confinement through the same points): +inf and TP_E_NONFINITE
    tp.tp_conf_upload(ctx, V, F)
    with pytest.raises(tp.TPError) as ei:
        tp.tp_conf_gradient(ctx, np.zeros_like(V))
    assert ei.value.status == tp._tp.TP_E_NONFINITE
    # the context stays usable
    tp.tp_conf_upload(ctx, 1.1 * V, F)
    assert np.isfinite(tp.tp_conf_gradient(ctx, None))


def test_conf_full_size_sampled(tp, ctx, oracle_mod):
    """327,680-triangle sphere in a 327,680-triangle confining sphere (radius 1.1):
    energy against the FP64 form of the library (pinned above) and the gradient at
    sampled vertices against the oracle computed vertex by vertex."""
    V, F = meshgen.perturbed_sphere(7, 0.005, 13)
    Vc, Fc = meshgen.icosphere(7)
    Vc = 1.1 * Vc
    tp.tp_mesh_upload(ctx, V, F)
    tp.tp_conf_upload(ctx, Vc, Fc)
    grad = np.zeros_like(V)
    e = tp.tp_conf_gradient(ctx, grad)
    e64 = tp.tp_conf_gradient(ctx, None, tp.tp_params_default(prec=tp._tp.TP_F64))
    assert abs(e - e64) <= E_TOL * e64
    verts = np.random.default_rng(5).choice(V.shape[0], 24, replace=False)
    go = oracle_mod.conf_vertex_gradient_sample(V, F, Vc, Fc, verts)
    assert rel(grad[verts], go) <= G_TOL, rel(grad[verts], go)
