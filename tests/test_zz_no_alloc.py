"""The allocation-free entry point against the regular one (needs a GPU).

tp_gradient_direct_noalloc serves callers that cannot allocate device
memory where they need the energy (graph recording, host-owned memory
pools, allocation-free control loops).  It must give the same energy and
gradient as tp_gradient in TP_DIRECT mode, within the direct path's
tolerances (energy 1e-6 relative, gradient 1e-5 relative L2), on two calls
in a row - its scratch array keeps the previous call's contents - and
after a call on a different mesh; it must also match the FP64 oracle
directly, refuse precisions and dtypes it does not implement, and turn a
bad face index into NaN outputs without touching memory out of bounds.
This file is collected last so that a run stopping at the first failure has
run every other test already.
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


def regular(tp, V, F, **kw):
    import torch

    ctx = tp.tp_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        tp.tp_mesh_upload(ctx, V, F)
        g = torch.zeros_like(V)
        e = tp.tp_gradient(ctx, g, tp.tp_params_default(**kw))
    finally:
        tp.tp_destroy(ctx)
    return e, g


def noalloc(tp, V, F, **kw):
    import torch

    e = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    g = torch.full_like(V, float("nan"))
    tp._tp.tp_gradient_direct_noalloc(V, F, e, g, tp.tp_params_default(**kw),
                                      stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return float(e.item()), g


def check(e, g, e_ref, g_ref):
    import torch

    assert abs(e - e_ref) <= E_TOL * abs(e_ref), (e, e_ref)
    assert float(torch.linalg.norm(g - g_ref) / torch.linalg.norm(g_ref)) <= G_TOL


def test_noalloc_matches_regular_entry_point(tp):
    import torch

    V, F = meshgen.workload("dish_l5")
    Vd = torch.tensor(V, device="cuda")
    Fd = torch.tensor(F, device="cuda")
    e_ref, g_ref = regular(tp, Vd, Fd)
    for _ in range(2):  # two calls in a row share the scratch array
        e, g = noalloc(tp, Vd, Fd)
        check(e, g, e_ref, g_ref)
    # a smaller mesh after a larger one: stale scratch must not leak in
    V2, F2 = meshgen.workload("sphere_l3")
    V2d = torch.tensor(V2, device="cuda")
    F2d = torch.tensor(F2, device="cuda")
    e2_ref, g2_ref = regular(tp, V2d, F2d, scale=1e-4 / 6.0)
    e2, g2 = noalloc(tp, V2d, F2d, scale=1e-4 / 6.0)
    check(e2, g2, e2_ref, g2_ref)


def test_noalloc_rejects_oversized_mesh(tp):
    import torch

    V, F = meshgen.icosphere(6)  # 81,920 triangles > 65,536
    Vd = torch.tensor(V, device="cuda")
    Fd = torch.tensor(F, device="cuda")
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.zeros_like(Vd)
    with pytest.raises(tp.TPError) as ei:
        tp._tp.tp_gradient_direct_noalloc(Vd, Fd, e, g, tp.tp_params_default())
    assert ei.value.status == tp._tp.TP_E_ARG
    assert "maximum" in str(ei.value)


def test_noalloc_matches_oracle(tp, oracle_mod):
    """Directly against the FP64 oracle, not only against the regular entry point."""
    import torch

    V, F = meshgen.workload("sphere_l3")
    E, g_ref = oracle_mod.gradient(V, F, c=0.5)
    e, g = noalloc(tp, torch.tensor(V, device="cuda"), torch.tensor(F, device="cuda"), scale=0.5)
    check(e, g, E, torch.tensor(g_ref, device="cuda"))
    gh = g.cpu().numpy()
    assert np.abs(gh - g_ref).max() <= G_TOL * np.abs(g_ref).max()


def test_noalloc_rejects_other_precisions_and_dtypes(tp):
    import torch

    V, F = meshgen.workload("sphere_l3")
    Vd = torch.tensor(V, device="cuda")
    Fd = torch.tensor(F, device="cuda")
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.zeros_like(Vd)
    for prec in (tp.TP_F64, tp._tp.TP_F32_KAHAN):
        with pytest.raises(tp.TPError) as ei:
            tp._tp.tp_gradient_direct_noalloc(Vd, Fd, e, g, tp.tp_params_default(prec=prec))
        assert ei.value.status == tp._tp.TP_E_ARG
    with pytest.raises(TypeError):
        tp._tp.tp_gradient_direct_noalloc(Vd.float(), Fd, e, g)
    with pytest.raises(TypeError):
        tp._tp.tp_gradient_direct_noalloc(Vd, Fd.long(), e, g)


def test_noalloc_bad_index_gives_nan(tp):
    """A face index outside [0, nv) is caught by the kernels' own bounds checks (the
    triangle's data becomes NaN and the pull-back skips it): NaN energy, status TP_OK."""
    import torch

    V, F = meshgen.workload("sphere_l3")
    bad = F.copy()
    bad[17, 1] = V.shape[0] + 5
    e, g = noalloc(tp, torch.tensor(V, device="cuda"), torch.tensor(bad, device="cuda"))
    assert np.isnan(e)
    # a later call on a good mesh is unaffected
    Vd = torch.tensor(V, device="cuda")
    Fd = torch.tensor(F, device="cuda")
    e_ref, g_ref = regular(tp, Vd, Fd)
    e2, g2 = noalloc(tp, Vd, Fd)
    check(e2, g2, e_ref, g_ref)
