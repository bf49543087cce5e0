"""Parity of the CUDA direct path with the FP64 oracle (needs a GPU).

Bars (from the accuracy the direct FP32 form is held to): energy within
1e-6 relative, gradient within 1e-5 relative L2 of the FP64 oracle; FP64
mode within 1e-11.  Integer/index work (Morton order) is bit-exact.
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


def maxrel(a, b):
    """Largest per-entry deviation relative to the largest reference entry."""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def params(tp, **kw):
    return tp.tp_params_default(**kw)


def closed_mesh_admitted(F, adj):
    """Ordered admitted pairs of a closed mesh: nt (nt - 1) minus twice the unordered pairs
    sharing a vertex (sum_v C(d_v, 2) - E) or an edge (E)."""
    nt = F.shape[0]
    E = 3 * nt // 2
    deg = np.bincount(F.ravel())
    excl = E if adj == 1 else int(np.sum(deg * (deg - 1) // 2)) - E
    return nt * (nt - 1) - 2 * excl


@pytest.fixture(scope="module")
def sphere3(oracle_mod):
    V, F = meshgen.workload("sphere_l3")
    E, g = oracle_mod.gradient(V, F)
    return V, F, E, g


@pytest.fixture(scope="module")
def dish5(oracle_mod):
    V, F = meshgen.workload("dish_l5")
    E, g = oracle_mod.gradient(V, F)
    return V, F, E, g


def test_tri_data_and_order_bitexact(tp, ctx, oracle_mod):
    for name in ("sphere_l3", "dish_l5"):
        V, F = meshgen.workload(name)
        tp.tp_mesh_upload(ctx, V, F)
        perm, x, nu, w = tp.tp_debug_tri_data(ctx, F.shape[0])
        xo, nuo, wo = oracle_mod.tri_data(V, F)
        t = oracle_mod.lbvh(xo, 30, 16)
        assert np.array_equal(perm, t["perm"])
        assert np.array_equal(x, xo[perm]) and np.array_equal(nu, nuo[perm]) and np.array_equal(w, wo[perm])


@pytest.mark.parametrize("mesh", ["sphere3", "dish5"])
def test_direct_energy_gradient(tp, ctx, mesh, request):
    V, F, E, g = request.getfixturevalue(mesh)
    tp.tp_mesh_upload(ctx, V, F)
    e = tp.tp_energy(ctx, params(tp))
    assert abs(e - E) <= E_TOL * E, (e, E)
    grad = np.zeros_like(V)
    e2 = tp.tp_gradient(ctx, grad, params(tp))
    assert abs(e2 - E) <= E_TOL * E, (e2, E)
    assert rel(grad, g) <= G_TOL, rel(grad, g)
    assert maxrel(grad, g) <= G_TOL, maxrel(grad, g)


@pytest.mark.parametrize("name", ["sphere_l3", "dish_l5"])
def test_admitted_pair_count(tp, ctx, oracle_mod, name):
    """The direct form's pair count (the numerator of the benchmark's rate) equals the
    oracle's count of the ordered pairs its sum runs over, for both exclusion rules."""
    V, F = meshgen.workload(name)
    tp.tp_mesh_upload(ctx, V, F)
    for adj, flags in ((0, 0), (1, tp._tp.TP_EXCLUDE_EDGE)):
        want = oracle_mod.admitted_pairs(F, adj=adj)
        grad = np.zeros_like(V)
        tp.tp_gradient(ctx, grad, params(tp, flags=flags))
        assert tp.tp_get_stats(ctx)["pairs_exact"] == want
        tp.tp_energy(ctx, params(tp, flags=flags))
        assert tp.tp_get_stats(ctx)["pairs_exact"] == want


@pytest.mark.parametrize("mesh", ["sphere3", "dish5"])
def test_direct_f64_mode(tp, ctx, mesh, request):
    V, F, E, g = request.getfixturevalue(mesh)
    tp.tp_mesh_upload(ctx, V, F)
    p = params(tp, prec=tp.TP_F64)
    e = tp.tp_energy(ctx, p)
    assert abs(e - E) <= 1e-11 * E
    grad = np.zeros_like(V)
    e2 = tp.tp_gradient(ctx, grad, p)
    assert abs(e2 - E) <= 1e-11 * E
    assert rel(grad, g) <= 1e-10


@pytest.mark.parametrize("mesh", ["sphere3", "dish5"])
def test_direct_kahan_mode(tp, ctx, oracle_mod, mesh, request):
    """TP_F32_KAHAN: FP32 pair terms with every per-triangle sum compensated in FP32 (no
    FP64 accumulation), held to the same bars as the FP64-accumulation form."""
    V, F, E, g = request.getfixturevalue(mesh)
    tp.tp_mesh_upload(ctx, V, F)
    p = params(tp, prec=tp._tp.TP_F32_KAHAN)
    e = tp.tp_energy(ctx, p)
    assert abs(e - E) <= E_TOL * E, (e, E)
    grad = np.zeros_like(V)
    e2 = tp.tp_gradient(ctx, grad, p)
    assert abs(e2 - E) <= E_TOL * E
    assert rel(grad, g) <= G_TOL and maxrel(grad, g) <= G_TOL, (rel(grad, g), maxrel(grad, g))
    gw, gnu, gx = tp.tp_debug_accum(ctx, F.shape[0])
    ow, onu, ox = oracle_mod.tri_accum(V, F)
    assert rel(gw, ow) <= E_TOL and rel(gnu, onu) <= G_TOL and rel(gx, ox) <= G_TOL
    Ee, ge = oracle_mod.gradient(V, F, adj=1)
    e3 = tp.tp_gradient(ctx, grad, params(tp, prec=tp._tp.TP_F32_KAHAN, flags=tp._tp.TP_EXCLUDE_EDGE))
    assert abs(e3 - Ee) <= E_TOL * Ee and rel(grad, ge) <= G_TOL
    E8, g8 = oracle_mod.gradient(V, F, 8.0, 16.0)
    e8 = tp.tp_gradient(ctx, grad, params(tp, prec=tp._tp.TP_F32_KAHAN, q=8, p=16))
    assert abs(e8 - E8) <= E_TOL * E8 and rel(grad, g8) <= G_TOL


def test_precision_options_of_other_forms(tp, ctx, sphere3):
    """The clustered forms run FP32 terms with FP64 sums only; other precisions are refused."""
    V, F, _, _ = sphere3
    tp.tp_mesh_upload(ctx, V, F)
    tp.tp_tree_build(ctx, 16, 30)
    for mode in (tp.TP_BH,):
        for prec in (tp._tp.TP_F32_KAHAN, tp.TP_F64):
            with pytest.raises(tp.TPError) as ei:
                tp.tp_energy(ctx, params(tp, mode=mode, prec=prec))
            assert ei.value.status == tp._tp.TP_E_ARG
    assert tp.tp_energy(ctx, params(tp, mode=tp.TP_BH)) > 0


def test_per_triangle_accumulators(tp, ctx, oracle_mod, sphere3):
    V, F, _, _ = sphere3
    tp.tp_mesh_upload(ctx, V, F)
    grad = np.zeros_like(V)
    tp.tp_gradient(ctx, grad, params(tp))
    gw, gnu, gx = tp.tp_debug_accum(ctx, F.shape[0])
    ow, onu, ox = oracle_mod.tri_accum(V, F)
    assert rel(gw, ow) <= 1e-6
    assert rel(gnu, onu) <= G_TOL
    assert rel(gx, ox) <= G_TOL


def test_scale_and_exponents(tp, ctx, oracle_mod, sphere3):
    V, F, E, g = sphere3
    tp.tp_mesh_upload(ctx, V, F)
    c = 1e-4 / 6.0
    e = tp.tp_energy(ctx, params(tp, scale=c))
    assert abs(e - c * E) <= E_TOL * c * E
    E8, g8 = oracle_mod.gradient(V, F, 8.0, 16.0)
    grad = np.zeros_like(V)
    e8 = tp.tp_gradient(ctx, grad, params(tp, q=8, p=16))
    assert abs(e8 - E8) <= E_TOL * E8
    assert rel(grad, g8) <= G_TOL


def test_edge_exclusion_mode(tp, ctx, oracle_mod, sphere3):
    V, F, _, _ = sphere3
    Ee, ge = oracle_mod.gradient(V, F, adj=1)
    tp.tp_mesh_upload(ctx, V, F)
    grad = np.zeros_like(V)
    e = tp.tp_gradient(ctx, grad, params(tp, flags=tp._tp.TP_EXCLUDE_EDGE))
    assert abs(e - Ee) <= E_TOL * Ee
    assert rel(grad, ge) <= G_TOL
    assert maxrel(grad, ge) <= G_TOL


@pytest.mark.parametrize("nt_keep", [1, 2, 37, 1023, 1025, 2049])
def test_ragged_sizes(tp, ctx, oracle_mod, nt_keep):
    """Open sub-meshes whose sizes do not fill a tile (and a 1-triangle mesh)."""
    V, F = meshgen.perturbed_sphere(4, 0.01, 3)
    F = np.ascontiguousarray(F[:nt_keep])
    E, g = oracle_mod.gradient(V, F)
    tp.tp_mesh_upload(ctx, V, F)
    grad = np.zeros_like(V)
    e = tp.tp_gradient(ctx, grad, params(tp))
    if E == 0.0:
        assert e == 0.0 and not grad.any()
        return
    assert abs(e - E) <= E_TOL * E
    assert rel(grad, g) <= G_TOL
    assert maxrel(grad, g) <= G_TOL
    assert tp.tp_get_stats(ctx)["pairs_exact"] == oracle_mod.admitted_pairs(F)
    assert abs(tp.tp_energy(ctx, params(tp)) - E) <= E_TOL * E
    grad = np.zeros_like(V)
    e_k = tp.tp_gradient(ctx, grad, params(tp, prec=tp._tp.TP_F32_KAHAN))
    assert abs(e_k - E) <= E_TOL * E and rel(grad, g) <= G_TOL
    tp.tp_gradient(ctx, grad, params(tp, flags=tp._tp.TP_EXCLUDE_EDGE))
    assert tp.tp_get_stats(ctx)["pairs_exact"] == oracle_mod.admitted_pairs(F, adj=1)


def test_empty_mesh(tp, ctx):
    V = np.zeros((4, 3))
    F = np.zeros((0, 3), dtype=np.int32)
    tp.tp_mesh_upload(ctx, V, F)
    assert tp.tp_energy(ctx, params(tp)) == 0.0
    grad = np.ones_like(V)
    assert tp.tp_gradient(ctx, grad, params(tp)) == 0.0
    assert not grad.any()


def test_device_pointers_and_f32_input(tp, ctx, sphere3):
    import torch

    V, F, E, g = sphere3
    Vd = torch.tensor(V, device="cuda")
    Fd = torch.tensor(F, device="cuda")
    tp.tp_mesh_upload(ctx, Vd, Fd)
    gd = torch.zeros_like(Vd)
    e = tp.tp_gradient(ctx, gd, params(tp))
    assert abs(e - E) <= E_TOL * E
    assert rel(gd.cpu().numpy(), g) <= G_TOL
    g32 = torch.zeros(V.shape, dtype=torch.float32, device="cuda")
    tp.tp_gradient(ctx, g32, params(tp))
    assert rel(g32.cpu().numpy(), g) <= 1e-5
    # float32 positions: compare with the oracle on the rounded positions
    V32 = V.astype(np.float32)
    tp.tp_mesh_upload(ctx, V32, F)
    import oracle

    E32 = oracle.energy(V32.astype(np.float64), F)
    assert abs(tp.tp_energy(ctx, params(tp)) - E32) <= E_TOL * E32


def test_positions_only_reupload(tp, ctx, oracle_mod, sphere3):
    V, F, _, _ = sphere3
    tp.tp_mesh_upload(ctx, V, F)
    V2 = V * 1.01 + 0.003 * np.sin(7 * V)
    tp.tp_mesh_upload(ctx, V2, None, flags=tp._tp.TP_POSITIONS_ONLY)
    E2, g2 = oracle_mod.gradient(V2, F)
    grad = np.zeros_like(V)
    e = tp.tp_gradient(ctx, grad, params(tp))
    assert abs(e - E2) <= E_TOL * E2
    assert rel(grad, g2) <= G_TOL


def test_error_statuses(tp, ctx):
    V, F = meshgen.icosphere(2)
    with pytest.raises(tp.TPError) as ei:
        tp.tp_energy(ctx, params(tp))
    assert ei.value.status == tp._tp.TP_E_STATE
    bad = F.copy()
    bad[5, 1] = V.shape[0] + 3
    with pytest.raises(tp.TPError) as ei:
        tp.tp_mesh_upload(ctx, V, bad)
    assert ei.value.status == tp._tp.TP_E_ARG
    deg = F.copy()
    deg[3, 2] = deg[3, 1]
    with pytest.raises(tp.TPError) as ei:
        tp.tp_mesh_upload(ctx, V, deg)
    assert ei.value.status == tp._tp.TP_E_NONFINITE
    Vn = V.copy()
    Vn[0, 0] = np.nan
    with pytest.raises(tp.TPError) as ei:
        tp.tp_mesh_upload(ctx, Vn, F)
    assert ei.value.status == tp._tp.TP_E_NONFINITE
    # the context stays usable
    tp.tp_mesh_upload(ctx, V, F)
    assert tp.tp_energy(ctx, params(tp)) > 0
    with pytest.raises(tp.TPError) as ei:
        tp.tp_energy(ctx, params(tp, q=5, p=10))
    assert ei.value.status == tp._tp.TP_E_ARG
    with pytest.raises(tp.TPError) as ei:
        tp.tp_energy(ctx, params(tp, mode=tp.TP_BH))
    assert ei.value.status == tp._tp.TP_E_STATE


def test_coincident_centroids_nonfinite(tp, ctx):
    """Two admitted triangles with the same centroid: not embedded, Phi = +inf."""
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.2, 0.2, -0.5], [0.2, 0.2, 0.5], [-0.4 + 0.6, 0.6 - 0.4 + 0.2, 0.0]])
    # triangle 0 centroid (1/3, 1/3, 0); triangle 1 = (3, 4, 5) with the same centroid
    V[5] = 3 * np.array([1 / 3, 1 / 3, 0.0]) - V[3] - V[4]
    F = np.array([[0, 1, 2], [3, 4, 5]], dtype=np.int32)
    tp.tp_mesh_upload(ctx, V, F)
    with pytest.raises(tp.TPError) as ei:
        tp.tp_energy(ctx, params(tp))
    assert ei.value.status == tp._tp.TP_E_NONFINITE


def test_autograd_function(tp, oracle_mod, dish5):
    import torch

    V, F, E, g = dish5
    tpe = tp.TangentPointEnergy(F)
    Vt = torch.tensor(V, device="cuda", requires_grad=True)
    e = tpe(Vt)
    e.backward()
    assert abs(float(e.detach()) - E) <= E_TOL * E
    assert rel(Vt.grad.cpu().numpy(), g) <= G_TOL
    # forward and backward together made one pass over the pairs
    assert tpe.calls == {"energy": 0, "gradient": 1}, tpe.calls
    # finite differences of the FP64 oracle energy (h = 1e-6, 32 seeded vertices)
    rng = np.random.default_rng(11)
    verts = rng.choice(V.shape[0], 32, replace=False)
    axes = rng.integers(0, 3, 32)
    gg = Vt.grad.cpu().numpy()
    h = 1e-6
    for v, k in zip(verts, axes):
        tris = oracle_mod.incident_triangles(F, [v])
        Vp, Vm = V.copy(), V.copy()
        Vp[v, k] += h
        Vm[v, k] -= h
        fd = (oracle_mod.energy_touching(Vp, F, tris) - oracle_mod.energy_touching(Vm, F, tris)) / (2 * h)
        assert abs(gg[v, k] - fd) <= 1e-5 * np.abs(g).max() + 1e-4 * abs(fd), (v, k, gg[v, k], fd)
    with torch.no_grad():
        e0 = tpe(torch.tensor(V, device="cuda"))
    assert abs(float(e0) - E) <= E_TOL * E and tpe.calls == {"energy": 1, "gradient": 1}, tpe.calls
    # the backward scales the kept gradient by the incoming one
    Vt.grad = None
    (3.0 * tpe(Vt)).backward()
    assert rel(Vt.grad.cpu().numpy(), 3.0 * g) <= G_TOL
    tpe.close()


def test_full_size_properties(tp, ctx, oracle_mod):
    """Level-7 SH-deformed sphere (327,680 triangles) in the benchmark's launch
    configuration: sampled per-triangle derivatives and vertex gradients
    against the oracle, and the invariants that hold at any size."""
    V, F = meshgen.workload("sh_l7")
    tp.tp_mesh_upload(ctx, V, F)
    grad = np.zeros_like(V)
    e = tp.tp_gradient(ctx, grad, params(tp))
    assert tp.tp_get_stats(ctx)["pairs_exact"] == closed_mesh_admitted(F, 0)
    e_only = tp.tp_energy(ctx, params(tp))
    assert abs(e - e_only) <= 1e-6 * e
    rng = np.random.default_rng(0)
    tris = rng.choice(F.shape[0], 48, replace=False)
    gw, gnu, gx = tp.tp_debug_accum(ctx, F.shape[0])
    ow, onu, ox = oracle_mod.tri_accum(V, F, tris)
    assert rel(gw[tris], ow) <= 1e-6
    assert rel(gnu[tris], onu) <= G_TOL
    assert rel(gx[tris], ox) <= G_TOL
    verts = rng.choice(V.shape[0], 12, replace=False)
    gs = oracle_mod.vertex_gradient_sample(V, F, verts)
    assert rel(grad[verts], gs) <= G_TOL
    assert maxrel(grad[verts], gs) <= G_TOL
    # the whole energy and gradient against the FP64 form (FP64 pair terms and sums, the
    # kernel test_direct_f64_mode holds to the oracle within 1e-11).  Per vertex the bar is
    # wider than in L2: a target's FP32 partial over one 1536-source item can lose up to
    # ~1536 u (u = 2^-24, about 1e-4) of the sum of its terms' magnitudes, and the forces on
    # a vertex cancel; measured 3.0e-5 of max |g| at this size against 6.2e-6 in L2
    g64 = np.zeros_like(V)
    e64 = tp.tp_gradient(ctx, g64, params(tp, prec=tp.TP_F64))
    assert abs(e - e64) <= E_TOL * e64, (e, e64)
    assert rel(grad, g64) <= G_TOL and maxrel(grad, g64) <= 1e-4, (rel(grad, g64), maxrel(grad, g64))
    scale = np.abs(grad).sum()
    assert np.abs(grad.sum(0)).max() <= 1e-6 * scale
    assert np.abs(np.cross(V, grad).sum(0)).max() <= 1e-6 * scale
    assert abs(np.sum(V * grad) + 2 * e) <= 1e-5 * e


@pytest.mark.parametrize("mesh", ["sphere3", "dish5"])
def test_triangle_fields(tp, ctx, oracle_mod, mesh, request):
    """tp_fields: per-triangle dPhi/dw, dPhi/dnu, dPhi/dx (caller's order, with the
    prefactor) against the oracle's, in the FP32 and FP64 forms, host and device
    outputs, and through the Barnes-Hut path at theta = 0 (no cluster admitted)."""
    import torch

    V, F, E, _ = request.getfixturevalue(mesh)
    c = 0.37
    gw, gnu, gx = oracle_mod.tri_accum(V, F)
    gw, gnu, gx = c * gw, c * gnu, c * gx
    tp.tp_mesh_upload(ctx, V, F)
    e, fw, fnu, fx = tp.tp_fields(ctx, F.shape[0], tp.tp_params_default(scale=c))
    assert abs(e - c * E) <= E_TOL * c * E
    assert rel(fw, gw) <= G_TOL and rel(fnu, gnu) <= G_TOL and rel(fx, gx) <= G_TOL, (rel(fw, gw), rel(fnu, gnu),
                                                                                   rel(fx, gx))
    e, fw, fnu, fx = tp.tp_fields(ctx, F.shape[0], tp.tp_params_default(scale=c, prec=tp._tp.TP_F64))
    assert rel(fw, gw) <= 1e-11 and rel(fnu, gnu) <= 1e-11 and rel(fx, gx) <= 1e-11
    d = [torch.zeros(F.shape[0], dtype=torch.float64, device="cuda"),
         torch.zeros((F.shape[0], 3), dtype=torch.float64, device="cuda"), None]
    tp.tp_fields(ctx, F.shape[0], tp.tp_params_default(scale=c), fw=d[0], fnu=d[1])
    torch.cuda.synchronize()
    assert rel(d[0].cpu().numpy(), gw) <= G_TOL and rel(d[1].cpu().numpy(), gnu) <= G_TOL
    tp.tp_tree_build(ctx, 16, 30)
    e, fw, fnu, fx = tp.tp_fields(ctx, F.shape[0], tp.tp_params_default(scale=c, mode=tp.TP_BH, theta=0.0))
    assert rel(fw, gw) <= G_TOL and rel(fnu, gnu) <= G_TOL and rel(fx, gx) <= G_TOL
