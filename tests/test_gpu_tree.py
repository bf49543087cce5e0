"""Parity of the CUDA cluster tree and Barnes-Hut form with the oracle (needs a GPU).

Bars: Morton codes, permutation, tree children, ranges and cluster leaves
bit-exact; FP64 moments and boxes bit-exact (same rounding order on both
sides); Barnes-Hut energy within 1e-6 relative and gradient within 1e-5
relative L2 of the oracle's Barnes-Hut at the same theta (identical
admissibility decisions, FP32 pair terms on the GPU); theta = 0 equals the
direct sum.
"""

import pathlib

import numpy as np
import pytest

from paper_2509_22110_gb300 import meshgen

ROOT = pathlib.Path(__file__).resolve().parents[1]

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


MESHES = {
    "sh_l4": lambda: meshgen.sh_deformed_sphere(4, 12, 0.05, 2),
    "dish_l5": lambda: meshgen.workload("dish_l5"),
    "open_777": lambda: (meshgen.perturbed_sphere(4, 0.01, 5)[0],
                         np.ascontiguousarray(meshgen.perturbed_sphere(4, 0.01, 5)[1][:777])),
}


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("leaf,bits", [(16, 30), (1, 30), (32, 15), (7, 24)])
def test_tree_bitexact(tp, ctx, oracle_mod, name, leaf, bits):
    V, F = MESHES[name]()
    nt = F.shape[0]
    tp.tp_mesh_upload(ctx, V, F)
    tp.tp_tree_build(ctx, leaf, bits)
    g = tp.tp_debug_tree(ctx, nt)
    x, nu, w = oracle_mod.tri_data(V, F)
    o = oracle_mod.lbvh(x, bits, leaf)
    assert np.array_equal(g["codes"], o["codes"])
    assert np.array_equal(g["perm"], o["perm"])
    assert np.array_equal(g["left"], o["left"]) and np.array_equal(g["right"], o["right"])
    assert np.array_equal(g["first"], o["first"]) and np.array_equal(g["last"], o["last"])
    assert np.array_equal(g["leaves"], o["leaves"])
    mom, box = oracle_mod.moments(V, F, o, soa=(x, nu, w))
    assert np.array_equal(g["mom"], mom)
    assert np.array_equal(g["box"], box)


def _sort_cases():
    rng = np.random.default_rng(21)
    for n in (1, 2, 31, 2047, 2048, 2049, 100003):
        for bits in (30, 8, 6, 31, 32):
            hi = 1 << bits
            yield n, bits, rng.integers(0, hi, n, dtype=np.uint64).astype(np.uint32)  # mostly distinct
            yield n, bits, rng.integers(0, min(hi, 37), n, dtype=np.uint64).astype(np.uint32)  # many ties
    yield 5000, 30, np.full(5000, 12345, dtype=np.uint32)  # all equal
    yield 5000, 30, np.arange(5000, 0, -1, dtype=np.uint32)  # reversed


def test_key_sort_and_compaction(tp, ctx):
    """The tree build's own stable radix sort (ties keep input order: the order of the
    keys code << 32 | index) and leaf compaction against numpy on adversarial inputs."""
    for n, bits, keys in _sort_cases():
        ko, po, co = tp._tp.tp_debug_sort(ctx, keys, bits, compact=True)
        want = np.argsort(keys, kind="stable")
        assert np.array_equal(po, want), (n, bits)
        assert np.array_equal(ko, keys[want]), (n, bits)
        k32 = keys.view(np.int32)
        assert np.array_equal(co, k32[k32 >= 0]), (n, bits)


def test_tree_single_triangle(tp, ctx, oracle_mod):
    V, F = meshgen.icosahedron()
    F = np.ascontiguousarray(F[:1])
    tp.tp_mesh_upload(ctx, V, F)
    tp.tp_tree_build(ctx, 16, 30)
    g = tp.tp_debug_tree(ctx, 1)
    assert list(g["leaves"]) == [0]
    p = tp.tp_params_default(mode=tp.TP_BH, theta=0.5)
    assert tp.tp_energy(ctx, p) == 0.0


@pytest.mark.parametrize("theta", [0.0, 0.125, 0.25, 0.5, 1.0])
def test_bh_parity_with_oracle(tp, ctx, oracle_mod, theta):
    V, F = meshgen.sh_deformed_sphere(5, 12, 0.05, 2)
    Eo, go, info = oracle_mod.bh_gradient(V, F, theta)
    tp.tp_mesh_upload(ctx, V, F)
    tp.tp_tree_build(ctx, 16, 30)
    p = tp.tp_params_default(mode=tp.TP_BH, theta=theta)
    grad = np.zeros_like(V)
    e = tp.tp_gradient(ctx, grad, p)
    st = tp.tp_get_stats(ctx)
    assert st["far_terms"] == info["far_terms"]
    assert st["pairs_exact"] == info["near_pairs"]
    # the near-field kernel's pairs (clusters apart from the leaf) are part of the exact pairs,
    # and its launch is part of the evaluation
    assert 0 < st["kernel_pairs"] <= st["pairs_exact"]
    assert 0.0 < st["ms_kernel"] <= st["ms_total"]
    assert abs(e - Eo) <= E_TOL * Eo, (e, Eo)
    assert rel(grad, go) <= G_TOL, rel(grad, go)
    assert abs(tp.tp_energy(ctx, p) - Eo) <= E_TOL * Eo


@pytest.mark.parametrize("leaf,q,adj", [(32, 6, 0), (24, 8, 1), (7, 8, 0), (1, 6, 1)])
def test_bh_parity_leaf_sizes_and_options(tp, ctx, oracle_mod, leaf, q, adj):
    """Leaves above 16 targets (one target per lane), small leaves, q = 8 and
    edge-only exclusion against the oracle's Barnes-Hut sums."""
    V, F = meshgen.sh_deformed_sphere(4, 12, 0.05, 3)
    Eo, go, info = oracle_mod.bh_gradient(V, F, 0.5, q=q, p=2 * q, adj=adj, leaf_size=leaf)
    tp.tp_mesh_upload(ctx, V, F)
    tp.tp_tree_build(ctx, leaf, 30)
    p = tp.tp_params_default(mode=tp.TP_BH, theta=0.5, q=q, p=2 * q,
                             flags=tp._tp.TP_EXCLUDE_EDGE if adj else 0)
    grad = np.zeros_like(V)
    e = tp.tp_gradient(ctx, grad, p)
    st = tp.tp_get_stats(ctx)
    assert st["far_terms"] == info["far_terms"] and info["far_terms"] > 0
    assert st["pairs_exact"] == info["near_pairs"]
    assert abs(e - Eo) <= E_TOL * Eo, (e, Eo)
    assert rel(grad, go) <= G_TOL, rel(grad, go)


def test_direct_after_tree_build_and_position_updates(tp, ctx):
    """The direct kernels' item lists follow a tree build (which re-sorts the
    triangles) and positions-only uploads: the direct sums then match a fresh
    context on the same positions."""
    import torch

    V, F = meshgen.sh_deformed_sphere(5, 12, 0.05, 7)
    V2 = V + 0.03 * np.sin(3.0 * V[:, [1, 2, 0]])  # smooth, changes the Morton order
    V3 = V2 + 0.01 * np.cos(2.0 * V2[:, [2, 0, 1]])
    tp.tp_mesh_upload(ctx, V, F)
    tp.tp_tree_build(ctx, 16, 30)
    tp.tp_mesh_upload(ctx, V2, None, flags=tp._tp.TP_POSITIONS_ONLY)
    tp.tp_tree_build(ctx, 16, 30)
    g2 = np.zeros_like(V2)
    e2 = tp.tp_gradient(ctx, g2)
    e2e = tp.tp_energy(ctx)
    tp.tp_mesh_upload(ctx, V3, None, flags=tp._tp.TP_POSITIONS_ONLY)
    g3 = np.zeros_like(V3)
    e3 = tp.tp_gradient(ctx, g3)
    c2 = tp.tp_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        # same positions and the same Morton order (computed from V2 in both): equal up to summation order
        tp.tp_mesh_upload(c2, V2, F)
        gf = np.zeros_like(V2)
        ef = tp.tp_gradient(c2, gf)
        assert abs(e2 - ef) <= 1e-12 * ef and abs(e2e - ef) <= 1e-6 * ef
        assert rel(g2, gf) <= 1e-12, rel(g2, gf)
        # V3 in the order of V2 against a fresh order of V3: both within the direct-form bars of the exact sums
        tp.tp_mesh_upload(c2, V3, F)
        gf = np.zeros_like(V3)
        ef = tp.tp_gradient(c2, gf)
        assert abs(e3 - ef) <= 2 * E_TOL * ef, (e3, ef)
        assert rel(g3, gf) <= 2 * G_TOL, rel(g3, gf)
    finally:
        tp.tp_destroy(c2)


def test_bh_and_learned_after_rebuilds_match_fresh_context(tp, ctx):
    """Node records and network features are written only for nodes the
    traversal can reach (the root and children of nodes above the leaf
    size); the other nodes keep what an earlier build left.  After builds
    with smaller and larger leaf sizes on other positions, the Barnes-Hut and
    learned results equal those of a fresh context (up to summation order)."""
    import torch

    model = str(ROOT / "paper_2509_22110_gb300" / "far_model_l7.bin")
    V, F = meshgen.sh_deformed_sphere(5, 12, 0.05, 9)
    V2 = V + 0.03 * np.sin(3.0 * V[:, [1, 2, 0]])  # smooth, changes the Morton order
    tp.tp_far_model_load(ctx, model)
    tp.tp_mesh_upload(ctx, V, F)
    g = np.zeros_like(V)
    for leaf in (4, 32):
        tp.tp_tree_build(ctx, leaf, 30)
        tp.tp_gradient(ctx, g, tp.tp_params_default(mode=tp.TP_BH, theta=0.5))
        tp.tp_gradient(ctx, g, tp.tp_params_default(mode=tp.TP_LEARNED, theta=0.5))
    tp.tp_mesh_upload(ctx, V2, None, flags=tp._tp.TP_POSITIONS_ONLY)
    tp.tp_tree_build(ctx, 16, 30)
    got = {}
    for mode in (tp.TP_BH, tp.TP_LEARNED):
        gm = np.zeros_like(V2)
        got[mode] = (tp.tp_gradient(ctx, gm, tp.tp_params_default(mode=mode, theta=0.5)), gm)
    c2 = tp.tp_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        tp.tp_far_model_load(c2, model)
        tp.tp_mesh_upload(c2, V2, F)
        tp.tp_tree_build(c2, 16, 30)
        for mode, tol in ((tp.TP_BH, 1e-12), (tp.TP_LEARNED, 1e-7)):
            gf = np.zeros_like(V2)
            ef = tp.tp_gradient(c2, gf, tp.tp_params_default(mode=mode, theta=0.5))
            e, gm = got[mode]
            assert abs(e - ef) <= tol * abs(ef), (mode, e, ef)
            assert rel(gm, gf) <= tol, (mode, rel(gm, gf))
    finally:
        tp.tp_destroy(c2)


@pytest.mark.parametrize("nt_keep", [2, 17, 33, 777, 2000])
def test_bh_ragged_sizes(tp, ctx, oracle_mod, nt_keep):
    """Open sub-meshes of sizes that fill no leaf, run or list evenly (two
    triangles that share a vertex give an empty sum), against the oracle's
    Barnes-Hut sums at theta = 0.5."""
    V, F = meshgen.perturbed_sphere(4, 0.01, 3)
    F = np.ascontiguousarray(F[:nt_keep])
    Eo, go, info = oracle_mod.bh_gradient(V, F, 0.5)
    tp.tp_mesh_upload(ctx, V, F)
    tp.tp_tree_build(ctx, 16, 30)
    grad = np.zeros_like(V)
    e = tp.tp_gradient(ctx, grad, tp.tp_params_default(mode=tp.TP_BH, theta=0.5))
    st = tp.tp_get_stats(ctx)
    assert st["far_terms"] == info["far_terms"] and st["pairs_exact"] == info["near_pairs"]
    # the learned form on the same tree: empty or tiny far lists, windows and runs
    tp.tp_far_model_load(ctx, str(ROOT / "paper_2509_22110_gb300" / "far_model_l7.bin"))
    gl = np.zeros_like(V)
    el = tp.tp_gradient(ctx, gl, tp.tp_params_default(mode=tp.TP_LEARNED, theta=0.5))
    stl = tp.tp_get_stats(ctx)
    assert stl["far_terms"] == info["far_terms"] and stl["learned_terms"] <= stl["far_terms"]
    assert np.isfinite(el) and np.all(np.isfinite(gl))
    if info["far_terms"] == 0:
        assert el == e and np.array_equal(gl, grad)
    if Eo == 0.0:
        assert e == 0.0 and not grad.any()
        return
    assert abs(e - Eo) <= E_TOL * Eo, (e, Eo)
    assert rel(grad, go) <= G_TOL, rel(grad, go)


def test_bh_theta_zero_equals_direct(tp, ctx):
    V, F = meshgen.workload("dish_l5")
    tp.tp_mesh_upload(ctx, V, F)
    gd = np.zeros_like(V)
    ed = tp.tp_gradient(ctx, gd, tp.tp_params_default())
    tp.tp_tree_build(ctx, 16, 30)
    gb = np.zeros_like(V)
    eb = tp.tp_gradient(ctx, gb, tp.tp_params_default(mode=tp.TP_BH, theta=0.0))
    assert tp.tp_get_stats(ctx)["far_terms"] == 0
    assert abs(eb - ed) <= 1e-6 * ed
    assert rel(gb, gd) <= 1e-5


def test_bh_accuracy_improves_with_theta(tp, ctx):
    V, F = meshgen.sh_deformed_sphere(6, 12, 0.05, 2)
    tp.tp_mesh_upload(ctx, V, F)
    gd = np.zeros_like(V)
    ed = tp.tp_gradient(ctx, gd, tp.tp_params_default(prec=tp.TP_F64))
    tp.tp_tree_build(ctx, 16, 30)
    errs = []
    thetas = (1.0, 0.5, 0.25, 0.125, 0.0625)
    for th in thetas:
        gb = np.zeros_like(V)
        eb = tp.tp_gradient(ctx, gb, tp.tp_params_default(mode=tp.TP_BH, theta=th))
        errs.append((abs(eb - ed) / ed, rel(gb, gd)))
    assert all(errs[i][0] > errs[i + 1][0] and errs[i][1] > errs[i + 1][1] for i in range(len(thetas) - 1)), errs
    # the monopole error falls about as theta^2; the stated opening angle for <= 1e-3 is 0.0625
    assert errs[-1][0] <= 1e-3 and errs[-1][1] <= 1e-3, errs


def test_bh_full_size_parity(tp, ctx, oracle_mod):
    """Level-7 SH sphere (327,680 triangles), theta = 0.5: full oracle BH parity."""
    V, F = meshgen.workload("sh_l7")
    Eo, go, info = oracle_mod.bh_gradient(V, F, 0.5)
    tp.tp_mesh_upload(ctx, V, F)
    tp.tp_tree_build(ctx, 16, 30)
    grad = np.zeros_like(V)
    e = tp.tp_gradient(ctx, grad, tp.tp_params_default(mode=tp.TP_BH, theta=0.5))
    st = tp.tp_get_stats(ctx)
    assert st["far_terms"] == info["far_terms"]
    assert abs(e - Eo) <= E_TOL * Eo
    assert rel(grad, go) <= G_TOL
