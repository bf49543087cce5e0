"""Failure paths on the GPU, produced without faulting it (needs a GPU).

- A device-side bounded wait that runs out: tp_debug_wait_timeout arms an
  mbarrier for bytes no copy delivers and waits on it with the pair kernels'
  bounded wait and a short limit; the kernel records the timeout and returns,
  the call reports TP_E_TIMEOUT, and the context evaluates correctly after.
- Allocation failures injected on the host (tp_debug_fail_alloc) at every
  allocation of an upload, a tree build and the first Barnes-Hut and energy
  evaluations: each gives TP_E_OOM, leaves no half-resized buffer behind, and
  after a fresh upload the context reproduces the oracle.
"""

import time

import numpy as np
import pytest

from paper_2509_22110_gb300 import meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_22110_gb300 import build

    build.build()
    import paper_2509_22110_gb300 as tpm

    return tpm


@pytest.fixture(scope="module")
def mesh(oracle_mod):
    V, F = meshgen.workload("sphere_l3")
    E = oracle_mod.energy(V, F)
    Eb, _, _ = oracle_mod.bh_gradient(V, F, 0.5)
    return V, F, E, Eb


def new_ctx(tp):
    import torch

    return tp.tp_create(0, torch.cuda.current_stream().cuda_stream)


def test_bounded_wait_runs_out(tp, mesh):
    V, F, E, _ = mesh
    ctx = new_ctx(tp)
    try:
        t0 = time.perf_counter()
        with pytest.raises(tp.TPError) as ei:
            tp._tp.tp_debug_wait_timeout(ctx, 20.0)
        dt = time.perf_counter() - t0
        assert ei.value.status == tp._tp.TP_E_TIMEOUT
        assert dt < 5.0  # the wait gave up on its limit, not on the poll backstop
        # the context (and the error word) are clean for the next call
        tp.tp_mesh_upload(ctx, V, F)
        assert abs(tp.tp_energy(ctx, tp.tp_params_default()) - E) <= 1e-6 * E
        with pytest.raises(tp.TPError) as ei:
            tp._tp.tp_debug_wait_timeout(ctx, 0.0)
        assert ei.value.status == tp._tp.TP_E_ARG
    finally:
        tp.tp_destroy(ctx)


def run_sequence(tp, ctx, V, F):
    """Upload, direct energy + gradient, tree build, Barnes-Hut energy."""
    tp.tp_mesh_upload(ctx, V, F)
    g = np.zeros_like(V)
    e = tp.tp_gradient(ctx, g, tp.tp_params_default())
    tp.tp_tree_build(ctx, 16, 30)
    eb = tp.tp_energy(ctx, tp.tp_params_default(mode=tp.TP_BH, theta=0.5))
    return e, eb


def test_allocation_failure_at_every_point(tp, mesh):
    """Each iteration starts from a fresh context, so that `after` walks through every
    allocation of a cold upload, evaluation, tree build and Barnes-Hut evaluation."""
    V, F, E, Eb = mesh
    failed = 0
    for after in range(400):
        ctx = new_ctx(tp)
        try:
            tp._tp.tp_debug_fail_alloc(ctx, after)
            try:
                run_sequence(tp, ctx, V, F)
                break  # the sequence needs no more than `after` allocations
            except tp.TPError as err:
                assert err.status == tp._tp.TP_E_OOM, err
                failed += 1
            # after the failure the mesh is gone until the next upload
            with pytest.raises(tp.TPError) as ei:
                tp.tp_energy(ctx, tp.tp_params_default())
            assert ei.value.status == tp._tp.TP_E_STATE
            e, eb = run_sequence(tp, ctx, V, F)
            assert abs(e - E) <= 1e-6 * E and abs(eb - Eb) <= 1e-6 * Eb, (after, e, E, eb, Eb)
        finally:
            tp.tp_destroy(ctx)
    assert 10 <= failed < 400, failed  # every allocation point was reached, and the walk ended
