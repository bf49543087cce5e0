"""The tensor-core (tcgen05) path of the learned far field's network (needs a GPU):
one 128 x N x K GEMM through the same shared-memory operand layout, descriptors and
accumulator read-back as the network kernel, against numpy on the BF16 inputs
(products of BF16 values are exact in FP32; only the FP32 summation differs)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tpm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_22110_gb300 import build

    build.build()
    import paper_2509_22110_gb300 as tp

    return tp


def bf16_bits(a):
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint16)


def bits_to_f64(b):
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("K,N", [(16, 16), (32, 64), (64, 64), (64, 16)])
def test_tc_gemm(tpm, K, N):
    rng = np.random.default_rng(K * 100 + N)
    A = bf16_bits(rng.standard_normal((128, K)))
    B = bf16_bits(rng.standard_normal((N, K)))
    D = tpm._tp.tp_debug_tc_gemm(A, B)
    ref = bits_to_f64(A) @ bits_to_f64(B).T
    err = np.max(np.abs(D - ref)) / np.max(np.abs(ref))
    assert err <= 1e-6, err
    # a structured case: one-hot rows pick single columns of B (catches any index permutation)
    A1 = np.zeros((128, K), np.float32)
    A1[np.arange(128), np.arange(128) % K] = 1.0
    D1 = tpm._tp.tp_debug_tc_gemm(bf16_bits(A1), B)
    np.testing.assert_array_equal(D1, bits_to_f64(B)[:, np.arange(128) % K].T.astype(np.float32))
