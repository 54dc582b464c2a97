"""The tensor-core building blocks (tcgen05.mma with BF16 operands and FP32
accumulation in tensor memory, shared-memory descriptors, mbarrier
completion, TMEM loads) against an exact host product: small integers make
every product and partial sum exact in FP32, so the comparison is bit-exact."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2309_08235_gb300 import build, priest

    build.build()
    return priest


def bf16_bits(x):
    """Round-to-nearest-even FP32 -> BF16 bit patterns (exact for small integers)."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    r = ((u >> 16) & 1) + 0x7FFF
    return ((u + r) >> 16).astype(np.uint16)


@pytest.mark.parametrize("n,k", [(48, 32), (16, 16), (256, 64), (112, 16)])
def test_tensor_core_product_exact(P, n, k):
    rng = np.random.default_rng(n * 100 + k)
    a = rng.integers(-8, 9, (128, k)).astype(np.float32)
    b = rng.integers(-8, 9, (n, k)).astype(np.float32)
    st, d = P.priest_tc_selftest(bf16_bits(a), bf16_bits(b))
    assert st == 0
    np.testing.assert_array_equal(d, a @ b.T)


def test_descriptor_strides_matter(P):
    """Exchanging the descriptor's two byte strides gives a different
    product: the layout check is not vacuous."""
    rng = np.random.default_rng(3)
    a = rng.integers(-8, 9, (128, 32)).astype(np.float32)
    b = rng.integers(-8, 9, (48, 32)).astype(np.float32)
    st, d = P.priest_tc_selftest(bf16_bits(a), bf16_bits(b), swap=1)
    assert st == 0
    assert not np.array_equal(d, a @ b.T)


def test_completion_wait_times_out_and_device_stays_usable(P):
    """The failure path of the tensor-core kernels' bounded waits: with no
    product and no completion signal issued (swap = 2) the kernel's wait for
    the MMA completion runs out, it frees its tensor memory and reports
    PRIEST_ERR_TIMEOUT; the next product on the same device is exact."""
    rng = np.random.default_rng(5)
    a = rng.integers(-8, 9, (128, 16)).astype(np.float32)
    b = rng.integers(-8, 9, (16, 16)).astype(np.float32)
    st, _ = P.priest_tc_selftest(bf16_bits(a), bf16_bits(b), swap=2)
    assert st == P.PRIEST_ERR_TIMEOUT
    st, d = P.priest_tc_selftest(bf16_bits(a), bf16_bits(b))
    assert st == 0
    np.testing.assert_array_equal(d, a @ b.T)
