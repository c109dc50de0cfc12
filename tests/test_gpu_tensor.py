"""The tensor-core building blocks on the GPU: the tcgen05 operand and
accumulator layouts (an exact product of small integers through the C ABI)
and the micro-benchmarks whose rates are the roofline denominators."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_02898_gb300 import mem as m
    m.lib()
    return m


@pytest.mark.parametrize("kind", [1, 2, 3])
@pytest.mark.parametrize("N", [16, 64, 256])
def test_tcgen05_layouts_exact(mem, kind, N):
    """A [128 x 64] and B [N x 64] hold values exact in BF16 (small integers)
    or TF32 (quarters up to 16); every partial sum is an integer multiple of
    1/16 below 2^20, so D = A B^T is exact in FP32 and must match bit for bit.
    A wrong descriptor offset, core-matrix order or accumulator lane would
    move entries and fail here."""
    rng = np.random.default_rng(7 + kind + N)
    # kind 3: TF32 operands through TMA tensor loads with the 128-byte swizzle
    if kind == 1:
        A = rng.integers(-8, 9, (128, 64)).astype(np.float32)
        B = rng.integers(-8, 9, (N, 64)).astype(np.float32)
    else:
        A = (rng.integers(-64, 65, (128, 64)) / 4.0).astype(np.float32)
        B = (rng.integers(-64, 65, (N, 64)) / 4.0).astype(np.float32)
    D = mem.tc_selftest(kind, A, B)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    assert np.array_equal(D.astype(np.float64), ref), np.argwhere(D != ref)[:5]


def test_micro_benchmarks_run(mem):
    """Each micro-benchmark completes and reports a rate of the right order
    for a GB300 (these are not the published figures, only sanity bounds)."""
    rates = {}
    for kind, iters in ((0, 2000), (1, 2000), (2, 2000), (3, 2000)):
        sec, work = mem.bench_peak(kind, iters)
        assert sec > 0 and work > 0
        rates[kind] = work / sec
    assert 10e12 < rates[0] < 200e12, rates      # FP32 FMA flop/s
    assert 1e12 < rates[1] < 50e12, rates        # exp2 / s
    assert 300e12 < rates[2] < 4e15, rates       # BF16 tensor flop/s
    assert 100e12 < rates[3] < 2e15, rates       # TF32 tensor flop/s
    print("peaks: fp32 %.1f TFLOP/s, ex2 %.2f T/s, bf16 %.0f TFLOP/s, tf32 %.0f TFLOP/s"
          % (rates[0] / 1e12, rates[1] / 1e12, rates[2] / 1e12, rates[3] / 1e12))
