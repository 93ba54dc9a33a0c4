"""pic_measure_ceilings: the throughput ceilings of the push kernels'
instruction mixes come out in the expected order of magnitude (FP32 FMA a
few tens of TFLOP/s on 152 SMs, FP64 far below it on this GPU, conflict-free
shared atomics faster than 32 lanes on one word) -- the numbers themselves
are recorded with the profiles."""
import pytest

from paper_2104_00642_gb300 import pic

pytestmark = pytest.mark.gpu


def test_ceilings_are_measured():
    c = pic.pic_measure_ceilings()
    print(c)
    assert 1e13 < c["fp32_flops"] < 3e14
    assert 0 < c["fp64_flops"] < 0.5 * c["fp32_flops"]
    assert c["shared_atomics_distinct"] > c["shared_atomics_same_word"] > 0
    assert c["warp_reduce_then_atomic_values"] > 0
