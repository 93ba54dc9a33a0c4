"""The allocation-free field-energy entry point, pic_field_energy_noalloc.

It serves callers that cannot call cudaMalloc -- for example a plugin inside a
host application that owns every device allocation through its own pool, or a
real-time loop that must not allocate -- and so cannot create a pic_sim.  They
pass their own device arrays and output; the library keeps the reduction's
scratch in a static device array.  This file checks the entry point, called
through the C ABI, against the field energies pic_diagnostics reports, on two
calls in a row that share that scratch.  It is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _sim_with_fields(seed):
    from paper_2104_00642_gb300 import pic
    rng = np.random.default_rng(seed)
    n, dx = (40, 24), (0.1, 0.12)
    sim = pic.pic_create(2, n, dx, 0.05, [(-1.0, 1.0, 0.1, 16)], precision=pic.FP64_PLAIN)
    for c in range(6):
        sim.pic_set_field(c, rng.uniform(-1.0, 1.0, sim.box()))
    return sim, dx[0] * dx[1]


def test_noalloc_field_energy_matches_diagnostics_on_two_calls():
    import torch

    from paper_2104_00642_gb300 import pic
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    results = []
    for call, seed in enumerate((1, 2)):
        sim, dV = _sim_with_fields(seed)
        if call == 1:
            sim.pic_step(3)  # a different field state for the second call
        d = sim.pic_diagnostics()
        dev = [torch.from_numpy(np.ascontiguousarray(sim.pic_fields(c))).to("cuda") for c in range(6)]
        torch.cuda.synchronize()
        pic.pic_field_energy_noalloc([t.data_ptr() for t in dev], dev[0].numel(), dV, out.data_ptr(),
                                     stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - d["U_E"]) <= 1e-10 * d["U_E"], (call, got[0], d["U_E"])
        assert abs(got[1] - d["U_B"]) <= 1e-10 * d["U_B"], (call, got[1], d["U_B"])
        results.append(got.copy())
        sim.close()
    assert not np.allclose(results[0], results[1])


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    from paper_2104_00642_gb300 import pic
    with pytest.raises(pic.PicError) as e:
        pic.pic_field_energy_noalloc([16] * 6, 67_108_864 + 1, 1.0, 16)
    assert "PIC_ERR_ARG" in str(e.value) and "static scratch" in str(e.value)
