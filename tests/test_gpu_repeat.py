"""Run-to-run repeat check (race detection without a sanitizer): two runs of
the same seeded state take the same decisions bit for bit -- cell indices,
momenta, identities, event outcomes and counts after every step -- through
the tiled pushes, the sort, the QED spawn, the photons appended since the
sort and, with the network, the candidate queue that the photon push fills
in the order of its atomic appends.

The workload is the QED collision with a weightless beam (n_peak = 0: no
current, so the fields are the laser's alone and carry no float-atomic
summation order); the window straddles the collision's peak, where the
Monte Carlo is busiest, with a sort every 4 steps."""
import numpy as np
import pytest

from paper_2104_00642_gb300 import pic, workloads as W

pytestmark = pytest.mark.gpu

STEPS = 12


def _state(sim, nsp):
    out = []
    for i in range(nsp):
        cells, _ = sim.pic_get_cells(i)
        p = sim.pic_get_particles(i)
        ids, tau = sim.pic_get_qed_state(i)
        out.append({"cells": cells, "ux": p["ux"], "uy": p["uy"], "uz": p["uz"], "ids": ids, "tau": tau})
    return out


@pytest.mark.parametrize("mode", ["table", "surrogate"])
def test_two_runs_take_the_same_decisions(mode):
    w = W.qed_collision_2d(n_beam=50_000, n_peak=0.0)
    pre = w.notes["steps_to_collision"] - STEPS // 2
    sims, nets = [], None
    for k in range(2):
        sim = pic.from_workload(w, sort_interval=4, seed=0x5EED)
        if mode == "surrogate":
            if nets is None:
                for p_ in (pic.QED_EMISSION, pic.QED_PAIR):
                    sim.pic_mlp_train(p_, seed=17)
                nets = {p_: sim.pic_mlp_get(p_) for p_ in (pic.QED_EMISSION, pic.QED_PAIR)}
            else:
                for p_, (P, info) in nets.items():
                    sim.pic_mlp_set(p_, P, info["chi_min"], info["chi_max"], info["mu"], info["sd"])
            sim.pic_set_qed(mode=pic.QED_SURROGATE, **w.qed)
        sim.pic_step(pre)
        sims.append(sim)
    nsp = len(w.species)
    events = 0
    for step in range(STEPS):
        for sim in sims:
            sim.pic_step(1)
        a, b = _state(sims[0], nsp), _state(sims[1], nsp)
        for i in range(nsp):
            for key in ("cells", "ux", "uy", "uz", "ids", "tau"):
                assert np.array_equal(a[i][key], b[i][key]), (step, i, key)
        events = len(a[2]["ids"])
    assert events > 1000  # photons were made in the window
    for sim in sims:
        sim.close()
