"""Write tests/golden/qed_field_sample.json: the FP64 oracle's run of the QED
field sample (paper_2104_00642_gb300.workloads.qed_field_sample; Sec. IV,
Method I with Eqs. (23) and (24)), the reference the GPU forms' errors are
measured against (tests/test_gpu_qed_sample.py, bench.py).

The sample's electrons do not interact (tiny weight, uniform field), so the
oracle runs them in independent chunks in parallel, each chunk's electrons
carrying their identities of the full load (their Philox streams are those
of the full run); the chunks' observables add up.

Run:  python tests/golden/make_qed_field_sample.py  (a few minutes on 8 cores)
"""
import json
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

SEED = 0x5A3D1E          # Philox key of the sample's Monte Carlo
CHUNKS = 64


def run_chunk(args):
    lo, hi = args
    from oracle import oracle as O
    from paper_2104_00642_gb300 import workloads as W
    from tests import qed_setup as Q
    w = W.qed_field_sample()
    o = O.OracleSim(1, (16,), (1.0,), w.dt)
    for s in w.species:
        o.add_species(s.q, s.m, s.w, s.capacity, kind=s.kind, qed=s.qed)
    o.set_qed(seed=SEED, **w.qed)
    o.set_field(O.BZ, np.full(o.box(), w.notes["B0"]))
    e = w.species[0]
    o.load(0, e.x[lo:hi], None, None, e.ux[lo:hi], e.uy[lo:hi], e.uz[lo:hi])
    o.set_ids(0, np.arange(lo, hi, dtype=np.uint64))  # (species 0 << 48) | load index
    hist = []
    for _ in range(w.steps):
        o.step(1)
        hist.append(float(np.sum(np.sqrt(1.0 + sum(o.particles(0)[k][o.particles(0)["alive"] == 1] ** 2
                                                    for k in ("ux", "uy", "uz"))))))
    fin = Q.sample_observables([o.particles(i) for i in range(3)], o.photon_lost())
    return hist, fin


def main():
    from paper_2104_00642_gb300 import workloads as W
    from tests import qed_setup as Q
    w = W.qed_field_sample()
    n = w.species[0].n
    cuts = np.linspace(0, n, CHUNKS + 1).astype(int)
    with mp.get_context("spawn").Pool(min(CHUNKS, os.cpu_count() or 4)) as pool:
        res = pool.map(run_chunk, list(zip(cuts[:-1], cuts[1:])))
    hist = np.sum([r[0] for r in res], axis=0).tolist()
    fin = Q.combine_observables([r[1] for r in res])
    out = {"what": "FP64 oracle run of workloads.qed_field_sample() (Sec. IV Method I, Eqs. 23-24)",
           "seed": SEED, "steps": w.steps, "history": hist, "final": fin}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "qed_field_sample.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, fin["photons"], fin["positrons"])


if __name__ == "__main__":
    main()
