"""Diagnostics log of a run: every `every` steps one CSV row of the FP64
diagnostics the library reduces on the device (pic_diagnostics): step, time,
field energies U_E and U_B, the kinetic energy and live count of each
species, the energy absorbed at the boundaries, the energy of photons below
the kept threshold, the charge and the Gauss residual.  Host logic only: the
simulation steps in the library, this writes what it reports."""
from __future__ import annotations

import csv


def _columns(nsp, names=None):
    names = list(names) if names is not None else [f"sp{i}" for i in range(nsp)]
    return (["step", "t", "U_E", "U_B"] + [f"U_kin_{n}" for n in names] + [f"n_{n}" for n in names]
            + ["E_absorbed", "E_photon_lost", "charge", "gauss_max"])


def _row(d):
    return ([d["step"], repr(float(d["t"])), repr(float(d["U_E"])), repr(float(d["U_B"]))]
            + [repr(float(u)) for u in d["U_kin"]] + [int(n) for n in d["n_alive"]]
            + [repr(float(d["E_absorbed"])), repr(float(d["E_photon_lost"])), repr(float(d["charge"])),
               repr(float(d["gauss_max"]))])


def run_logged(sim, steps: int, every: int, path: str, names=None) -> list[dict]:
    """advance sim by `steps` steps in calls of `every` steps (the last one
    shorter), writing the diagnostics before the first call and after each
    one to the CSV file `path`; returns the diagnostics written"""
    if every < 1 or steps < 0:
        raise ValueError("run_logged: every >= 1 and steps >= 0")
    out = []
    with open(path, "w", newline="") as f:
        w = csv.writer(f)
        d = sim.pic_diagnostics()
        w.writerow(_columns(len(d["U_kin"]), names))
        w.writerow(_row(d))
        out.append(d)
        done = 0
        while done < steps:
            k = min(every, steps - done)
            sim.pic_step(k)
            done += k
            d = sim.pic_diagnostics()
            w.writerow(_row(d))
            out.append(d)
    return out
