"""The diagnostics log (paper_2104_00642_gb300.diaglog) against a fake
simulation that counts its steps: rows every `every` steps, the last call
shorter, values written at full FP64 precision.  No GPU."""
import csv

import pytest

from paper_2104_00642_gb300 import diaglog


class FakeSim:
    def __init__(self, nsp=2):
        self.step, self.nsp, self.calls = 0, nsp, []

    def pic_step(self, n):
        self.calls.append(n)
        self.step += n

    def pic_diagnostics(self):
        s = self.step
        return {"step": s, "t": 0.1 * s, "U_E": 1.0 / 3.0 + s, "U_B": 2.0 * s, "U_kin": [s + 0.5] * self.nsp,
                "n_alive": [100 + s] * self.nsp, "E_absorbed": 1e-300 * s, "E_photon_lost": 0.0,
                "charge": -1.0, "gauss_max": 1e-16}


def test_rows_every_k_steps(tmp_path):
    sim = FakeSim()
    path = tmp_path / "diag.csv"
    out = diaglog.run_logged(sim, 10, 4, str(path), names=["electron", "ion"])
    assert sim.calls == [4, 4, 2]
    rows = list(csv.reader(open(path)))
    assert rows[0][:4] == ["step", "t", "U_E", "U_B"] and "U_kin_electron" in rows[0] and "n_ion" in rows[0]
    assert [int(r[0]) for r in rows[1:]] == [0, 4, 8, 10]
    assert float(rows[2][2]) == 1.0 / 3.0 + 4  # full precision
    assert float(rows[4][rows[0].index("E_absorbed")]) == 1e-300 * 10
    assert len(out) == 4


def test_bad_arguments():
    with pytest.raises(ValueError):
        diaglog.run_logged(FakeSim(), 5, 0, "unused.csv")
