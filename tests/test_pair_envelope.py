"""The analytic envelope of the pair rate that the surrogate form's thinned
pair sampler drains the optical depth with (csrc/qed.cuh, pair_envelope_f32:
c chi^(2/3) exp(-8/(3 chi)), up to the top of the network's chi range,
chi = 100; below chi ~ 0.03 it underflows in FP32) lies above the rate of
Eq. (24) -- the oracle's quadrature -- with a margin larger than the
network's rate error (a few per cent) and the tables' (below the network's
range the candidates take the tables' rate), so that the acceptance
W / W_env of a candidate stays below one.  No GPU."""
import math
import os
import re

import numpy as np

from oracle import oracle as O

QED_CUH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", "paper_2104_00642_gb300", "csrc", "qed.cuh")


def _constant():
    m = re.search(r"constexpr float kPairEnvelope = ([0-9.]+)f;", open(QED_CUH).read())
    assert m, "kPairEnvelope not found"
    return float(m.group(1))


def test_envelope_bounds_the_pair_rate_with_margin():
    c = _constant()
    L = O.lib()
    worst = np.inf
    for chi in np.geomspace(0.03, 100.0, 281):
        g = L.or_qed_Gpair(chi)
        env = c * chi ** (2.0 / 3.0) * math.exp(-8.0 / (3.0 * chi))
        worst = min(worst, env / g)
    print("smallest envelope / rate", worst)
    assert worst >= 1.04, worst


def test_envelope_is_not_wasteful_at_large_chi():
    """at the top of the range, where conversions happen, at most 1.2 times
    the rate (the candidates the network evaluates in vain stay few)"""
    c = _constant()
    g = O.lib().or_qed_Gpair(100.0)
    env = c * 100.0 ** (2.0 / 3.0) * math.exp(-8.0 / 300.0)
    assert env / g <= 1.2
