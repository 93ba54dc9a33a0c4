"""The thinned pair sampler of the FP32 + surrogate form (Lewis-Shedler
thinning of the Sec. IV pair process) samples the same process as Method I's
optical depth, on the oracle's rate of Eq. (24).  No GPU.

A photon crosses a Gaussian pulse: chi_n = chi0 exp(-((n - n0)/s)^2) over
the steps n, the per-step decrement of Method I is w_n = c G_pair(chi_n)
(c: the prefactor of the rate over k, times dt), the envelope's is
a_n = c G_env(chi_n) >= w_n (the analytic envelope of csrc/qed.cuh).  In
discrete steps the exact survival probabilities are

  Method I  (tau_0 ~ Exp(1), convert at the first n with sum w >= tau_0):
            S_N = exp(-sum_n w_n)
  thinning  (drain a_n; at tau <= 0 a candidate, accepted with w_n / a_n,
            tau restarted from Exp(1) after every candidate): a step holds a
            candidate with probability 1 - exp(-a_n) whatever came before
            (the residual of an exponential is exponential), so
            S_N = prod_n (1 - (1 - exp(-a_n)) w_n / a_n)

Both samplers are simulated on 200,000 photons and their conversion curves
compared with these closed forms at every tenth step (binomial error, 5
sigma); the two closed forms differ by O(sum a_n w_n) only.  A sampler that
does not restart after a rejected candidate, or accepts with a_n / w_n, or
drains at w_n, fails."""
import math
import os
import re

import numpy as np
import pytest

from oracle import oracle as O

QED_CUH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", "paper_2104_00642_gb300", "csrc", "qed.cuh")
N_PHOTONS = 200_000
STEPS = 400


def _envelope_constant():
    m = re.search(r"constexpr float kPairEnvelope = ([0-9.]+)f;", open(QED_CUH).read())
    assert m, "kPairEnvelope not found"
    return float(m.group(1))


def _pulse(chi0):
    """per-step chi, Method I decrements w and envelope decrements a, scaled
    so that sum w = 1 (about 63 % convert)"""
    n = np.arange(STEPS)
    chi = chi0 * np.exp(-(((n - STEPS / 2) / (STEPS / 6)) ** 2))
    L = O.lib()
    G = np.array([L.or_qed_Gpair(c) if c > 0.03 else 0.0 for c in chi])
    cenv = _envelope_constant()
    Genv = np.where(chi > 0.03, cenv * chi ** (2.0 / 3.0) * np.exp(-8.0 / (3.0 * np.maximum(chi, 1e-30))), 0.0)
    c = 1.0 / G.sum()
    return chi, c * G, c * Genv


def _method1(w, rng):
    tau = rng.exponential(size=N_PHOTONS)
    alive = np.ones(N_PHOTONS, bool)
    conv_step = np.full(N_PHOTONS, -1)
    for n in range(STEPS):
        tau[alive] -= w[n]
        hit = alive & (tau <= 0.0)
        conv_step[hit] = n
        alive &= ~hit
    return conv_step


def _thinned(w, a, rng):
    tau = rng.exponential(size=N_PHOTONS)
    alive = np.ones(N_PHOTONS, bool)
    conv_step = np.full(N_PHOTONS, -1)
    for n in range(STEPS):
        if a[n] == 0.0:
            continue
        tau[alive] -= a[n]
        cand = alive & (tau <= 0.0)
        idx = np.nonzero(cand)[0]
        accept = rng.random(len(idx)) < w[n] / a[n]
        conv_step[idx[accept]] = n
        alive[idx[accept]] = False
        tau[idx] = rng.exponential(size=len(idx))  # restart after every candidate
    return conv_step


def _curve(conv_step):
    done = np.array([np.sum((conv_step >= 0) & (conv_step <= n)) for n in range(STEPS)]) / N_PHOTONS
    return 1.0 - done  # survival after step n


@pytest.mark.parametrize("chi0", [0.08, 1.0, 20.0])
def test_thinned_sampler_samples_the_method1_process(chi0):
    chi, w, a = _pulse(chi0)
    assert np.all(a >= w)  # the envelope bounds the rate (the closed forms hold at any step size)
    s_m1 = np.exp(-np.cumsum(w))
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(a > 0, w / a, 0.0)
    s_th = np.cumprod(1.0 - (1.0 - np.exp(-a)) * r)
    # the two discrete processes differ by O(sum a w) only
    assert np.max(np.abs(np.log(s_th) - np.log(s_m1))) <= np.sum(a * w) + 1e-12
    rng = np.random.default_rng(2104 + int(chi0 * 100))
    got_m1 = _curve(_method1(w, rng))
    got_th = _curve(_thinned(w, a, rng))
    for got, exact in ((got_m1, s_m1), (got_th, s_th)):
        sig = np.sqrt(exact * (1.0 - exact) / N_PHOTONS) + 1e-12
        z = np.abs(got - exact)[::10] / sig[::10]
        assert z.max() < 5.0, z.max()
    # and against each other at the end (the conversion probability, ~63 %)
    sig = math.sqrt(2.0 * s_m1[-1] * (1.0 - s_m1[-1]) / N_PHOTONS)
    assert abs(got_th[-1] - got_m1[-1]) < 5.0 * sig + np.sum(a * w)


def test_a_sampler_without_the_restart_is_caught():
    """the check above sees the plausible mistake: a rejected candidate that
    keeps draining its exhausted depth (no restart) converts at the next
    step with probability w/a again and again -- far too often"""
    chi, w, a = _pulse(1.0)
    rng = np.random.default_rng(7)
    tau = rng.exponential(size=N_PHOTONS)
    alive = np.ones(N_PHOTONS, bool)
    for n in range(STEPS):
        if a[n] == 0.0:
            continue
        tau[alive] -= a[n]
        cand = alive & (tau <= 0.0)
        idx = np.nonzero(cand)[0]
        alive[idx[rng.random(len(idx)) < w[n] / a[n]]] = False
    s_exact = float(np.exp(-np.sum(w)))
    sig = math.sqrt(s_exact * (1.0 - s_exact) / N_PHOTONS)
    assert abs(alive.mean() - s_exact) > 10.0 * sig
