"""The order-4 shape (Sec. II.D, Eq. (18): W_4 on five nodes, Esirkepov on a
7-node window) on the GPU against the oracle, and the self-heating test of
Sec. III(b) (Fig. 6) that compares shape orders, ppc and the two precision
forms."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_00642_gb300 import pic, workloads as W
from tests.helpers import boundary_ambiguous, oracle_from_workload, random_state, window_scale

pytestmark = pytest.mark.gpu

PRECS = [pic.FP32_CELLOFF, pic.FP64_PLAIN]
TOL = {pic.FP32_CELLOFF: 1e-5, pic.FP64_PLAIN: 1e-10}
GRIDS = {1: ((37,), (0.1,)), 2: ((20, 13), (0.1, 0.12)), 3: ((12, 10, 9), (0.1, 0.12, 0.11))}


def _dt(dx, frac=0.9):
    return frac / math.sqrt(sum(1.0 / d ** 2 for d in dx))


def _pair(dim, prec, seed):
    n, dx = GRIDS[dim]
    w, F = random_state(dim, n, dx, _dt(dx), 3, seed, umax=0.5)
    sim = pic.from_workload(w, precision=prec, order=4)
    o = oracle_from_workload(w)
    o.set_order(4)
    for c in range(9):
        sim.pic_set_field(c, F[c])
        o.set_field(c, F[c])
    return w, F, sim, o


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dim", [1, 2, 3])
def test_order4_gather_matches_oracle(dim, prec):
    w, F, sim, o = _pair(dim, prec, 500 + dim)
    got = sim.pic_gather(0)
    s = w.species[0]
    oabs = oracle_from_workload(w)
    oabs.set_order(4)
    for c in range(6):
        oabs.set_field(c, np.abs(F[c]))
    for p in range(s.n):
        x = (s.x[p], s.y[p], s.z[p])[:dim]
        ref, scale = o.gather(x), oabs.gather(x)
        assert np.all(np.abs(got[p] - ref) <= TOL[prec] * scale + 1e-300), (p, got[p], ref)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dim", [1, 2, 3])
def test_order4_one_step_matches_oracle(dim, prec):
    """one step at order 4: momenta, positions, cells and the 7-node
    Esirkepov current against the oracle"""
    w, F, sim, o = _pair(dim, prec, 600 + dim)
    sim.pic_step(1)
    o.step(1)
    tol = TOL[prec]
    pg, po = sim.pic_get_particles(0), o.particles(0)
    keys = ("x", "y", "z")
    for d in range(dim):
        assert np.max(np.abs(pg[keys[d]] - po[keys[d]])) <= 10 * tol * w.dx[d]
    umag = np.sqrt(po["ux"] ** 2 + po["uy"] ** 2 + po["uz"] ** 2)
    for k in ("ux", "uy", "uz"):
        assert np.all(np.abs(pg[k] - po[k]) <= tol * umag + 1e-2 * tol)
    cells, bits = sim.pic_get_cells(0)
    for d in range(dim):
        ref_c = np.floor(po[keys[d]] / w.dx[d]).astype(np.int64)
        got_c = (cells.astype(np.int64) >> sum(bits[:d])) & ((1 << bits[d]) - 1)
        a = boundary_ambiguous(po[keys[d]], w.dx[d])
        assert np.array_equal(got_c[~a], ref_c[~a])
    pre = o.particles(0)
    for c, ax in ((pic.JX, 0), (pic.JY, 1), (pic.JZ, 2)):
        scale = window_scale(pre, w, dim, ax, reach=4)  # 7-node windows one cell wider than order 2's
        assert np.all(np.abs(sim.pic_fields(c) - o.field(c)) <= tol * scale + 1e-30), c


@pytest.mark.parametrize("prec", PRECS)
def test_order4_langmuir_energy_history_and_gauss(prec):
    """the cold Langmuir run at order 4 for 200 steps: field and kinetic
    energy histories within 1e-3 of the run's maximum of the oracle's, and
    the Gauss residual constant after the first step (as at order 2: to
    2e-5 in FP32, 1e-11 in FP64; the background density is 1)"""
    w = W.langmuir_1d(steps=200)
    sim = pic.from_workload(w, precision=prec, order=4)
    o = oracle_from_workload(w)
    o.set_order(4)
    hist_g, hist_o, gauss = [], [], []
    for _ in range(10):
        sim.pic_step(20)
        o.step(20)
        dg, do = sim.pic_diagnostics(), o.diagnostics()
        hist_g.append((dg["U_E"], dg["U_kin"][0]))
        hist_o.append((do["U_E"], do["U_kin"][0]))
        gauss.append(dg["gauss_max"])
    hg, ho = np.array(hist_g), np.array(hist_o)
    scale = ho.max(axis=0)
    assert np.all(np.abs(hg - ho) <= 1e-3 * scale), (np.abs(hg - ho) / scale).max()
    assert max(gauss) - min(gauss) <= (2e-5 if prec == pic.FP32_CELLOFF else 1e-11)


def _heating(order, ppc, prec, steps=3000):
    w = W.self_heating_2d(ppc=ppc, steps=steps)
    sim = pic.from_workload(w, precision=prec, sort_interval=16, order=order)
    d0 = sim.pic_diagnostics()
    e0 = d0["U_E"] + d0["U_B"] + sum(d0["U_kin"])
    sim.pic_step(steps)
    d = sim.pic_diagnostics()
    sim.close()
    return (d["U_E"] + d["U_B"] + sum(d["U_kin"])) / e0 - 1.0


def test_self_heating_falls_with_order_and_ppc():
    """Sec. III(b), Fig. 6 set-up (T = 1 keV, 320 cells per plasma
    wavelength, periodic): the relative energy growth after 3000 steps is
    smaller with the order-4 shape than with order 2 and smaller with more
    particles per cell, and the FP32 cell+offset form heats like the plain
    FP64 form (within the spread of the measurement)"""
    r = {}
    for order in (2, 4):
        for ppc in (4, 16):
            for prec in PRECS:
                r[(order, ppc, prec)] = _heating(order, ppc, prec)
    print({f"order {k[0]} ppc {k[1]} {'fp64' if k[2] else 'fp32'}": v for k, v in r.items()})
    for ppc in (4, 16):
        for prec in PRECS:
            assert r[(4, ppc, prec)] < r[(2, ppc, prec)], r
    for order in (2, 4):
        for prec in PRECS:
            assert r[(order, 16, prec)] < r[(order, 4, prec)], r
    for order in (2, 4):
        for ppc in (4, 16):
            a, b = r[(order, ppc, pic.FP32_CELLOFF)], r[(order, ppc, pic.FP64_PLAIN)]
            assert abs(a - b) <= 0.25 * max(abs(a), abs(b)) + 1e-5, r
