"""Pins of the oracle's order-4 shape (Sec. II.D, Eq. (18): S_4 and its cell
integral W_4 on five nodes), as used by the gather (Eq. 19), the Esirkepov
deposit (Eqs. 20-22, the same shape as the gather) and the charge density.
No GPU."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O


def _S4(xi):
    """Eq. (18) as printed: 2/3 - |xi|^2 + |xi|^3/2 inside |xi| <= 1,
    (4/3)(1 - |xi|/2)^3 for 1 < |xi| <= 2"""
    a = abs(xi)
    if a <= 1.0:
        return 2.0 / 3.0 - a * a + 0.5 * a ** 3
    if a <= 2.0:
        return (4.0 / 3.0) * (1.0 - 0.5 * a) ** 3
    return 0.0


def _w4_numeric(delta):
    out = np.zeros(5)
    for k, m in enumerate(range(-2, 3)):
        out[k] = integrate.quad(lambda xi: _S4(xi - delta), m - 0.5, m + 0.5,
                                points=[delta - 2, delta - 1, delta, delta + 1, delta + 2], epsabs=1e-15)[0]
    return out


@pytest.mark.parametrize("delta", np.linspace(-0.5, 0.4999, 17))
def test_w4_is_cell_integral_of_s4(delta):
    assert np.max(np.abs(O.weights4(delta) - _w4_numeric(delta))) < 1e-14


def test_w4_moments_and_node_values():
    """sum 1, first moment 0 (linear functions are reproduced), second moment
    5/12 = 1/3 (S_4) + 1/12 (the cell); at a node (1, 76, 230, 76, 1)/384"""
    m = np.arange(-2, 3, dtype=float)
    for delta in np.linspace(-0.5, 0.49, 41):
        w = O.weights4(delta)
        assert abs(w.sum() - 1.0) < 1e-15
        assert abs(((m - delta) * w).sum()) < 1e-15
        assert abs((((m - delta) ** 2) * w).sum() - 5.0 / 12.0) < 1e-15
        assert np.all(w >= 0.0)
    assert np.max(np.abs(O.weights4(0.0) - np.array([1, 76, 230, 76, 1]) / 384.0)) < 4e-16


YEE = {O.EX: (0.5, 0.0, 0.0), O.EY: (0.0, 0.5, 0.0), O.EZ: (0.0, 0.0, 0.5),
       O.BX: (0.0, 0.5, 0.5), O.BY: (0.5, 0.0, 0.5), O.BZ: (0.5, 0.5, 0.0)}


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_order4_gather_reproduces_linear_fields(dim):
    rng = np.random.default_rng(70 + dim)
    n = (14, 12, 11)[:dim]
    dx = (0.3, 0.25, 0.2)[:dim]
    o = O.OracleSim(dim, n, dx, 0.01)
    o.set_order(4)
    coef = {}
    for c in range(6):
        a0, s = rng.uniform(-1, 1), rng.uniform(0.5, 2.0, 3) * rng.choice([-1, 1], 3)
        coef[c] = (a0, s)
        zz, yy, xx = np.meshgrid(*[np.arange(m) for m in o.box()], indexing="ij")
        pos = [(xx + YEE[c][0]) * o.dx[0], (yy + YEE[c][1]) * o.dx[1], (zz + YEE[c][2]) * o.dx[2]]
        o.set_field(c, a0 + sum(s[d] * pos[d] for d in range(dim)))
    for _ in range(100):
        x = [rng.uniform(3.0 * dx[d], (n[d] - 3.0) * dx[d]) for d in range(dim)]
        got = o.gather(x)
        for c in range(6):
            a0, s = coef[c]
            want = a0 + sum(s[d] * x[d] for d in range(dim))
            assert abs(got[c] - want) <= 1e-12 * (1.0 + abs(want)), (c, x)


def _rho4(x, n, dx, dim):
    """charge shape on nodes from the numerically integrated W_4"""
    rho = np.zeros((n[2] if dim > 2 else 1, n[1] if dim > 1 else 1, n[0]))
    ws, ics = [], []
    for d in range(3):
        if d < dim:
            X = x[d] / dx[d]
            ic = int(math.floor(X + 0.5))
            ws.append(_w4_numeric(X - ic))
            ics.append(ic)
        else:
            ws.append(np.array([0.0, 0.0, 1.0, 0.0, 0.0]))
            ics.append(0)
    for c in range(5):
        for b in range(5):
            for a in range(5):
                w = ws[0][a] * ws[1][b] * ws[2][c]
                if w == 0:
                    continue
                rho[(ics[2] + c - 2) % n[2] if dim > 2 else 0, (ics[1] + b - 2) % n[1] if dim > 1 else 0,
                    (ics[0] + a - 2) % n[0]] += w
    return rho


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_order4_esirkepov_continuity(dim):
    """the order-4 current satisfies the discrete continuity equation with
    the W_4 charge shape, to round-off (Eqs. 20-22 with the gather's shape)"""
    rng = np.random.default_rng(80 + dim)
    n, dx, dt = (12, 11, 10), (0.1, 0.15, 0.12), 0.07
    s = O.OracleSim(dim, n[:dim], dx[:dim], dt)
    s.set_order(4)
    for _ in range(15):
        x0 = [rng.uniform(0, n[d] * dx[d]) if d < dim else 0.0 for d in range(3)]
        x1 = [x0[d] + (rng.uniform(-0.95, 0.95) * dx[d] if d < dim else 0.0) for d in range(3)]
        v, qw = rng.uniform(-0.5, 0.5, 3), -0.37
        Jx, Jy, Jz = s.deposit_one(x0, x1, v, qw)
        res = (_rho4(x1, n, dx, dim) - _rho4(x0, n, dx, dim)) * qw / dt + (Jx - np.roll(Jx, 1, 2)) / dx[0]
        if dim > 1:
            res += (Jy - np.roll(Jy, 1, 1)) / dx[1]
        if dim > 2:
            res += (Jz - np.roll(Jz, 1, 0)) / dx[2]
        assert np.max(np.abs(res)) < 1e-12 * abs(qw) / dt
        nz = np.count_nonzero(np.abs(Jx) > 1e-300, axis=2)
        assert nz.max() >= 5  # the order-4 window is wider than order 2's


def test_order4_inactive_axis_current_is_time_average_of_shape():
    n, dx, dt = (12,), (0.1,), 0.07
    s = O.OracleSim(1, n, dx, dt)
    s.set_order(4)
    x0, x1 = [0.513, 0, 0], [0.574, 0, 0]
    v, qw = np.array([0.3, -0.2, 0.45]), 0.8
    Jx, Jy, Jz = s.deposit_one(x0, x1, v, qw)
    S0 = _rho4(x0, n, dx, 1)[0, 0]
    S1 = _rho4(x1, n, dx, 1)[0, 0]
    avg = 0.5 * (S0 + S1)
    assert np.max(np.abs(Jz[0, 0] - qw * v[2] * avg)) < 1e-15
    assert np.max(np.abs(Jy[0, 0] - qw * v[1] * avg)) < 1e-15


def test_order4_particle_at_rest_deposits_nothing():
    s = O.OracleSim(3, (10, 10, 10), (0.1, 0.1, 0.1), 0.05)
    s.set_order(4)
    Jx, Jy, Jz = s.deposit_one([0.33, 0.41, 0.27], [0.33, 0.41, 0.27], [0, 0, 0], 1.0)
    assert not Jx.any() and not Jy.any() and not Jz.any()


def test_order4_langmuir_keeps_gauss_and_energy():
    """a cold Langmuir run at order 4 (the langmuir_1d workload, 300 steps):
    the Gauss residual stays at its first-step value to round-off and the
    total energy is conserved to 1e-3, as at order 2"""
    from paper_2104_00642_gb300 import workloads as W
    w = W.langmuir_1d(steps=300)
    o = O.OracleSim(1, w.n[:1], w.dx[:1], w.dt, rho_bg=w.rho_bg)
    o.set_order(4)
    s = w.species[0]
    o.add_species(s.q, s.m, s.w, s.capacity)
    o.load(0, s.x, None, None, s.ux, s.uy, s.uz)
    o.step(1)
    d1 = o.diagnostics()
    e1 = d1["U_E"] + d1["U_B"] + sum(d1["U_kin"])
    o.step(299)
    d = o.diagnostics()
    assert abs(d["gauss_max"] - d1["gauss_max"]) <= 1e-11
    e = d["U_E"] + d["U_B"] + sum(d["U_kin"])
    assert abs(e - e1) <= 1e-3 * e1
