"""More pins of the FP64 oracle against what the paper and the mathematics fix
(no GPU):

* the staggered gather of Eq. (19) in 2D and 3D: the W_2 weights reproduce
  linear functions exactly, so a field linear in x, y, z sampled at each
  component's own Yee position must gather to that linear function at the
  particle (a component taken at the wrong (half-)node is off by half a cell
  times its slope); plus a brute-force evaluation of Eq. (19) with weights
  integrated from the hat shape S_2 directly;
* the quantum parameter chi of Sec. IV in its closed forms (pure B,
  longitudinal E, head-on and co-propagating plane waves, photons) and the
  Schwinger field the paper prints;
* the Method I Monte Carlo (optical-depth form): with a constant rate the
  events of a particle form a Bernoulli process with p = 1 - exp(-W dt) per
  step; in the classical limit W is the textbook photon number rate
  5 alpha omega_B / (2 sqrt3), at chi ~ 1 the rate of Eq. (23);
* energy bookkeeping of laser runs: field + kinetic + absorbed energy minus
  the initial energy equals the laser energy that entered through x-min, up
  to the scheme's second-order discretisation error (checked by halving the
  cell size: the error falls four-fold and extrapolates to zero).
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import oracle as O
from paper_2104_00642_gb300 import workloads as W

ALPHA = 1.0 / 137.035999084

# standard Yee cell (Fig. 1 of the paper is missing from the text): the
# offset of every component's sample point from node (i, j, k), in cells
YEE = {O.EX: (0.5, 0.0, 0.0), O.EY: (0.0, 0.5, 0.0), O.EZ: (0.0, 0.0, 0.5),
       O.BX: (0.0, 0.5, 0.5), O.BY: (0.5, 0.0, 0.5), O.BZ: (0.5, 0.5, 0.0)}


def _hat_cell_integral(xi):
    """Integral of the hat S_2(t) = max(0, 1 - |t|) over [xi - 1/2, xi + 1/2]."""
    def prim(t):  # antiderivative of the hat from -1, constant outside its support
        t = min(max(t, -1.0), 1.0)
        return (t + 1.0) ** 2 / 2.0 if t < 0 else 0.5 + t - t * t / 2.0
    return prim(xi + 0.5) - prim(xi - 0.5)


def _yee_linear(o, dim, rng):
    n, dx = o.n, o.dx
    coef = {}
    for c in range(6):
        a0 = rng.uniform(-1, 1)
        s = rng.uniform(0.5, 2.0, 3) * rng.choice([-1, 1], 3)
        coef[c] = (a0, s)
        zz, yy, xx = np.meshgrid(*[np.arange(m) for m in o.box()], indexing="ij")
        pos = [(xx + YEE[c][0]) * dx[0], (yy + YEE[c][1]) * dx[1], (zz + YEE[c][2]) * dx[2]]
        f = a0 + sum(s[d] * pos[d] for d in range(dim))
        o.set_field(c, f)
    return coef


@pytest.mark.parametrize("dim", [2, 3])
def test_staggered_gather_reproduces_linear_fields(dim):
    """Eq. (19) with the Yee placement: every component of a field linear in
    x, y, z (sampled at that component's own staggered position) gathers to
    the linear function at the particle, to round-off, anywhere in the cell."""
    rng = np.random.default_rng(40 + dim)
    n = (12, 10, 9)[:dim]
    dx = (0.3, 0.25, 0.2)[:dim]
    o = O.OracleSim(dim, n, dx, 0.01)
    coef = _yee_linear(o, dim, rng)
    for _ in range(200):
        x = [rng.uniform(2.0 * dx[d], (n[d] - 2.0) * dx[d]) for d in range(dim)]
        got = o.gather(x)
        for c in range(6):
            a0, s = coef[c]
            want = a0 + sum(s[d] * x[d] for d in range(dim))
            assert abs(got[c] - want) <= 1e-12 * (1.0 + abs(want)), (c, x, got[c], want)


def test_gather_brute_force_three_particles_3d():
    """Eq. (19) by brute force for three particles in a random 3D field: every
    node within reach, its weight the product over axes of the hat S_2
    integrated over the node's cell (no closed-form W_2, no nearest node)."""
    rng = np.random.default_rng(7)
    n, dx = (8, 9, 10), (0.4, 0.3, 0.5)
    o = O.OracleSim(3, n, dx, 0.01)
    F = {}
    for c in range(6):
        F[c] = rng.uniform(-1.0, 1.0, o.box())
        o.set_field(c, F[c])
    for x in ([1.234, 0.777, 2.903], [0.05, 2.68, 4.99], [3.199, 1.5, 0.251]):
        got = o.gather(x)
        for c in range(6):
            X = [x[d] / dx[d] - YEE[c][d] for d in range(3)]  # position in the component's own index space
            acc = 0.0
            for k in range(int(math.floor(X[2])) - 2, int(math.floor(X[2])) + 3):
                wz = _hat_cell_integral(k - X[2])
                for j in range(int(math.floor(X[1])) - 2, int(math.floor(X[1])) + 3):
                    wy = _hat_cell_integral(j - X[1])
                    for i in range(int(math.floor(X[0])) - 2, int(math.floor(X[0])) + 3):
                        w = _hat_cell_integral(i - X[0]) * wy * wz
                        if w != 0.0:
                            acc += w * F[c][k % n[2], j % n[1], i % n[0]]
            assert abs(got[c] - acc) <= 1e-13, (c, x, got[c], acc)


def test_hat_cell_integral_is_w2():
    """the test's own weights: the three nonzero cell integrals of the hat sum
    to one and equal (1/8, 3/4, 1/8) at a node"""
    assert [_hat_cell_integral(v) for v in (-1.0, 0.0, 1.0)] == [0.125, 0.75, 0.125]
    for d in np.linspace(-0.5, 0.49, 11):
        assert abs(sum(_hat_cell_integral(m - d) for m in (-2, -1, 0, 1, 2)) - 1.0) < 1e-15


# ----------------------------------------------------------------------
# chi (Sec. IV)
# ----------------------------------------------------------------------

def _qed_oracle(lambda_r_m=1e-6):
    o = O.OracleSim(1, (8,), (1.0,), 0.1)
    o.add_species(-1.0, 1.0, 1e-12, 8, kind=0, qed=1)
    o.add_species(0.0, 0.0, 1e-12, 8, kind=1, qed=0)
    o.set_qed(photon_sp=1, lambda_r_m=lambda_r_m)
    return o


def test_schwinger_field_matches_the_printed_value():
    """E_s in units of m c omega_r / e for lambda_r = 1 um, times that unit in
    V/cm, is the critical field the paper prints, 1.3e16 V/cm (Sec. IV)."""
    o = _qed_oracle()
    me, c, e = 9.1093837015e-31, 2.99792458e8, 1.602176634e-19
    omega = 2.0 * math.pi * c / 1e-6
    E_unit_V_per_cm = me * c * omega / e / 100.0
    assert round(o.Es * E_unit_V_per_cm, -15) == 1.3e16  # two significant digits, as printed


def test_chi_closed_forms():
    o = _qed_oracle()
    Es = o.Es
    u = 1999.0
    g = math.sqrt(1.0 + u * u)
    B, E = 37.0, 11.0
    # pure B perpendicular to u: chi = |u| B / E_s; parallel to u: 0
    assert o.chi(g, [0, u, 0], [0, 0, 0, 0, 0, B]) == pytest.approx(u * B / Es, rel=1e-14)
    assert o.chi(g, [0, 0, u], [0, 0, 0, 0, 0, B]) == 0.0
    # longitudinal E: Lorentz invariance leaves chi = E/E_s whatever |u|
    assert o.chi(g, [u, 0, 0], [E, 0, 0, 0, 0, 0]) == pytest.approx(E / Es, rel=1e-9)
    assert o.chi(1.0, [0, 0, 0], [0, E, 0, 0, 0, 0]) == pytest.approx(E / Es, rel=1e-14)
    # plane wave moving along +x (E_y = B_z): head-on electron (u along -x)
    # sees (gamma + |u|) E, a co-moving one (gamma - |u|) E
    wave = [0, E, 0, 0, 0, E]
    assert o.chi(g, [-u, 0, 0], wave) == pytest.approx((g + u) * E / Es, rel=1e-14)
    assert o.chi(g, [u, 0, 0], wave) == pytest.approx((g - u) * E / Es, rel=1e-6)
    # photons (|k| in place of gamma): across B, and along the wave (chi = 0)
    k = 5000.0
    assert o.chi(k, [k, 0, 0], [0, 0, 0, 0, B, 0]) == pytest.approx(k * B / Es, rel=1e-14)
    assert o.chi(k, [k, 0, 0], wave) <= 1e-12 * k * E / Es


# ----------------------------------------------------------------------
# Method I event statistics (Sec. IV)
# ----------------------------------------------------------------------

def _gyrating_electrons(n_e, gamma, chi, dt, dx, seed):
    """n_e electrons of energy gamma with u in the x-y plane, in a uniform
    B_z giving them quantum parameter chi (1D periodic grid, tiny weight so
    self-fields vanish); photons are collected, pair creation is off"""
    o = O.OracleSim(1, (16,), (dx,), dt)
    o.add_species(-1.0, 1.0, 1e-14, n_e, kind=0, qed=1)
    o.add_species(0.0, 0.0, 1e-14, 64 * n_e, kind=1, qed=0)
    o.set_qed(photon_sp=1, lambda_r_m=1e-6, photon_emin=0.0, seed=seed)
    u = math.sqrt(gamma * gamma - 1.0)
    B = chi * o.Es / u
    o.set_field(O.BZ, np.full(o.box(), B))
    rng = np.random.default_rng(seed)
    x = (np.arange(n_e) + 0.5) * (16.0 * dx / n_e)
    ang = rng.uniform(0.0, 2.0 * math.pi, n_e)
    z = np.zeros(n_e)
    o.load(0, x, None, None, u * np.cos(ang), u * np.sin(ang), z)
    return o, B, u


def _events_per_step(o, steps):
    """per step, which electrons emitted: a child is born at its parent's
    x^{n+1} before either moves again, so new photons are matched to
    electrons by position"""
    ev = []
    n_ph = 0
    for _ in range(steps):
        o.step(1)
        xe = o.particles(0)["x"]
        ph = o.particles(1)["x"]
        new = ph[n_ph:]
        n_ph = len(ph)
        hit = np.zeros(len(xe), dtype=int)
        for xp in new:
            i = np.nonzero(xe == xp)[0]
            assert len(i) == 1
            hit[i[0]] += 1
        ev.append(hit)
    return np.array(ev)  # steps x electrons, entries 0/1


def test_method_one_events_are_bernoulli_at_the_classical_rate():
    """chi = 1e-4 (classical limit): the rate is the synchrotron photon number
    rate W = 5 alpha B v / (2 sqrt3) (units of Eq. (8), omega_B = B),
    independent of E_s and gamma; recoil is ~1e-4 of gamma, so W stays
    constant and every electron's events are a Bernoulli process with
    p = 1 - exp(-W dt): the total is Binomial(N T, p), the per-step counts
    are Binomial(N, p), the per-electron counts Binomial(T, p)."""
    n_e, T, gamma, chi = 64, 16, 10.0, 1e-4
    dt, dx = 8.2, 10.0
    o, B, u = _gyrating_electrons(n_e, gamma, chi, dt, dx, seed=0xC1A551C)
    W_cl = 5.0 * ALPHA * B * (u / gamma) / (2.0 * math.sqrt(3.0))
    p = 1.0 - math.exp(-W_cl * dt)
    ev = _events_per_step(o, T)
    assert ev.max() <= 1
    N = n_e * T
    tot = ev.sum()
    assert abs(tot - N * p) <= 4.0 * math.sqrt(N * p * (1 - p)), (tot, N * p)
    # dispersion of the per-electron counts (mean T p, variance T p (1 - p))
    per = ev.sum(axis=0)
    stat = np.sum((per - T * p) ** 2) / (T * p * (1 - p))
    assert n_e - 5.0 * math.sqrt(2 * n_e) < stat < n_e + 5.0 * math.sqrt(2 * n_e), stat
    # per-step counts: same mean and variance across steps
    st = ev.sum(axis=1)
    stat2 = np.sum((st - n_e * p) ** 2) / (n_e * p * (1 - p))
    assert stat2 < T + 5.0 * math.sqrt(2 * T), stat2


def _G_rad_scipy(chi):
    """G(chi) = Int_0^1 F(u, chi) du of Eq. (23) with scipy's K_nu"""
    def F(u):
        y = 2.0 * u / (3.0 * chi * (1.0 - u))
        ik = integrate.quad(lambda t: special.kv(1.0 / 3.0, t), y, np.inf, limit=200)[0]
        return ((1.0 - u) + 1.0 / (1.0 - u)) * special.kv(2.0 / 3.0, y) - ik
    # substitute u = s^3 (the u^(-2/3) behaviour at small u)
    return integrate.quad(lambda s: 3.0 * s * s * F(s ** 3), 0.0, 1.0, limit=200, epsrel=1e-10)[0]


@pytest.mark.parametrize("chi", [1.0, 5.0])
def test_method_one_first_events_follow_the_quantum_rate(chi):
    """chi ~ 1: the first event of each electron comes at a geometric step
    with p = 1 - exp(-W dt), W = alpha E_s G(chi) / (sqrt3 pi gamma) from
    Eq. (23) (G by scipy quadrature); the number of electrons that have
    emitted by step T is Binomial(N, 1 - (1 - p)^T)."""
    n_e, T, gamma = 96, 6, 1000.0
    dt, dx = 0.02, 1.0
    o, B, u = _gyrating_electrons(n_e, gamma, chi, dt, dx, seed=0xF1857 + int(chi))
    W = ALPHA * o.Es * _G_rad_scipy(chi) / (math.sqrt(3.0) * math.pi * gamma)
    p = 1.0 - math.exp(-W * dt)
    ev = _events_per_step(o, T)
    first = ev.cumsum(axis=0) > 0
    for t in range(T):
        q = 1.0 - (1.0 - p) ** (t + 1)
        k = first[t].sum()
        assert abs(k - n_e * q) <= 4.0 * math.sqrt(n_e * q * (1.0 - q)) + 1.0, (t, k, n_e * q)


# ----------------------------------------------------------------------
# energy bookkeeping of laser runs (Secs. II.B, III(a))
# ----------------------------------------------------------------------

def _laser_foil_energy_error(dim, cells_per_lambda, pol):
    """A laser (a0 = 10, 5 fs intensity FWHM, uniform across the periodic
    transverse axes) enters through x-min and hits a 1-lambda foil of 5 n_c
    (electrons and protons, 1 keV).  At a time when the whole pulse has
    entered and no reflected light has come back to x-min, field + kinetic +
    absorbed energy minus the initial energy, over the energy the laser
    carried in (a0^2/2 per unit area and time for linear, a0^2 for circular
    polarisation, integrated over the Gaussian intensity envelope), minus 1."""
    lam = 2.0 * math.pi
    dx = lam / cells_per_lambda
    dt = 0.95 * dx / math.sqrt(dim)
    fwhm = 5e-15 * 2.0 * math.pi * 2.99792458e8 / 1e-6
    tp = 3.0 * fwhm
    t_end = tp + 3.2 * fwhm
    f0 = 6 * cells_per_lambda
    f1 = f0 + cells_per_lambda
    nx = f1 + int(round(0.3 * t_end / dx)) + 8
    nt = 4
    a0, n0, ppc = 10.0, 5.0, 4
    o = O.OracleSim(dim, [nx, nt, nt][:dim], [dx] * dim, dt, bc=[O.ABSORB] + [O.PERIODIC] * (dim - 1))
    rng = np.random.Generator(np.random.Philox(7))
    fw = f1 - f0
    ncell = fw * nt ** (dim - 1)
    N = ncell * ppc
    ci = np.repeat(np.arange(ncell), ppc)
    cx, rest = f0 + ci % fw, ci // fw
    for q, m in ((-1.0, 1.0), (1.0, W.M_PROTON)):
        i = o.add_species(q, m, n0 / ppc, N)
        x = (cx + rng.random(N)) * dx
        y = ((rest % nt) + rng.random(N)) * dx if dim >= 2 else None
        z = ((rest // nt) + rng.random(N)) * dx if dim >= 3 else None
        o.load(i, x, y, z, *W.maxwell_juttner_u(rng, N, (1.0 / W.MEC2_KEV) / m))
    o.set_laser(a0, 1e7, fwhm, tp, f0 * dx, 0.0, 0.0, pol)

    def total():
        d = o.diagnostics()
        return d["U_E"] + d["U_B"] + sum(d["U_kin"]) + d["E_absorbed"]

    area = (nt * dx) ** (dim - 1)
    U_in = a0 * a0 * (1.0 if pol else 0.5) * fwhm * math.sqrt(math.pi / (4.0 * math.log(2.0))) * area
    e0 = total()
    o.step(int(t_end / dt))
    return (total() - e0) / U_in - 1.0


@pytest.mark.parametrize("dim,res,pol,tol", [(1, (32, 64), 0, 1e-3), (2, (32, 64), 0, 1.5e-3),
                                             (3, (16, 32), 1, 6e-3)])
def test_laser_energy_bookkeeping_converges_to_the_injected_energy(dim, res, pol, tol):
    """The error is the scheme's O(dx^2) discretisation error of the injected
    wave: at the finer resolution within tol, four times smaller than at the
    coarser one, and its Richardson extrapolation (4 e_fine - e_coarse)/3
    within 1e-4 of exact bookkeeping."""
    e_c = _laser_foil_energy_error(dim, res[0], pol)
    e_f = _laser_foil_energy_error(dim, res[1], pol)
    assert abs(e_f) <= tol, (e_c, e_f)
    assert 3.5 <= e_c / e_f <= 4.5, (e_c, e_f)
    assert abs((4.0 * e_f - e_c) / 3.0) <= 1e-4, (e_c, e_f)
