"""Strong-field corners of the push and the in-step error paths, on the GPU
against the oracle:

* Vay's pusher (Sec. II.C's alternative to Eqs. 13-16) when the magnetic
  rotation parameter tau = |q/m| B dt / 2 is 10-30 and the particle is slow:
  the closed-form gamma of the second half kick must not cancel in FP32
  (every push kernel: tiled 2D and 3D, the simple kernel, the QED kernels);
* the FP64 island of the FP32 form above gamma ~ 1e4 (1 + u^2 is computed
  in FP64 there): one step of particles at gamma 1.2e4 - 1e6;
* errors raised inside pic_step: a non-finite field makes particle momenta
  NaN (PIC_ERR_NONFINITE, not a Courant violation); pair creation beyond a
  species' capacity (PIC_ERR_CAPACITY; the excess is not stored).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_00642_gb300 import pic, workloads as W
from tests import qed_setup as Q
from tests.helpers import oracle_from_workload, random_state

pytestmark = pytest.mark.gpu

TOL = {pic.FP32_CELLOFF: 1e-5, pic.FP64_PLAIN: 1e-10}
GRIDS = {1: ((37,), (0.1,)), 2: ((40, 21), (0.1, 0.12)), 3: ((12, 12, 12), (0.1, 0.12, 0.11))}


def _dt(dx, frac=0.9):
    return frac / math.sqrt(sum(1.0 / d ** 2 for d in dx))


def _strong_B(F, dt, rng, tau_lo=10.0, tau_hi=30.0):
    """uniform B of random direction with |q/m| |B| dt / 2 in [tau_lo, tau_hi]
    plus a small random ripple; E of order one"""
    tau = rng.uniform(tau_lo, tau_hi)
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    B = 2.0 * tau / dt
    for k, c in enumerate((pic.BX, pic.BY, pic.BZ)):
        F[c] = B * d[k] * (1.0 + 0.01 * F[c])
    return tau


def _pair(dim, prec, variant, pusher, seed, umax, fields_fn, qed=False, tile=None):
    n, dx = GRIDS[dim]
    dt = _dt(dx)
    w, F = random_state(dim, n, dx, dt, 3, seed, umax=umax)
    rng = np.random.default_rng(seed + 1)
    info = fields_fn(F, dt, rng)
    if qed:
        # the QED push kernels without events: no photon species
        w.species[0].qed = 1
    t = tile if tile is not None else w.tile
    sim = pic.from_workload(w, precision=prec, sort_interval=1 if variant == pic.PUSH_AUTO else 0,
                            push_variant=variant, pusher=pusher, tile=t, load=False)
    if qed:
        sim.pic_set_qed(photon_sp=-1, electron_sp=-1, positron_sp=-1, lambda_r_m=1e-6)
    s = w.species[0]
    sim.pic_load_particles(0, s.x, s.y if dim > 1 else None, s.z if dim > 2 else None, s.ux, s.uy, s.uz)
    o = oracle_from_workload(w, sort_interval=1 if variant == pic.PUSH_AUTO else 0, tile=t)
    o.set_pusher(pusher)
    for c in range(9):
        sim.pic_set_field(c, F[c])
        o.set_field(c, F[c])
    return w, sim, o, info


def _check_one_step(w, sim, o, prec, dim):
    sim.pic_step(1)
    o.step(1)
    tol = TOL[prec]
    pg, po = sim.pic_get_particles(0), o.particles(0)
    umag = np.sqrt(po["ux"] ** 2 + po["uy"] ** 2 + po["uz"] ** 2)
    for k in ("ux", "uy", "uz"):
        err = np.abs(pg[k] - po[k])
        assert np.all(err <= tol * umag + 1e-2 * tol), (k, np.max(err / (umag + 1e-30)))
    for d, k in enumerate(("x", "y", "z")[:dim]):
        L = w.n[d] * w.dx[d]
        dd = np.abs(pg[k] - po[k])
        dd = np.minimum(dd, L - dd)
        assert np.max(dd) <= 10 * tol * w.dx[d] + 1e-12 * L, (k, np.max(dd))


KERNELS = [  # (dim, precision, push variant, tile, QED kernel)
    (2, pic.FP32_CELLOFF, pic.PUSH_AUTO, (16, 16, 1), False),   # tiled 2D
    (3, pic.FP32_CELLOFF, pic.PUSH_AUTO, (4, 4, 4), False),     # tiled 3D
    (1, pic.FP32_CELLOFF, pic.PUSH_SIMPLE, None, False),
    (2, pic.FP32_CELLOFF, pic.PUSH_SIMPLE, None, False),
    (3, pic.FP64_PLAIN, pic.PUSH_SIMPLE, None, False),
    (2, pic.FP32_CELLOFF, pic.PUSH_AUTO, None, True),           # QED push, FP32
    (3, pic.FP64_PLAIN, pic.PUSH_AUTO, None, True),             # QED push, FP64
]


@pytest.mark.parametrize("pusher", [pic.PUSHER_VAY, pic.PUSHER_BORIS])
@pytest.mark.parametrize("dim,prec,variant,tile,qed", KERNELS)
def test_strong_magnetic_field_slow_particles_one_step(dim, prec, variant, tile, qed, pusher):
    """tau = 10-30 with |u| <= 0.5: Vay's sigma = 1 + |u'|^2 - tau^2 is about
    -tau^2, where the textbook form of gamma_new cancels to tau^2 * eps;
    momenta must still be the oracle's within 1e-5 |u| (FP32)."""
    w, sim, o, tau = _pair(dim, prec, variant, pusher, seed=900 + dim, umax=0.5, fields_fn=_strong_B, qed=qed,
                           tile=tile)
    assert tau >= 10.0
    _check_one_step(w, sim, o, prec, dim)


def _moderate(F, dt, rng):
    for c in range(6):
        F[c] = 10.0 * F[c]
    return None


def _ultra_relativistic(w, rng):
    s = w.species[0]
    g = np.exp(rng.uniform(np.log(1.2e4), np.log(1e6), s.n))
    d = rng.normal(size=(3, s.n))
    d /= np.linalg.norm(d, axis=0)
    u = np.sqrt(g * g - 1.0)
    s.ux, s.uy, s.uz = u * d[0], u * d[1], u * d[2]


@pytest.mark.parametrize("dim,prec,variant,tile,qed", KERNELS)
def test_fp64_gamma_island_above_1e4_one_step(dim, prec, variant, tile, qed):
    """gamma 1.2e4 - 1e6 (u^2 > 1e8, where 1 + u^2 loses the 1 in FP32): the
    FP32 form takes 1/gamma in FP64 there; one step matches the oracle."""
    n, dx = GRIDS[dim]
    dt = _dt(dx)
    w, F = random_state(dim, n, dx, dt, 3, 950 + dim, umax=0.5)
    _ultra_relativistic(w, np.random.default_rng(951 + dim))
    _moderate(F, dt, None)
    if qed:
        w.species[0].qed = 1
    t = tile if tile is not None else w.tile
    sim = pic.from_workload(w, precision=prec, sort_interval=1 if variant == pic.PUSH_AUTO else 0,
                            push_variant=variant, tile=t, load=False)
    if qed:
        sim.pic_set_qed(photon_sp=-1, electron_sp=-1, positron_sp=-1, lambda_r_m=1e-6)
    s = w.species[0]
    sim.pic_load_particles(0, s.x, s.y if dim > 1 else None, s.z if dim > 2 else None, s.ux, s.uy, s.uz)
    o = oracle_from_workload(w, sort_interval=1 if variant == pic.PUSH_AUTO else 0, tile=t)
    for c in range(9):
        sim.pic_set_field(c, F[c])
        o.set_field(c, F[c])
    _check_one_step(w, sim, o, prec, dim)
    # the kinetic energy (FP64 diagnostics, gamma - 1 = u^2 / (gamma + 1))
    dg, do = sim.pic_diagnostics(), o.diagnostics()
    assert abs(dg["U_kin"][0] / do["U_kin"][0] - 1.0) <= 10 * TOL[prec]


@pytest.mark.parametrize("prec,variant", [(pic.FP32_CELLOFF, pic.PUSH_AUTO), (pic.FP32_CELLOFF, pic.PUSH_SIMPLE),
                                          (pic.FP64_PLAIN, pic.PUSH_SIMPLE)])
def test_non_finite_field_reports_nonfinite(prec, variant):
    """A NaN written into E through pic_set_field reaches the particles near
    it: pic_step returns PIC_ERR_NONFINITE (the NaN position that follows
    must not be reported as a Courant violation), and the simulation stays
    usable (its next call answers)."""
    n, dx = GRIDS[2]
    w, F = random_state(2, n, dx, _dt(dx), 3, seed=970)
    sim = pic.from_workload(w, precision=prec, sort_interval=1 if variant == pic.PUSH_AUTO else 0,
                            push_variant=variant)
    for c in range(9):
        sim.pic_set_field(c, F[c])
    bad = F[pic.EX].copy()
    bad[0, 10, 20] = np.nan
    sim.pic_set_field(pic.EX, bad)
    with pytest.raises(pic.PicError) as e:
        sim.pic_step(1)
    assert e.value.code == -5, str(e.value)
    assert sim.pic_particle_count(0) == w.species[0].n
    with pytest.raises(pic.PicError) as e2:
        sim.pic_diagnostics()
    assert e2.value.code == -5


@pytest.mark.parametrize("prec", [pic.FP32_CELLOFF, pic.FP64_PLAIN])
def test_pair_creation_beyond_capacity_reports_capacity(prec):
    """Positrons with room for two: the QED set-up of the event tests creates
    more pairs than that within 25 steps; pic_step returns PIC_ERR_CAPACITY,
    no more than the capacity is stored, and a photon whose pair found no room
    stays alive (energy is not lost)."""
    spec = Q.species_spec()
    spec[1] = (spec[1][0], spec[1][1], spec[1][2], 2, spec[1][4], spec[1][5])
    s = pic.pic_create(1, (16,), (1.0,), Q.DT, spec, seed=Q.SEED, precision=prec)
    s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA)
    s.pic_set_field(pic.BZ, np.full(s.box(), Q.B0))
    s.pic_load_particles(0, *Q.electrons())
    e0 = Q.total_energy(s.pic_get_particles(0), s.pic_get_particles(1), s.pic_get_particles(2))
    code = None
    for _ in range(40):
        try:
            s.pic_step(1)
        except pic.PicError as e:
            code = e.code
            break
    assert code == -4
    assert s.pic_particle_count(1) <= 2
    e1 = Q.total_energy(s.pic_get_particles(0), s.pic_get_particles(1), s.pic_get_particles(2))
    assert abs(e1 - e0) <= (1e-9 if prec == pic.FP64_PLAIN else 2e-5) * e0
