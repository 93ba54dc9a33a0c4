"""QED Monte Carlo on the GPU (Sec. IV, Eqs. (23), (24)) against the oracle:
tabulated total rates, the inverse-CDF samplers (the single-particle spectra
of Fig. 8 at chi = 0.49, 4.9, 49), and the fused optical-depth Monte Carlo
in the push (event identities, photon energies, energy conservation)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_00642_gb300 import pic
from tests import qed_setup as Q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sim_tables():
    s = pic.pic_create(1, (16,), (1.0,), 0.02, Q.species_spec(cap=16), seed=Q.SEED)
    s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA)
    return s


def test_rate_tables_match_oracle_quadrature(sim_tables):
    L = O.lib()
    chi = np.logspace(-3, 2.5, 23)
    g = sim_tables.pic_qed_eval(pic.QED_EMISSION, chi)
    ref = np.array([L.or_qed_Grad(c) for c in chi])
    assert np.max(np.abs(g / ref - 1.0)) < 2e-5
    chi_p = np.logspace(-1, 2.5, 15)
    gp = sim_tables.pic_qed_eval(pic.QED_PAIR, chi_p)
    refp = np.array([L.or_qed_Gpair(c) for c in chi_p])
    assert np.max(np.abs(gp / refp - 1.0)) < 1e-4


@pytest.mark.parametrize("chi", [0.49, 4.9, 49.0])
@pytest.mark.parametrize("process", [pic.QED_EMISSION, pic.QED_PAIR])
def test_sampler_reproduces_the_spectrum(sim_tables, chi, process):
    """Fig. 8 setup: 1e6 draws of the energy fraction at fixed chi, histogram
    against the spectrum of Eq. (23) / (24) integrated per bin by the oracle
    (chi-square, 24 bins)."""
    L = O.lib()
    rng = np.random.default_rng(12)
    N = 1_000_000
    r = (np.floor(rng.random(N) * 2 ** 24) + 0.5) * 2.0 ** -24
    f = sim_tables.pic_qed_eval(process, np.full(N, chi), r)
    cdf = L.or_qed_cdf_rad if process == pic.QED_EMISSION else L.or_qed_cdf_pair
    if process == pic.QED_EMISSION:
        edges = np.linspace(0.0, 1.0, 25) ** 3
    else:
        edges = np.linspace(0.0, 1.0, 25)
    counts, _ = np.histogram(f, edges)
    c = np.array([cdf(e, chi) for e in edges])
    expect = np.diff(c) * N
    ok = expect > 20
    stat = np.sum((counts[ok] - expect[ok]) ** 2 / expect[ok])
    assert stat < ok.sum() + 6.0 * np.sqrt(2.0 * ok.sum()), (stat, ok.sum())
    # pointwise: the table inverse stays close to the exact inverse
    samp = L.or_qed_sample_rad if process == pic.QED_EMISSION else L.or_qed_sample_pair
    rs = np.array([0.05, 0.3, 0.5, 0.8, 0.97])
    got = sim_tables.pic_qed_eval(process, np.full(len(rs), chi), rs)
    ref = np.array([samp(chi, x) for x in rs])
    assert np.max(np.abs(got - ref)) < 2e-3


def test_monte_carlo_matches_oracle_event_by_event():
    """Same seed, same identities, same Philox draws: the photons created by
    the GPU and the oracle must be the same events (identities derived from
    the parent's stream) with the same energies.  The GPU uses tables, the
    oracle exact quadrature, so an event whose optical depth crosses zero
    within the rate difference may flip: at most a few such flips."""
    o = Q.make_oracle()
    s = pic.pic_create(1, (16,), (1.0,), Q.DT, Q.species_spec(), seed=Q.SEED)
    s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA)
    s.pic_set_field(pic.BZ, np.full(s.box(), Q.B0))
    s.pic_load_particles(0, *Q.electrons())
    e0 = Q.total_energy(s.pic_get_particles(0), s.pic_get_particles(1), s.pic_get_particles(2))
    s.pic_step(25)
    o.step(25)
    gid, _ = s.pic_get_qed_state(2)
    oid, _ = o.qed_state(2)
    common = np.intersect1d(gid, oid)
    info = {"photons": (len(gid), len(oid)), "electrons": (s.pic_particle_count(0), len(o.particles(0)["ux"])),
            "positrons": (s.pic_particle_count(1), len(o.particles(1)["ux"])), "common": len(common)}
    assert len(oid) > 30, info
    assert len(gid) - len(common) <= 3 and len(oid) - len(common) <= 3, info
    gk = s.pic_get_particles(2)
    ok = o.particles(2)
    ge = np.sqrt(gk["ux"] ** 2 + gk["uy"] ** 2 + gk["uz"] ** 2)
    oe = np.sqrt(ok["ux"] ** 2 + ok["uy"] ** 2 + ok["uz"] ** 2)
    gmap = dict(zip(gid.tolist(), ge.tolist()))
    omap = dict(zip(oid.tolist(), oe.tolist()))
    rel = np.array([abs(gmap[i] / omap[i] - 1.0) for i in common.tolist()])
    assert np.median(rel) < 1e-3 and np.max(rel) < 5e-2
    # pairs: positron identities are the electron identity + 1
    pid, _ = s.pic_get_qed_state(1)
    opid, _ = o.qed_state(1)
    assert abs(len(pid) - len(opid)) <= 2 and len(opid) >= 2
    # energy conservation of the whole ensemble (FP32 particles)
    e1 = Q.total_energy(s.pic_get_particles(0), s.pic_get_particles(1), s.pic_get_particles(2))
    assert abs(e1 - e0) <= 2e-5 * e0


def test_monte_carlo_fp64_form_matches_oracle():
    """The plain FP64 form (absolute positions, FP64 tables) against the
    oracle: the same events with the same photon energies, tighter than the
    FP32 form, and energy conserved to FP64 round-off."""
    o = Q.make_oracle()
    s = pic.pic_create(1, (16,), (1.0,), Q.DT, Q.species_spec(), seed=Q.SEED, precision=pic.FP64_PLAIN)
    s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA)
    s.pic_set_field(pic.BZ, np.full(s.box(), Q.B0))
    s.pic_load_particles(0, *Q.electrons())
    e0 = Q.total_energy(s.pic_get_particles(0), s.pic_get_particles(1), s.pic_get_particles(2))
    s.pic_step(25)
    o.step(25)
    gid, gtau = s.pic_get_qed_state(2)
    oid, otau = o.qed_state(2)
    common = np.intersect1d(gid, oid)
    assert len(oid) > 30 and len(gid) - len(common) <= 2 and len(oid) - len(common) <= 2, (len(gid), len(oid))
    gk, ok = s.pic_get_particles(2), o.particles(2)
    ge = dict(zip(gid.tolist(), np.sqrt(gk["ux"] ** 2 + gk["uy"] ** 2 + gk["uz"] ** 2).tolist()))
    oe = dict(zip(oid.tolist(), np.sqrt(ok["ux"] ** 2 + ok["uy"] ** 2 + ok["uz"] ** 2).tolist()))
    rel = np.array([abs(ge[i] / oe[i] - 1.0) for i in common.tolist()])
    assert np.median(rel) < 1e-4 and np.max(rel) < 5e-2, (np.median(rel), np.max(rel))
    e1 = Q.total_energy(s.pic_get_particles(0), s.pic_get_particles(1), s.pic_get_particles(2))
    assert abs(e1 - e0) <= 1e-9 * e0
    d = s.pic_diagnostics()  # converted photons stay in the arrays, dead, until the next sort
    assert d["n_alive"][2] == int(gk["alive"].sum()) and d["U_kin"][2] > 0.0


_N3, _DX3 = (8, 8, 8), (2.0, 2.0, 2.0)


def _electrons_3d():
    rng = np.random.default_rng(31)
    x = [rng.uniform(0.0, _N3[d] * _DX3[d], Q.N_E) for d in range(3)]
    u = np.sqrt(Q.GAMMA0 ** 2 - 1.0)
    ang = rng.uniform(0.0, 2.0 * np.pi, Q.N_E)
    return x[0], x[1], x[2], u * np.cos(ang), u * np.sin(ang), np.zeros(Q.N_E)


@pytest.fixture(scope="module")
def oracle_3d():
    """the oracle's 25 steps of the 3D set-up (shared by both forms)"""
    o = O.OracleSim(3, _N3, _DX3, Q.DT)
    for sp in Q.species_spec():
        o.add_species(sp[0], sp[1], sp[2], sp[3], kind=sp[4], qed=sp[5])
    o.set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA, photon_emin=0.0, seed=Q.SEED)
    o.set_field(O.BZ, np.full(o.box(), Q.B0))
    o.load(0, *_electrons_3d())
    o.step(25)
    return o


@pytest.mark.parametrize("prec", [pic.FP32_CELLOFF, pic.FP64_PLAIN])
def test_monte_carlo_3d_matches_oracle_event_by_event(prec, oracle_3d):
    """The same set-up on a periodic 8^3 grid with the electrons spread in 3D
    (the 3D QED push, photon push and spawn kernels): the photons and pairs
    are the oracle's events, with the oracle's photon energies and emission
    points, and the ensemble energy is conserved."""
    o = oracle_3d
    s = pic.pic_create(3, _N3, _DX3, Q.DT, Q.species_spec(), seed=Q.SEED, precision=prec)
    s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA)
    s.pic_set_field(pic.BZ, np.full(s.box(), Q.B0))
    s.pic_load_particles(0, *_electrons_3d())
    e0 = Q.total_energy(s.pic_get_particles(0), s.pic_get_particles(1), s.pic_get_particles(2))
    s.pic_step(25)
    gid, _ = s.pic_get_qed_state(2)
    oid, _ = o.qed_state(2)
    common = np.intersect1d(gid, oid)
    flips = 2 if prec == pic.FP64_PLAIN else 3
    assert len(oid) > 30 and len(gid) - len(common) <= flips and len(oid) - len(common) <= flips, (len(gid), len(oid))
    gk, ok = s.pic_get_particles(2), o.particles(2)
    ge = dict(zip(gid.tolist(), np.sqrt(gk["ux"] ** 2 + gk["uy"] ** 2 + gk["uz"] ** 2).tolist()))
    oe = dict(zip(oid.tolist(), np.sqrt(ok["ux"] ** 2 + ok["uy"] ** 2 + ok["uz"] ** 2).tolist()))
    rel = np.array([abs(ge[i] / oe[i] - 1.0) for i in common.tolist()])
    assert np.median(rel) < (1e-4 if prec == pic.FP64_PLAIN else 1e-3) and np.max(rel) < 5e-2
    # photons move at c along k from the parent's position (photons that
    # converted to pairs stay in the arrays, dead, until the next sort)
    gx = dict(zip(gid.tolist(), zip(gk["x"], gk["y"], gk["z"], gk["alive"])))
    ox = dict(zip(oid.tolist(), zip(ok["x"], ok["y"], ok["z"], ok["alive"])))
    L = np.array([_N3[d] * _DX3[d] for d in range(3)])
    both = [i for i in common.tolist() if gx[i][3] and ox[i][3]]
    assert len(both) >= 30
    for i in both[:50]:
        dd = np.abs(np.array(gx[i][:3]) - np.array(ox[i][:3]))
        dd = np.minimum(dd, L - dd)
        assert np.all(dd < 1e-3 * _DX3[0]), (i, gx[i], ox[i])
    pid, _ = s.pic_get_qed_state(1)
    opid, _ = o.qed_state(1)
    assert abs(len(pid) - len(opid)) <= 2 and len(opid) >= 2
    e1 = Q.total_energy(s.pic_get_particles(0), s.pic_get_particles(1), s.pic_get_particles(2))
    assert abs(e1 - e0) <= (1e-9 if prec == pic.FP64_PLAIN else 2e-5) * e0
