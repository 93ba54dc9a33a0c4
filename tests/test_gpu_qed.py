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
    rs = np.array([1e-4, 1e-3, 0.01, 0.05, 0.3, 0.5, 0.8, 0.97, 0.999, 0.9999])
    got = sim_tables.pic_qed_eval(process, np.full(len(rs), chi), rs)
    ref = np.array([samp(chi, x) for x in rs])
    # relative, in the fraction and in its complement (the recoil 1 - u)
    assert np.max(np.abs(got / ref - 1.0)) < 1e-3, got / ref - 1.0
    assert np.max(np.abs((1.0 - got) / (1.0 - ref) - 1.0)) < 1e-3, (1.0 - got) / (1.0 - ref) - 1.0


# relative difference of the GPU's total rates from the oracle's quadrature:
# tables within 2e-5 (emission) and 1e-4 (pairs) of it
# (test_rate_tables_match_oracle_quadrature), plus FP32 chi and rate in the
# FP32 form
DELTA = {pic.FP32_CELLOFF: (5e-5, 2e-4), pic.FP64_PLAIN: (3e-5, 1.5e-4)}


@pytest.mark.parametrize("pusher", [pic.PUSHER_BORIS, pic.PUSHER_VAY])
@pytest.mark.parametrize("prec", [pic.FP32_CELLOFF, pic.FP64_PLAIN])
def test_monte_carlo_matches_oracle_event_by_event(prec, pusher):
    """Same seed, same identities, same Philox draws, stepped together: the
    initial optical depths are identical, every decision (emission, pair
    creation) is the oracle's except flips whose optical depth ended within
    the band the rate difference explains, optical depths agree within that
    difference between events, photons of common events carry the oracle's
    energy within 1e-3, and the ensemble energy is conserved.  Both pushers
    (the QED push kernels carry Boris and Vay)."""
    o = Q.make_oracle()
    o.set_pusher(pusher)
    s = pic.pic_create(1, (16,), (1.0,), Q.DT, Q.species_spec(), seed=Q.SEED, precision=prec, pusher=pusher)
    s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA)
    s.pic_set_field(pic.BZ, np.full(s.box(), Q.B0))
    s.pic_load_particles(0, *Q.electrons())
    e0 = Q.total_energy(s.pic_get_particles(0), s.pic_get_particles(1), s.pic_get_particles(2))
    r = Q.compare_events(s, o, 25, *DELTA[prec], Q.photon_chi_in_bz(o.Es))
    assert r["events"] >= 150 and r["conversions"] >= 5 and r["energies"] >= 150, r
    assert r["flips"] <= 0.05 * r["events"], r
    e1 = Q.total_energy(s.pic_get_particles(0), s.pic_get_particles(1), s.pic_get_particles(2))
    assert abs(e1 - e0) <= (1e-9 if prec == pic.FP64_PLAIN else 2e-5) * e0
    d = s.pic_diagnostics()  # converted photons stay in the arrays, dead, until the next sort
    assert d["n_alive"][2] == int(s.pic_get_particles(2)["alive"].sum()) and d["U_kin"][2] > 0.0


_N3, _DX3 = (8, 8, 8), (2.0, 2.0, 2.0)


def _electrons_3d():
    rng = np.random.default_rng(31)
    x = [rng.uniform(0.0, _N3[d] * _DX3[d], Q.N_E) for d in range(3)]
    u = np.sqrt(Q.GAMMA0 ** 2 - 1.0)
    ang = rng.uniform(0.0, 2.0 * np.pi, Q.N_E)
    return x[0], x[1], x[2], u * np.cos(ang), u * np.sin(ang), np.zeros(Q.N_E)


def _oracle_3d():
    o = O.OracleSim(3, _N3, _DX3, Q.DT)
    for sp in Q.species_spec():
        o.add_species(sp[0], sp[1], sp[2], sp[3], kind=sp[4], qed=sp[5])
    o.set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA, photon_emin=0.0, seed=Q.SEED)
    o.set_field(O.BZ, np.full(o.box(), Q.B0))
    o.load(0, *_electrons_3d())
    return o


@pytest.mark.parametrize("prec,tiled", [(pic.FP32_CELLOFF, False), (pic.FP64_PLAIN, False),
                                        (pic.FP32_CELLOFF, True)])
def test_monte_carlo_3d_matches_oracle_event_by_event(prec, tiled):
    """The same set-up on a periodic 8^3 grid with the electrons spread in 3D
    (the 3D QED push, photon push and spawn kernels; tiled: 4^3 tiles and a
    sort every 4 steps, the leptons' Monte Carlo fused into the 3D tiled
    push), compared step by step as in 1D; live photons of common events sit
    where the oracle's are (they move at c along k from the parent's
    position), and the ensemble energy is conserved."""
    o = _oracle_3d()
    kw = dict(sort_interval=4, tile=(4, 4, 4)) if tiled else {}
    s = pic.pic_create(3, _N3, _DX3, Q.DT, Q.species_spec(), seed=Q.SEED, precision=prec, **kw)
    s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA)
    s.pic_set_field(pic.BZ, np.full(s.box(), Q.B0))
    s.pic_load_particles(0, *_electrons_3d())
    e0 = Q.total_energy(s.pic_get_particles(0), s.pic_get_particles(1), s.pic_get_particles(2))
    r = Q.compare_events(s, o, 25, *DELTA[prec], Q.photon_chi_in_bz(o.Es))
    assert r["events"] >= 150 and r["conversions"] >= 5 and r["flips"] <= 0.05 * r["events"], r
    gid, _ = s.pic_get_qed_state(2)
    oid, _ = o.qed_state(2)
    common = np.intersect1d(gid, oid)
    gk, ok = s.pic_get_particles(2), o.particles(2)
    gx = dict(zip(gid.tolist(), zip(gk["x"], gk["y"], gk["z"], gk["alive"])))
    ox = dict(zip(oid.tolist(), zip(ok["x"], ok["y"], ok["z"], ok["alive"])))
    L = np.array([_N3[d] * _DX3[d] for d in range(3)])
    both = [i for i in common.tolist() if gx[i][3] and ox[i][3]]
    assert len(both) >= 30
    for i in both:
        dd = np.abs(np.array(gx[i][:3]) - np.array(ox[i][:3]))
        dd = np.minimum(dd, L - dd)
        assert np.all(dd < 1e-3 * _DX3[0]), (i, gx[i], ox[i])
    e1 = Q.total_energy(s.pic_get_particles(0), s.pic_get_particles(1), s.pic_get_particles(2))
    assert abs(e1 - e0) <= (1e-9 if prec == pic.FP64_PLAIN else 2e-5) * e0


_N2, _DX2 = (32, 32), (1.0, 1.0)


def _electrons_2d():
    rng = np.random.default_rng(37)
    x = [rng.uniform(0.0, _N2[d] * _DX2[d], Q.N_E) for d in range(2)]
    u = np.sqrt(Q.GAMMA0 ** 2 - 1.0)
    ang = rng.uniform(0.0, 2.0 * np.pi, Q.N_E)
    return x[0], x[1], None, u * np.cos(ang), u * np.sin(ang), np.zeros(Q.N_E)


def _oracle_2d():
    o = O.OracleSim(2, _N2, _DX2, Q.DT)
    for sp in Q.species_spec():
        o.add_species(sp[0], sp[1], sp[2], sp[3], kind=sp[4], qed=sp[5])
    o.set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA, photon_emin=0.0, seed=Q.SEED)
    o.set_field(O.BZ, np.full(o.box(), Q.B0))
    o.load(0, *_electrons_2d())
    return o


def test_monte_carlo_2d_tiled_matches_oracle_event_by_event():
    """FP32 on a periodic 32^2 grid with 8x8 tiles and a sort every 4 steps:
    after the first sort the leptons' Monte Carlo runs fused into the tiled
    push (the sorted particles' work items; pairs appended since the sort on
    the one-thread-per-particle kernel), compared with the oracle step by
    step as in 1D.  The tiled path is the one taken: with it the push phase
    issues more launches (the tiled kernel and the appended tail) than with
    the simple kernel alone."""
    o = _oracle_2d()
    s = pic.pic_create(2, _N2, _DX2, Q.DT, Q.species_spec(), seed=Q.SEED, sort_interval=4, tile=(8, 8))
    s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA)
    s.pic_set_field(pic.BZ, np.full(s.box(), Q.B0))
    s.pic_load_particles(0, *_electrons_2d())
    e0 = Q.total_energy(s.pic_get_particles(0), s.pic_get_particles(1), s.pic_get_particles(2))
    s.pic_profile(True)
    r = Q.compare_events(s, o, 25, *DELTA[pic.FP32_CELLOFF], Q.photon_chi_in_bz(o.Es))
    assert r["events"] >= 150 and r["conversions"] >= 5 and r["flips"] <= 0.05 * r["events"], r
    e1 = Q.total_energy(s.pic_get_particles(0), s.pic_get_particles(1), s.pic_get_particles(2))
    assert abs(e1 - e0) <= 2e-5 * e0
    tiled = s.pic_profile_read()["launches"]["push"]
    s.close()
    ref = pic.pic_create(2, _N2, _DX2, Q.DT, Q.species_spec(), seed=Q.SEED, sort_interval=4, tile=(8, 8),
                         push_variant=pic.PUSH_SIMPLE)
    ref.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA)
    ref.pic_set_field(pic.BZ, np.full(ref.box(), Q.B0))
    ref.pic_load_particles(0, *_electrons_2d())
    ref.pic_profile(True)
    for _ in range(25):
        ref.pic_step(1)
    simple = ref.pic_profile_read()["launches"]["push"]
    ref.close()
    print("push-phase launches, tiled vs simple:", tiled, simple)
    assert tiled > simple, (tiled, simple)
