"""Pins of the oracle's QED functions (Sec. IV, Eqs. (23), (24)) to closed
forms, library Bessel functions and known asymptotic expansions."""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import oracle as O


@pytest.fixture(scope="module")
def L():
    return O.lib()


@pytest.mark.parametrize("nu", [1.0 / 3.0, 2.0 / 3.0])
@pytest.mark.parametrize("x", [1e-5, 1e-2, 0.3, 2.0, 17.0, 80.0])
def test_bessel_k_matches_library(L, nu, x):
    assert abs(L.or_bessel_k(nu, x) / special.kv(nu, x) - 1.0) < 1e-12


@pytest.mark.parametrize("y", [1e-3, 0.2, 1.5, 9.0])
def test_int_k13_matches_quadrature_of_library(L, y):
    ref, _ = integrate.quad(lambda x: special.kv(1.0 / 3.0, x), y, np.inf, epsabs=1e-14, epsrel=1e-12)
    assert abs(L.or_int_k13(y) / ref - 1.0) < 1e-9


def test_int_k13_total_is_pi_over_sqrt3(L):
    # Int_0^inf K_1/3 = pi / (2 cos(pi/6)) = pi / sqrt(3); the remainder near 0 is O(y^{2/3})
    assert abs(L.or_int_k13(1e-15) - math.pi / math.sqrt(3.0)) < 1e-8


def test_emission_rate_classical_limit(L):
    """gamma W_rad -> 5 alpha chi E_s / (2 sqrt 3): Int_0^1 Frad du -> 5 pi chi / 2,
    with the first quantum correction 1 - (8 sqrt3 / 15) chi"""
    for chi in (1e-4, 3e-4):
        g = L.or_qed_Grad(chi) / chi
        # the next term is +3.5 chi^2 (measured): allow 5 chi^2
        assert abs(g / (2.5 * math.pi) - (1.0 - 8.0 * math.sqrt(3.0) / 15.0 * chi)) < 5.0 * chi * chi + 1e-9


def test_radiated_power_larmor_limit(L):
    """Int_0^1 u Frad du -> 2 pi chi^2 / sqrt 3 (Larmor), correction 1 - (55 sqrt3 / 16) chi"""
    for chi in (1e-4, 3e-4):
        p = L.or_qed_Prad(chi) / (chi * chi)
        assert abs(p / (2.0 * math.pi / math.sqrt(3.0)) - (1.0 - 55.0 * math.sqrt(3.0) / 16.0 * chi)) < 60 * chi * chi


def test_pair_rate_small_chi_limit(L):
    """Int_0^1 Fpair dv of Eq. (24) -> (9 pi / (16 sqrt 2)) chi exp(-8 / (3 chi))
    as chi -> 0: with the prefactor alpha E_s / (sqrt3 pi k) of the rate,
    the known pair-creation limit W = (3 sqrt3 / (16 sqrt2)) alpha E_s chi
    exp(-8/(3 chi)) / k of a photon in a weak field.  The ratio approaches 1
    linearly in chi; its straight-line extrapolation to chi = 0 from three
    small chi gives 1 within 2e-4 (a factor 2 or a wrong exponent fails by
    orders of magnitude, a wrong power of chi by 10 %)"""
    chis = np.array([0.01, 0.02, 0.04])
    ratio = np.array([L.or_qed_Gpair(c) / (9.0 * math.pi / (16.0 * math.sqrt(2.0)) * c * math.exp(-8.0 / (3.0 * c)))
                      for c in chis])
    slope, intercept = np.polyfit(chis, ratio, 1)
    assert abs(intercept - 1.0) < 2e-4, (intercept, slope)
    assert np.all(np.abs(ratio - 1.0) < 0.25 * chis), ratio


def test_pair_spectrum_symmetric_and_positive(L):
    for chi in (0.5, 5.0, 50.0):
        for v in (0.05, 0.2, 0.37, 0.49):
            a, b = L.or_qed_Fpair(v, chi), L.or_qed_Fpair(1.0 - v, chi)
            assert a > 0 and abs(a - b) <= 1e-13 * a


def test_cdfs_monotone_from_zero_to_one(L):
    for chi in (0.49, 4.9, 49.0):
        us = np.linspace(0.0, 1.0, 21)
        c = [L.or_qed_cdf_rad(u, chi) for u in us]
        assert c[0] == 0.0 and abs(c[-1] - 1.0) < 1e-15 and np.all(np.diff(c) > 0)
        cp = [L.or_qed_cdf_pair(u, chi) for u in us]
        assert cp[0] == 0.0 and abs(cp[-1] - 1.0) < 1e-15 and np.all(np.diff(cp) >= 0)
        assert abs(L.or_qed_cdf_pair(0.5, chi) - 0.5) < 1e-10  # symmetry (quadrature accuracy)


def test_inverse_cdf_sampler_inverts_the_cdf(L):
    for chi, r in ((0.49, 0.1), (4.9, 0.6), (49.0, 0.93)):
        u = L.or_qed_sample_rad(chi, r)
        assert abs(L.or_qed_cdf_rad(u, chi) - r) < 1e-10
        v = L.or_qed_sample_pair(chi, r)
        assert abs(L.or_qed_cdf_pair(v, chi) - r) < 1e-10


def test_method_two_reproduces_the_spectrum(L):
    """Method II (u0 = r1^3 accepted when r2 < 3 r1^2 dW/du dt) draws from the
    same normalised spectrum as Method I: chi-square against Eq. (23)."""
    rng = np.random.default_rng(8)
    chi = 4.9
    # 3 r^2 Frad(r^3) -> 3 Gamma(2/3) (3 chi)^(2/3) as r -> 0; keep the
    # acceptance probability below one
    pmax = 3.0 * math.gamma(2.0 / 3.0) * (3.0 * chi) ** (2.0 / 3.0)
    dwdt = 0.5 / pmax
    acc = []
    r1 = rng.random(120000)
    r2 = rng.random(120000)
    for a, b in zip(r1, r2):
        u = L.or_qed_method2_rad(chi, dwdt, a, b)
        assert u != -2.0
        if u >= 0:
            acc.append(u)
    acc = np.array(acc)
    edges = np.linspace(0.0, 1.0, 11) ** 3
    counts, _ = np.histogram(acc, edges)
    cdf = np.array([L.or_qed_cdf_rad(e, chi) for e in edges])
    expect = np.diff(cdf) * len(acc)
    stat = np.sum((counts - expect) ** 2 / expect)
    assert len(acc) > 2000
    assert stat < 35.0  # chi^2 with 9 dof: p ~ 1e-4


# --------------------------------------------------------------------------
# the optical-depth Monte Carlo inside the oracle's step
# --------------------------------------------------------------------------

def test_qed_monte_carlo_conserves_energy_in_pure_B():
    """Electrons gyrating in a uniform B emit photons that convert to pairs;
    the magnetic field does no work, Boris keeps gamma, emission keeps
    gamma_e + eps_gamma and pair creation keeps eps_+ + eps_- = k, so the
    total energy is conserved to round-off.  The run must produce photons and
    pairs (otherwise the check would be empty)."""
    from tests import qed_setup as Q
    o = Q.make_oracle()
    e0 = Q.total_energy(o.particles(0), o.particles(1), o.particles(2))
    o.step(25)
    pe, pp, pg = o.particles(0), o.particles(1), o.particles(2)
    e1 = Q.total_energy(pe, pp, pg)
    assert len(pg["ux"]) > 30
    assert len(pp["ux"]) >= 2 and len(pe["ux"]) == Q.N_E + len(pp["ux"])
    assert abs(e1 - e0) <= 1e-12 * e0
    # every photon carries an identity drawn from its parent's Philox stream
    ids, tau = o.qed_state(2)
    assert len(np.unique(ids)) == len(ids) and np.all(tau > 0)


@pytest.mark.parametrize("chi", [0.01, 1.0, 50.0])
def test_total_emission_rate_matches_library_quadrature(L, chi):
    """Int_0^1 Frad du by scipy quad (with the Bessel functions of the
    library), split at u = 1/2 into s = u^(1/3) and t = (1-u)^(1/3)."""
    def F(u):
        y = 2 * u / (3 * chi * (1 - u))
        if y > 700:
            return 0.0
        ik = integrate.quad(lambda x: special.kv(1 / 3, x), y, np.inf, epsabs=0, epsrel=1e-12, limit=200)[0]
        return ((1 - u) + 1 / (1 - u)) * special.kv(2 / 3, y) - ik
    wh = 0.5 ** (1 / 3)
    a = integrate.quad(lambda s: 3 * s * s * F(s ** 3), 0, wh, epsabs=0, epsrel=1e-10, limit=400)[0]
    b = integrate.quad(lambda t: 3 * t * t * F(1 - t ** 3), 0, wh, epsabs=0, epsrel=1e-10, limit=400)[0]
    assert abs(L.or_qed_Grad(chi) / (a + b) - 1.0) < 1e-7


def test_caller_given_identities_restart_their_optical_depths():
    """A sample keeps the identities of its full load: set_ids gives a
    particle the identity and the initial optical depth that a load at that
    index draws."""
    def make():
        o = O.OracleSim(1, (16,), (1.0,), 0.02)
        o.add_species(-1.0, 1.0, 1e-12, 16, qed=1)
        o.set_qed(photon_sp=-1, electron_sp=0, lambda_r_m=1e-6, seed=99)
        return o

    full = make()
    z = np.zeros(10)
    full.load(0, np.linspace(0.5, 9.5, 10), None, None, z, z, z)
    ids, tau = full.qed_state(0)
    sub = make()
    pick = np.array([7, 2, 9])
    sub.load(0, np.linspace(0.5, 9.5, 10)[pick], None, None, z[:3], z[:3], z[:3])
    sub.set_ids(0, ids[pick])
    sids, stau = sub.qed_state(0)
    assert np.array_equal(sids, ids[pick]) and np.array_equal(stau, tau[pick])
    assert len(set(tau.tolist())) == 10
