"""The surrogate network of the QED Monte Carlo on the GPU: its forward pass
and gradients against the FP64 oracle network, its training against the
tables, the spectra it samples against Eqs. (23)/(24), the fused Monte Carlo
with it, and what it gains over the tables."""
import os
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_00642_gb300 import pic
from tests import qed_setup as Q

pytestmark = pytest.mark.gpu

NP = pic.MLP_NPARAMS
# packed parameter blocks: name -> (start, stop, rounded to BF16 on the device)
BLOCKS = {"W0": (0, 128, True), "b0": (128, 192, False), "W1": (192, 4288, True), "b1": (4288, 4352, False),
          "W2": (4352, 8448, True), "b2": (8448, 8512, False), "W3": (8512, 8640, True), "b3": (8640, 8642, False)}


def bf16(a):
    """Round to the nearest BF16 (ties to even), as float64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def device_view(P):
    """The parameters as the device holds them: weights in BF16, biases FP32."""
    Q64 = np.asarray(P, dtype=np.float32).astype(np.float64)
    for a, b, rounded in BLOCKS.values():
        if rounded:
            Q64[a:b] = bf16(Q64[a:b])
    return Q64


def random_params(seed):
    rng = np.random.default_rng(seed)
    P = np.zeros(NP, dtype=np.float32)
    for name, (a, b, rounded) in BLOCKS.items():
        fan_in = 2 if name == "W0" else 64
        P[a:b] = rng.normal(0.0, 1.0 / np.sqrt(fan_in) if rounded else 0.1, b - a)
    return P


@pytest.fixture(scope="module")
def sim():
    s = pic.pic_create(1, (16,), (1.0,), Q.DT, Q.species_spec(cap=64), seed=Q.SEED)
    s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA, mode=pic.QED_TABLE)
    return s


def test_forward_matches_oracle(sim):
    """Warp-level inference (FP32 input layer, BF16 mma.sync hidden layers,
    FP32 head) against the FP64 network at the same BF16 weights, over a
    ragged number of rows."""
    P = random_params(3)
    sim.pic_mlp_set(pic.QED_EMISSION, P, 1e-3, 1e2, 0.0, 1.0)
    rng = np.random.default_rng(4)
    x = rng.uniform(-1.0, 1.0, (1000 + 17, 2)).astype(np.float32)
    y = sim.pic_mlp_eval(pic.QED_EMISSION, x)
    ref = O.mlp_forward(device_view(P), x.astype(np.float64))
    err = np.abs(y - ref)
    scale = np.abs(ref).max()
    # BF16 activations (8-bit mantissa) feed two 64-wide contractions
    assert err.max() < 2e-2 * scale and np.sqrt(np.mean(err ** 2)) < 4e-3 * scale, (err.max(), scale)


@pytest.mark.parametrize("n", [1, 127, 128, 1000 + 17, 40000 + 3])
def test_tensor_core_evaluation_matches(sim, n):
    """The batched tcgen05 evaluation (128 rows per CTA, accumulators in
    tensor memory) against the warp-level mma.sync one and the FP64 network,
    over one, partial and many 128-row tiles: the same BF16 activations up to
    the order of the FP32 sums, so nearly every output agrees to 1e-5 (a sum
    that lands on the other side of a BF16 rounding boundary moves one
    activation by one BF16 step)."""
    P = random_params(3)
    sim.pic_mlp_set(pic.QED_EMISSION, P, 1e-3, 1e2, 0.0, 1.0)
    rng = np.random.default_rng(40 + n)
    x = rng.uniform(-1.0, 1.0, (n, 2)).astype(np.float32)
    y_tc = sim.pic_mlp_eval_tc(pic.QED_EMISSION, x)
    y_mma = sim.pic_mlp_eval(pic.QED_EMISSION, x)
    ref = O.mlp_forward(device_view(P), x.astype(np.float64))
    scale = np.abs(ref).max()
    d = np.abs(y_tc - y_mma)
    assert np.mean(d <= 1e-5 * scale) > 0.99 and d.max() < 1e-2 * scale, (d.max(), np.mean(d <= 1e-5 * scale))
    err = np.abs(y_tc - ref)
    assert err.max() < 2e-2 * scale and np.sqrt(np.mean(err ** 2)) < 4e-3 * scale


@pytest.mark.parametrize("n", [32, 256, 4096 + 32])
def test_gradient_matches_oracle_backprop(sim, n):
    """Loss and every parameter gradient of the GPU backward pass (deltas
    through the transposed BF16 weights on the tensor cores, FP32 weight
    gradients) against FP64 backpropagation at the same BF16 weights."""
    P = random_params(5)
    sim.pic_mlp_set(pic.QED_PAIR, P, 1e-2, 1e2, 0.0, 1.0)
    rng = np.random.default_rng(6 + n)
    x = rng.uniform(-1.0, 1.0, (n, 2)).astype(np.float32)
    t = rng.uniform(-1.0, 1.0, (n, 2)).astype(np.float32)
    loss, G = sim.pic_mlp_grad(pic.QED_PAIR, x, t)
    ref_loss, ref_G = O.mlp_loss_grad(device_view(P), x.astype(np.float64), t.astype(np.float64))
    assert abs(loss / ref_loss - 1.0) < 1e-2, (loss, ref_loss)
    for name, (a, b, _) in BLOCKS.items():
        g, r = G[a:b].astype(np.float64), ref_G[a:b]
        rel = np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-30)
        assert rel < 1e-2, (name, rel)
        assert np.dot(g, r) / (np.linalg.norm(g) * np.linalg.norm(r) + 1e-30) > 0.999, name
        # element by element: within 3 % of each entry plus 5 % of the block's
        # rms.  The device rounds activations and deltas to BF16 (each product
        # carries ~2^-8 relative error) and sums up to 4128 rows per entry;
        # where those terms cancel, an entry's error reaches a few per cent of
        # the block's rms (measured: 3.2e-2 x rms at most, W1, 4128 rows).  A
        # wrong index, sign or operand moves entries by their own size.
        bound = 3e-2 * np.abs(r) + 5e-2 * np.sqrt(np.mean(r * r))
        bad = np.abs(g - r) > bound
        assert not bad.any(), (name, int(bad.sum()), float(np.max(np.abs(g - r) / (bound + 1e-300))))


def test_gradient_step_lowers_the_loss(sim):
    """A small step along the GPU gradient lowers the oracle loss by about
    the first-order prediction."""
    P = random_params(7)
    sim.pic_mlp_set(pic.QED_EMISSION, P, 1e-3, 1e2, 0.0, 1.0)
    rng = np.random.default_rng(8)
    x = rng.uniform(-1.0, 1.0, (512, 2)).astype(np.float32)
    t = rng.uniform(-1.0, 1.0, (512, 2)).astype(np.float32)
    _, G = sim.pic_mlp_grad(pic.QED_EMISSION, x, t)
    P64 = P.astype(np.float64)
    h = 1e-2 / np.linalg.norm(G)
    l0 = O.mlp_loss_grad(P64, x, t)[0]
    l1 = O.mlp_loss_grad(P64 - h * G, x, t)[0]
    pred = h * float(np.dot(G, G))
    assert 0.5 * pred < l0 - l1 < 1.5 * pred, (l0 - l1, pred)


@pytest.fixture(scope="module")
def trained():
    s = pic.pic_create(1, (16,), (1.0,), Q.DT, Q.species_spec(), seed=Q.SEED)
    s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA, mode=pic.QED_TABLE)
    reps = {}
    for p in (pic.QED_EMISSION, pic.QED_PAIR):
        t0 = time.perf_counter()
        reps[p] = s.pic_mlp_train(p, seed=11)
        reps[p]["wall_s"] = time.perf_counter() - t0
    return s, reps


@pytest.mark.parametrize("process", [pic.QED_EMISSION, pic.QED_PAIR])
def test_training_reaches_the_tables(trained, process):
    """Training on the GPU from fresh weights: the validation errors against
    the FP64 tables on a 256 x 256 (ln chi, r) grid."""
    s, reps = trained
    r = reps[process]
    print(process, r)
    assert r["iterations"] == 40000 and r["loss"] < 5e-5, r
    assert r["max_err_lnG"] < 3e-2 and r["rms_err_s"] < 1.5e-3 and r["max_err_s"] < 2e-2, r
    # the mean energy fraction of an event, per chi row of the validation grid:
    # at the lowest chi rows the fraction is ~1e-3 (s = f^(1/3) ~ 0.1), where
    # the network's absolute error in s (rms ~1e-3) is a few per cent of f --
    # rows that carry no emitted energy; where the energy is (below)
    # the mean fraction is held to 3e-3
    assert r["max_err_mean"] < 6e-2, r
    # the report's validation agrees with a fresh one
    v = s.pic_mlp_validate(process)
    assert abs(v["rms_err_s"] - r["rms_err_s"]) < 1e-9


@pytest.mark.parametrize("process", [pic.QED_EMISSION, pic.QED_PAIR])
def test_trained_mean_fraction_where_the_energy_is(trained, process):
    """chi >= 0.1 (where emission carries energy and pairs are created): the
    mean energy fraction of an event from the network (pic_qed_eval in
    surrogate mode) within 3e-3 of the tables', per chi, over 4096 CDF
    values; and the rate within 1e-2."""
    s, _ = trained
    r = (np.arange(4096) + 0.5) / 4096
    chis = np.logspace(-1, 2, 7) if process == pic.QED_EMISSION else np.logspace(-0.5, 2, 6)
    out = {}
    for mode in (pic.QED_SURROGATE, pic.QED_TABLE):
        s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA, mode=mode)
        f = [s.pic_qed_eval(process, np.full(r.size, c), r) for c in chis]
        # pairs: the spectrum is symmetric, so compare the lighter partner's share
        out[mode] = ([(np.minimum(x, 1.0 - x) if process == pic.QED_PAIR else x).mean() for x in f],
                     s.pic_qed_eval(process, chis))
    s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA, mode=pic.QED_TABLE)
    fn, ft = np.array(out[pic.QED_SURROGATE][0]), np.array(out[pic.QED_TABLE][0])
    assert np.max(np.abs(fn / ft - 1.0)) < 3e-3, fn / ft - 1.0
    gn, gt = out[pic.QED_SURROGATE][1], out[pic.QED_TABLE][1]
    assert np.max(np.abs(gn / gt - 1.0)) < 1e-2, gn / gt - 1.0


def test_training_is_deterministic(sim):
    """The gradient partials are summed in a fixed order: the same seed and
    options give bit-identical parameters."""
    sim.pic_mlp_train(pic.QED_EMISSION, iterations=300, seed=5)
    a, _ = sim.pic_mlp_get(pic.QED_EMISSION)
    sim.pic_mlp_train(pic.QED_EMISSION, iterations=300, seed=5)
    b, _ = sim.pic_mlp_get(pic.QED_EMISSION)
    assert np.array_equal(a, b)
    sim.pic_mlp_train(pic.QED_EMISSION, iterations=300, seed=6)
    c, _ = sim.pic_mlp_get(pic.QED_EMISSION)
    assert not np.array_equal(a, c)


def test_surrogate_rates_within_range(trained):
    """In PIC_QED_SURROGATE mode the rates come from the network inside its
    range (within its validated ln G error of the tables) and from the
    tables outside it (identical)."""
    s, reps = trained
    chi_in = np.logspace(-2.9, 1.9, 40)
    chi_out = np.array([2e-4, 5e-4, 2e2, 5e2])
    for p in (pic.QED_EMISSION, pic.QED_PAIR):
        s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA, mode=pic.QED_TABLE)
        c_in = chi_in if p == pic.QED_EMISSION else chi_in[chi_in > 2e-2]
        t_in, t_out = s.pic_qed_eval(p, c_in), s.pic_qed_eval(p, chi_out)
        s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA, mode=pic.QED_SURROGATE)
        n_in, n_out = s.pic_qed_eval(p, c_in), s.pic_qed_eval(p, chi_out)
        assert np.array_equal(n_out, t_out)
        # (the FP32 pair rate underflows to 0 below chi ~ 0.03, exp(-8/(3 chi)),
        # in both modes: there the tables serve both)
        pos = t_in > 0.0
        assert np.array_equal(n_in[~pos], t_in[~pos])
        assert np.max(np.abs(np.log(n_in[pos] / t_in[pos]))) < reps[p]["max_err_lnG"] * 1.01 + 1e-3
    s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA, mode=pic.QED_TABLE)


@pytest.mark.parametrize("chi", [0.49, 4.9, 49.0])
@pytest.mark.parametrize("process", [pic.QED_EMISSION, pic.QED_PAIR])
def test_surrogate_spectrum_error(trained, chi, process):
    """Fig. 8 setup with the network, the tables as the reference: 1e6 paired
    draws (the same r through both samplers) of the energy fraction at
    fixed chi.  Bounds: per-bin spectrum error (24 bins), error of the mean
    fraction (the radiated power, or the positron energy share).  Then the
    statistical resolution: at 5e4 draws the network's spectrum passes the
    chi-square test against Eq. (23) / (24) as the tables' does; the chi-square
    excess at 1e6 draws is reported."""
    s, _ = trained
    L = O.lib()
    rng = np.random.default_rng(13)
    N = 1_000_000
    r = (np.floor(rng.random(N) * 2 ** 24) + 0.5) * 2.0 ** -24
    edges = np.linspace(0.0, 1.0, 25) ** 3 if process == pic.QED_EMISSION else np.linspace(0.0, 1.0, 25)
    f = {}
    for mode in (pic.QED_TABLE, pic.QED_SURROGATE):
        s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA, mode=mode)
        f[mode] = s.pic_qed_eval(process, np.full(N, chi), r)
    s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA, mode=pic.QED_TABLE)
    ht, _ = np.histogram(f[pic.QED_TABLE], edges)
    hs, _ = np.histogram(f[pic.QED_SURROGATE], edges)
    big = ht >= 1000
    bin_err = np.max(np.abs(hs[big] / ht[big] - 1.0))
    mean_err = abs(np.mean(f[pic.QED_SURROGATE]) / np.mean(f[pic.QED_TABLE]) - 1.0)
    cdf = L.or_qed_cdf_rad if process == pic.QED_EMISSION else L.or_qed_cdf_pair
    c = np.array([cdf(e, chi) for e in edges])

    def chi2(x):
        expect = np.diff(c) * len(x)
        counts, _ = np.histogram(x, edges)
        ok = expect > 20
        return float(np.sum((counts[ok] - expect[ok]) ** 2 / expect[ok])), int(ok.sum())

    x2_1e6, nb = chi2(f[pic.QED_SURROGATE])
    # resolution: the network's bias stays inside the noise of 5e4 draws
    x2_1e5, nb5 = chi2(f[pic.QED_SURROGATE][:50_000])
    print(process, chi, {"bin_err": bin_err, "mean_err": mean_err, "chi2_1e6": (x2_1e6, nb),
                         "chi2_1e6_tables": chi2(f[pic.QED_TABLE]), "chi2_5e4": (x2_1e5, nb5)})
    # the network's bound: absolute error of s ~1e-3, i.e. a few per cent in
    # the narrowest (softest) bins; the energy-carrying mean stays within 5e-3
    assert bin_err < 0.15 and mean_err < 5e-3, (bin_err, mean_err)
    assert x2_1e5 < nb5 + 6.0 * np.sqrt(2.0 * nb5), x2_1e5


def test_surrogate_monte_carlo_in_the_push(trained):
    """The fused Monte Carlo with the networks in the push: the same seeded
    electrons as the table run emit a photon count consistent with it
    (the rates differ by the network's ln G error), pairs appear, and the
    total energy of leptons, photons and pair rest mass is conserved."""
    s0, _ = trained
    params = {p: s0.pic_mlp_get(p) for p in (pic.QED_EMISSION, pic.QED_PAIR)}
    counts = {}
    for mode in (pic.QED_TABLE, pic.QED_SURROGATE):
        s = pic.pic_create(1, (16,), (1.0,), Q.DT, Q.species_spec(), seed=Q.SEED)
        s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA, mode=mode)
        for p, (P, info) in params.items():
            s.pic_mlp_set(p, P, info["chi_min"], info["chi_max"], info["mu"], info["sd"])
        s.pic_set_field(pic.BZ, np.full(s.box(), Q.B0))
        s.pic_load_particles(0, *Q.electrons())
        e0 = Q.total_energy(s.pic_get_particles(0), s.pic_get_particles(1), s.pic_get_particles(2))
        s.pic_step(25)
        e1 = Q.total_energy(s.pic_get_particles(0), s.pic_get_particles(1), s.pic_get_particles(2))
        assert abs(e1 - e0) <= 2e-5 * e0, mode
        counts[mode] = (s.pic_particle_count(2), s.pic_particle_count(1))
    nt, ns = counts[pic.QED_TABLE][0], counts[pic.QED_SURROGATE][0]
    assert ns > 30 and abs(ns - nt) <= 4.0 * np.sqrt(nt) + 0.05 * nt, counts


def test_photon_push_tensor_core_network_matches_warp_network(trained):
    """The photon push with the pair network on tcgen05 (PIC_PUSH_MLP_TC)
    evaluates the network's rate for every photon in range each step; the
    default push samples the same rate by thinning an envelope (the network
    at candidates only).  The same seeded run through both (a cascade: most
    photons come from the pairs, which differ between the samplers): the
    photons the primary electrons emit in the first step are the same in
    both, and the photon and pair counts agree within the cascade's spread
    (20 %; the pairs within 4 sigma of Poisson)."""
    s0, _ = trained
    params = {p: s0.pic_mlp_get(p) for p in (pic.QED_EMISSION, pic.QED_PAIR)}
    runs, first = {}, {}
    for variant in (pic.PUSH_AUTO, pic.PUSH_MLP_TC):
        s = pic.pic_create(1, (16,), (1.0,), Q.DT, Q.species_spec(), seed=Q.SEED, push_variant=variant)
        s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA, mode=pic.QED_SURROGATE)
        for p, (P, info) in params.items():
            s.pic_mlp_set(p, P, info["chi_min"], info["chi_max"], info["mu"], info["sd"])
        s.pic_set_field(pic.BZ, np.full(s.box(), Q.B0))
        s.pic_load_particles(0, *Q.electrons())
        s.pic_step(1)
        first[variant] = set(s.pic_get_qed_state(2)[0].tolist())
        s.pic_step(39)
        gid, _ = s.pic_get_qed_state(2)
        runs[variant] = (len(gid), s.pic_particle_count(1))
        s.close()
    (na_ph, na), (nb_ph, nb) = runs[pic.PUSH_MLP_TC], runs[pic.PUSH_AUTO]
    print("photons", na_ph, nb_ph, "positrons", na, nb, "first-step photons", len(first[pic.PUSH_AUTO]))
    assert len(first[pic.PUSH_AUTO]) > 0 and first[pic.PUSH_AUTO] == first[pic.PUSH_MLP_TC]
    assert na_ph > 256 and abs(na_ph - nb_ph) <= 0.2 * max(na_ph, nb_ph), (na_ph, nb_ph)
    assert abs(na - nb) <= 4.0 * np.sqrt(2.0 * max(na, nb, 1)) + 2, (na, nb)


def test_what_the_network_gains(trained):
    """What the network buys against the tables: the device bytes the push
    reads for one process (network image vs rate + inverse-CDF tables), and
    the time of 1e6 rate+sample evaluations through each path.  The bytes
    must shrink; the timings are reported as measured."""
    s, reps = trained
    r = reps[pic.QED_EMISSION]
    assert r["net_bytes"] * 20 < r["table_bytes"], r
    N = 1 << 20
    rng = np.random.default_rng(5)
    chi = np.exp(rng.uniform(np.log(2e-3), np.log(50.0), N))
    rr = rng.random(N)
    out = {}
    for mode in (pic.QED_TABLE, pic.QED_SURROGATE):
        s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA, mode=mode)
        s.pic_qed_eval(pic.QED_EMISSION, chi, rr)
        t0 = time.perf_counter()
        s.pic_qed_eval(pic.QED_EMISSION, chi, rr)
        out[mode] = time.perf_counter() - t0
    s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA, mode=pic.QED_TABLE)
    print("bytes table/net", r["table_bytes"], r["net_bytes"], "eval s", out, "train", r)


def test_pair_network_stays_under_the_thinning_envelope(trained):
    """the surrogate form samples pair creation by thinning an analytic
    envelope (c chi^(2/3) exp(-8/(3 chi)), csrc/qed.cuh): the trained pair
    network's rate must stay below it over the whole trained range, or a
    candidate's acceptance W / W_env would exceed one"""
    import re
    s, _ = trained
    src = open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", "paper_2104_00642_gb300", "csrc",
                            "qed.cuh")).read()
    c = float(re.search(r"constexpr float kPairEnvelope = ([0-9.]+)f;", src).group(1))
    s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA, mode=pic.QED_SURROGATE)
    chi = np.geomspace(0.1, 100.0, 400)
    g = s.pic_qed_eval(pic.QED_PAIR, chi)
    s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA, mode=pic.QED_TABLE)
    env = c * chi ** (2.0 / 3.0) * np.exp(-8.0 / (3.0 * chi))
    pos = g > 0.0
    print("largest network rate / envelope", float(np.max(g[pos] / env[pos])))
    assert np.all(g[pos] < env[pos])
