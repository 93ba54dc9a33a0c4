"""A shared QED test setup: ultra-relativistic electrons gyrating in a
uniform magnetic field B_z on a small periodic 1D grid, with photon emission
and pair creation on.  The particle weight is tiny so that self-fields do not
matter; B does no work, so the total energy of electrons, positrons, photons
and pair rest mass is conserved exactly by the method (collinear emission
with recoil gamma (1 - u), pair energies summing to the photon's)."""
import math

import numpy as np

LAMBDA = 1e-6
GAMMA0 = 2000.0
B0 = 3000.0       # chi ~ gamma B / E_s ~ 14.6
DT = 0.02
N_E = 24
W = 1e-12
SEED = 0x5EED5EED12345


def electrons():
    x = (np.arange(N_E) + 0.37) * (16.0 / N_E)
    z = np.zeros(N_E)
    u = np.sqrt(GAMMA0 ** 2 - 1.0)
    uy = np.full(N_E, u)
    return x, z.copy(), z.copy(), z.copy(), uy, z.copy()


def species_spec(cap=4000):
    # (q, m, w, capacity, kind, qed): electrons, positrons, photons
    return [(-1.0, 1.0, W, cap, 0, 1), (1.0, 1.0, W, cap, 0, 1), (0.0, 0.0, W, 4 * cap, 1, 0)]


def total_energy(parts_e, parts_p, parts_g):
    def lep(p):
        if len(p["ux"]) == 0:
            return 0.0
        a = p["alive"] == 1
        uu = p["ux"][a] ** 2 + p["uy"][a] ** 2 + p["uz"][a] ** 2
        return float(np.sum(np.sqrt(1.0 + uu)))  # gamma including rest mass

    def ph(p):
        if len(p["ux"]) == 0:
            return 0.0
        a = p["alive"] == 1
        return float(np.sum(np.sqrt(p["ux"][a] ** 2 + p["uy"][a] ** 2 + p["uz"][a] ** 2)))

    return lep(parts_e) + lep(parts_p) + ph(parts_g)


def make_oracle():
    from oracle import oracle as O
    o = O.OracleSim(1, (16,), (1.0,), DT)
    for s in species_spec():
        o.add_species(s[0], s[1], s[2], s[3], kind=s[4], qed=s[5])
    o.set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=LAMBDA, photon_emin=0.0, seed=SEED)
    o.set_field(O.BZ, np.full(o.box(), B0))
    o.load(0, *electrons())
    return o


# ----------------------------------------------------------------------
# event-by-event comparison of a GPU run with the oracle, step by step
# ----------------------------------------------------------------------

def child_id(parent_id, step, purpose):
    """identity of the child of an event (Philox counter (id, step, purpose),
    words 2-3), as both sides derive it"""
    from oracle import oracle as O
    pid = int(parent_id)
    w = O.philox4x32_10([pid & 0xFFFFFFFF, pid >> 32, int(step) & 0xFFFFFFFF, purpose],
                        [SEED & 0xFFFFFFFF, SEED >> 32])
    return (int(w[3]) << 32) | int(w[2])


def _state_gpu(s, sp):
    ids, tau = s.pic_get_qed_state(sp)
    p = s.pic_get_particles(sp)
    return ids, tau, p


def _state_oracle(o, sp):
    ids, tau = o.qed_state(sp)
    return ids, tau, o.particles(sp)


def photon_chi_in_bz(Es, B=B0):
    """chi of a photon of momentum k in the uniform B_z of these set-ups"""
    return lambda kx, ky, kz: math.hypot(kx, ky) * B / Es


def compare_events(s, o, steps, delta, delta_pair, photon_chi, e_sp=0, ph_sp=2, pos_sp=1, energy_tol=1e-3,
                   reset_tol=None):
    """Advance the GPU simulation s and the oracle o one step at a time and
    compare their Monte Carlo event by event (Sec. IV, Method I in the
    optical-depth form).

    Both sides draw from the same Philox stream, so they take the same
    decisions except where the optical depth ends a step within the band the
    two sides' rate difference explains.  The GPU evaluates W from tables
    (FP32 chi and rate in the FP32 form), the oracle by quadrature: a
    relative difference of at most `delta` (emission) or `delta_pair` (pair
    creation) at equal chi.  A particle whose energy differs between the two
    sides by the relative amount e (from the sampled fractions of earlier
    events) also sees its rate differ by about e times d ln W / d ln energy:
    at most 1 for leptons (W ~ G(chi)/gamma with chi ~ gamma), 2 + 8/(3 chi)
    for photons (G_pair ~ exp(-8/(3 chi)) at small chi; photon_chi(k) gives
    chi).  Per particle and step, with D the oracle's decrement of the step:
      * same decision, no event: |tau_gpu - tau_oracle| <= the band,
        accumulated since the last event as the sum of (delta + c e) D;
      * same decision, event: both restart tau from the same draw
        (-ln r, equal to a few ulp);
      * different decisions (a flip): the side without the event must have
        been left with 0 < tau <= |tau_gpu - tau_oracle| before the step +
        2 (delta + c e) D; the particle is then no longer compared (its
        histories differ from here on).
    Photons of common events must carry the same energy within energy_tol
    relative.  After an event both sides restart tau from the same draw, and
    children start from their identity's draw: -ln r in FP64 on the oracle,
    in FP32 in the FP32 form (within reset_tol
    of the oracle's relative to max(1, tau): 5e-7 there, 1e-12 in FP64; the
    band of the following steps starts from that difference).  Photon
    conversions (pair creation) are classified the same way, a conversion
    seen as the photon dying.  Returns a summary dict."""
    ulp = 1e-12
    if reset_tol is None:
        reset_tol = 5e-7 if getattr(s, "precision", 1) == 0 else ulp
    out = {"events": 0, "conversions": 0, "flips": 0, "checked_tau": 0, "max_rel_energy": 0.0,
           "energies": 0, "max_band_use": 0.0}
    band = {}         # id -> accumulated allowed |tau_gpu - tau_oracle| since the last event
    lost = set()      # ids no longer compared (after a flip, and their children)
    gone = set()      # photons that converted on both sides

    def energy_map(ids, p, photon):
        uu = p["ux"] ** 2 + p["uy"] ** 2 + p["uz"] ** 2
        e = np.sqrt(uu) if photon else np.sqrt(1.0 + uu)
        return dict(zip(ids.tolist(), e.tolist()))

    prev = {}
    for sp in (e_sp, pos_sp, ph_sp):
        gi, gt, _ = _state_gpu(s, sp)
        oi, ot, _ = _state_oracle(o, sp)
        assert set(gi.tolist()) == set(oi.tolist())
        om = dict(zip(oi.tolist(), ot.tolist()))
        for i, t in zip(gi.tolist(), gt.tolist()):
            # identical initial draws (Philox on both sides, -ln r within ulps)
            assert abs(t - om[i]) <= ulp * max(1.0, abs(t)), (i, t, om[i])
        prev[sp] = (dict(zip(gi.tolist(), gt.tolist())), om)
    seen_ph = set()
    for step in range(steps):
        k0 = o.step_count
        s.pic_step(1)
        o.step(1)
        cur, eg, eo, kvec = {}, {}, {}, {}
        for sp in (e_sp, pos_sp, ph_sp):
            gi, gt, gp = _state_gpu(s, sp)
            oi, ot, op = _state_oracle(o, sp)
            cur[sp] = (dict(zip(gi.tolist(), gt.tolist())), dict(zip(oi.tolist(), ot.tolist())))
            eg[sp] = energy_map(gi, gp, sp == ph_sp)
            eo[sp] = energy_map(oi, op, sp == ph_sp)
            if sp == ph_sp:
                galive = dict(zip(gi.tolist(), gp["alive"].tolist()))
                oalive = dict(zip(oi.tolist(), op["alive"].tolist()))
                kvec = dict(zip(oi.tolist(), zip(op["ux"].tolist(), op["uy"].tolist(), op["uz"].tolist())))
        gnew = set(cur[ph_sp][0].keys()) - seen_ph
        onew = set(cur[ph_sp][1].keys()) - seen_ph
        for sp in (e_sp, pos_sp, ph_sp):
            g0, o0 = prev[sp]
            g1, o1 = cur[sp]
            for i in g0.keys() & o0.keys():
                if i in lost or i not in g1 or i not in o1:
                    continue
                if sp == ph_sp:
                    if i in gone:
                        continue  # converted on both sides in an earlier step
                    ev_g, ev_o = not galive[i], not oalive[i]
                    chi = photon_chi(*kvec[i])
                    c = 2.0 + 8.0 / (3.0 * max(chi, 1e-300))
                    dl = delta_pair
                else:
                    ch = child_id(i, k0, 0)
                    ev_g, ev_o = ch in gnew, ch in onew
                    c = 1.0
                    dl = delta
                e_rel = abs(eg[sp][i] / eo[sp][i] - 1.0)
                if ev_g == ev_o:
                    if not ev_g:
                        d_o = o0[i] - o1[i]
                        band[i] = band.get(i, 0.0) + (dl + c * e_rel) * abs(d_o)
                        assert abs(g1[i] - o1[i]) <= band[i] + ulp, (sp, i, step, g1[i], o1[i], band[i], e_rel)
                        out["checked_tau"] += 1
                    elif sp == ph_sp:
                        out["conversions"] += 1
                        gone.add(i)
                    else:
                        out["events"] += 1
                        band[i] = reset_tol * max(1.0, o1[i])
                        assert abs(g1[i] - o1[i]) <= reset_tol * max(1.0, o1[i]), (sp, i, step, g1[i], o1[i])
                        ch = child_id(i, k0, 0)
                        if ch in eg[ph_sp] and ch in eo[ph_sp]:
                            r = abs(eg[ph_sp][ch] / eo[ph_sp][ch] - 1.0)
                            out["max_rel_energy"] = max(out["max_rel_energy"], r)
                            out["energies"] += 1
                            assert r <= energy_tol, (i, step, eg[ph_sp][ch], eo[ph_sp][ch])
                else:
                    # flip: the side that did not take the event kept tau > 0
                    left = o1[i] if ev_g else g1[i]
                    d = (o0[i] - o1[i]) if ev_g else (g0[i] - g1[i])
                    lim = abs(g0[i] - o0[i]) + 2.0 * (dl + c * e_rel) * abs(d) + ulp
                    assert 0.0 < left <= lim, (sp, i, step, ev_g, ev_o, left, lim)
                    out["max_band_use"] = max(out["max_band_use"], left / lim)
                    out["flips"] += 1
                    lost.add(i)
                    if sp != ph_sp:
                        lost.add(child_id(i, k0, 0))
        # children of compared parents start their own comparison
        for sp in (e_sp, pos_sp, ph_sp):
            g1, o1 = cur[sp]
            for i in (g1.keys() & o1.keys()) - prev[sp][0].keys():
                if i in lost:
                    continue
                assert abs(g1[i] - o1[i]) <= reset_tol * max(1.0, o1[i]), (sp, i, g1[i], o1[i])
                band[i] = reset_tol * max(1.0, o1[i])  # the band starts from that difference
        seen_ph |= gnew | onew
        prev = cur
    return out


# ----------------------------------------------------------------------
# observables of the QED field sample (workloads.qed_field_sample), the same
# for a GPU simulation and the oracle: energy history of the emitters,
# photon count, energy and spectrum, pair count
# ----------------------------------------------------------------------

SPECTRUM_EDGES = np.logspace(np.log10(2.0), np.log10(3000.0), 25)  # photon energy, m c^2


def sample_observables(parts, lost):
    """parts: particle dicts of (electrons, positrons, photons); lost: energy
    of photons below photon_emin (tally)"""
    def alive(p):
        return p["alive"] == 1

    e, po, ph = parts
    ge = np.sqrt(1.0 + e["ux"] ** 2 + e["uy"] ** 2 + e["uz"] ** 2)[alive(e)]
    gp = np.sqrt(1.0 + po["ux"] ** 2 + po["uy"] ** 2 + po["uz"] ** 2)[alive(po)] if len(po["ux"]) else np.zeros(0)
    k = np.sqrt(ph["ux"] ** 2 + ph["uy"] ** 2 + ph["uz"] ** 2)[alive(ph)] if len(ph["ux"]) else np.zeros(0)
    return {"electron_energy": float(ge.sum()), "electrons": int(len(ge)), "positrons": int(len(gp)),
            "positron_energy": float(gp.sum()), "photons": int(len(k)), "photon_energy": float(k.sum()),
            "photon_lost": float(lost), "spectrum": np.histogram(k, SPECTRUM_EDGES)[0].astype(int).tolist()}


def combine_observables(parts):
    """sum of the observables of independent chunks of one sample"""
    out = {}
    for k in parts[0]:
        if k == "spectrum":
            out[k] = np.sum([p[k] for p in parts], axis=0).astype(int).tolist()
        else:
            out[k] = sum(p[k] for p in parts)
    return out


def sample_errors(form, ref):
    """errors of one form's observables against the oracle's: relative
    differences of the totals, the worst relative difference of the emitters'
    energy history, and the two-sample chi-square of the photon spectra per
    compared bin (about 1 for spectra that agree within Monte-Carlo noise)"""
    hist_f, hist_o = np.array(form["history"]), np.array(ref["history"])
    a, b = np.array(form["final"]["spectrum"], dtype=float), np.array(ref["final"]["spectrum"], dtype=float)
    use = (a + b) >= 20
    chi2 = float(np.sum((a[use] - b[use]) ** 2 / (a[use] + b[use])) / max(use.sum(), 1))
    f, r = form["final"], ref["final"]
    rel = lambda x, y: abs(x / y - 1.0) if y else (0.0 if not x else float("inf"))
    return {"electron_energy_history_max_rel": float(np.max(np.abs(hist_f - hist_o)) / hist_o[0]),
            "photon_count_rel": rel(f["photons"], r["photons"]),
            "photon_energy_rel": rel(f["photon_energy"], r["photon_energy"]),
            "sub_threshold_photon_energy_rel": rel(f["photon_lost"], r["photon_lost"]),
            "pairs": [f["positrons"], r["positrons"]],
            "spectrum_chi2_per_bin": chi2, "spectrum_bins": int(use.sum())}
