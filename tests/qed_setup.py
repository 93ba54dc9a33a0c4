"""A shared QED test setup: ultra-relativistic electrons gyrating in a
uniform magnetic field B_z on a small periodic 1D grid, with photon emission
and pair creation on.  The particle weight is tiny so that self-fields do not
matter; B does no work, so the total energy of electrons, positrons, photons
and pair rest mass is conserved exactly by the method (collinear emission
with recoil gamma (1 - u), pair energies summing to the photon's)."""
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
