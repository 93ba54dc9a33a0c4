"""Seeded synthetic inputs shaped like the paper's laser-plasma runs.

This module holds no arithmetic of the PIC method itself: it only draws
particle positions and momenta and derives grid sizes and weights from the
workload description.  Both the CUDA path (tests, bench) and the CPU oracle
read their inputs from here, so that they start from identical FP64 states.

All quantities are in the normalised units of Eq. (8) of Song, Wang & Li
(arXiv:2104.00642, Sec. II.A): c = m_e = e = 1, time in 1/omega_r, length in
c/omega_r, density in n_r.  Workloads:

* ``langmuir_1d``: cold Langmuir oscillation, 1D periodic, quiet start, fixed
  ion background (omega_r = omega_p).
* ``laser_foil_2d``: hydrogen slab hit by a linearly polarised Gaussian laser
  entering from x-min; absorbing x, periodic y (omega_r = omega_L).
* ``thermal_3d``: uniform Maxwellian electrons on a neutralising background,
  3D periodic (omega_r = omega_p).
* ``qed_collision_2d``: a GeV electron beam against an a0 = 200 laser, with
  photon emission and pair creation (Sec. IV; omega_r = omega_L).
* ``qed_foil_3d``: a circularly polarised a0 = 300 laser on a 100 n_c
  electron-proton foil in 3D, photon emission and pair creation on
  (Sec. III-IV; omega_r = omega_L).
* ``qed_field_sample``: the collision's QED regime (beam energies, peak chi)
  in a uniform field, small enough for the FP64 oracle.
* ``cascade``: seed replicas of one electron of Lorentz factor gamma0 moving
  across a uniform magnetic field B0 = b B_cr, photon emission and pair
  creation by Method II (Sec. IV: gamma0 = 1000 in 0.001 / 0.009 B_cr for
  the spectra of Fig. 9, gamma0 = 2e5 in 0.2 B_cr for the pair count of
  Fig. 10).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PERIODIC, ABSORB = 0, 1
M_PROTON = 1836.15267343
MEC2_KEV = 510.99895
SEED0 = 20210401
HBARC_EV_M = 1.973269804e-7  # hbar c (eV m)


@dataclass
class Species:
    name: str
    q: float
    m: float
    w: float
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    uz: np.ndarray
    capacity: int = 0
    kind: int = 0  # 0 massive, 1 photon
    qed: int = 0   # 1: takes part in the QED Monte Carlo

    @property
    def n(self) -> int:
        return int(self.ux.shape[0])


@dataclass
class Laser:
    a0: float
    waist: float
    fwhm: float
    t_peak: float
    x_focus: float
    yc: float = 0.0
    zc: float = 0.0
    pol: int = 0  # 0 linear along y, 1 circular


@dataclass
class Workload:
    name: str
    dim: int
    n: tuple
    dx: tuple
    dt: float
    bc: tuple
    species: list
    steps: int
    rho_bg: float = 0.0
    laser: Laser | None = None
    tile: tuple = (8, 8, 8)
    notes: dict = field(default_factory=dict)
    # QED Monte Carlo: species indices, reference wavelength (m), photon_emin
    qed: dict | None = None

    @property
    def n_particles(self) -> int:
        return sum(s.n for s in self.species)

    @property
    def n_cells(self) -> int:
        return int(np.prod(self.n[: self.dim]))


def _rng(seed):
    return np.random.Generator(np.random.Philox(seed))


def maxwell_juttner_u(rng, n, theta):
    """|u| drawn from u^2 exp(-(gamma-1)/theta) by inverse CDF on a fine grid,
    with isotropic direction (input generation only)."""
    umax = math.sqrt((1.0 + 60.0 * theta) ** 2 - 1.0)
    ug = np.linspace(0.0, umax, 200001)
    g = np.sqrt(1.0 + ug * ug)
    pdf = ug * ug * np.exp(-(g - 1.0) / theta)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (pdf[1:] + pdf[:-1]) * np.diff(ug))])
    cdf /= cdf[-1]
    umag = np.interp(rng.random(n), cdf, ug)
    ct = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    st = np.sqrt(1.0 - ct * ct)
    return umag * st * np.cos(ph), umag * st * np.sin(ph), umag * ct


def langmuir_1d(n_cells=256, dx=0.05, ppc=100, amp=0.01, steps=1000, courant=0.95):
    """Cold Langmuir oscillation: quiet start x = (i + (k+1/2)/ppc) dx,
    u_x = amp sin(2 pi x / L), electrons of density 1 on an ion background."""
    L = n_cells * dx
    i = np.repeat(np.arange(n_cells), ppc)
    k = np.tile(np.arange(ppc), n_cells)
    x = (i + (k + 0.5) / ppc) * dx
    ux = amp * np.sin(2.0 * math.pi * x / L)
    z0 = np.zeros_like(x)
    e = Species("electron", -1.0, 1.0, 1.0 / ppc, x, z0.copy(), z0.copy(), ux, z0.copy(), z0.copy(),
                capacity=x.size)
    return Workload("langmuir_1d", 1, (n_cells, 1, 1), (dx, 1.0, 1.0), courant * dx,
                    (PERIODIC, PERIODIC, PERIODIC), [e], steps, rho_bg=1.0, tile=(16, 1, 1),
                    notes={"L": L, "k": 2.0 * math.pi / L, "amp": amp})


def thermal_3d(n=(256, 256, 256), dx=0.1, ppc=8, T_keV=10.0, steps=200, courant=0.95,
               seed=SEED0 + 3, tile=(4, 4, 4)):
    """Uniform Maxwellian electrons (u_i ~ N(0, T/mc^2)) at Philox-uniform
    positions on a neutralising background, periodic in all axes."""
    rng = _rng(seed)
    nc = int(np.prod(n))
    N = nc * ppc
    theta = T_keV / MEC2_KEV
    x = rng.random(N) * (n[0] * dx)
    y = rng.random(N) * (n[1] * dx)
    z = rng.random(N) * (n[2] * dx)
    s = math.sqrt(theta)
    ux, uy, uz = (rng.standard_normal(N) * s for _ in range(3))
    e = Species("electron", -1.0, 1.0, 1.0 / ppc, x, y, z, ux, uy, uz, capacity=N)
    dt = courant * dx / math.sqrt(3.0)
    return Workload("thermal_3d", 3, tuple(n), (dx, dx, dx), dt, (PERIODIC,) * 3, [e], steps,
                    rho_bg=1.0, tile=tile, notes={"theta": theta, "ppc": ppc})


def thermal_2d(n=(256, 256), dx=0.1, ppc=16, T_keV=10.0, steps=100, courant=0.95, seed=SEED0 + 6,
               tile=(16, 16, 1)):
    """2D3V version of ``thermal_3d`` (small parity case)."""
    rng = _rng(seed)
    nc = n[0] * n[1]
    N = nc * ppc
    theta = T_keV / MEC2_KEV
    x = rng.random(N) * (n[0] * dx)
    y = rng.random(N) * (n[1] * dx)
    s = math.sqrt(theta)
    ux, uy, uz = (rng.standard_normal(N) * s for _ in range(3))
    e = Species("electron", -1.0, 1.0, 1.0 / ppc, x, y, np.zeros(N), ux, uy, uz, capacity=N)
    dt = courant * dx / math.sqrt(2.0)
    return Workload("thermal_2d", 2, (n[0], n[1], 1), (dx, dx, 1.0), dt, (PERIODIC,) * 3, [e], steps,
                    rho_bg=1.0, tile=tile, notes={"theta": theta, "ppc": ppc})


def self_heating_2d(n=(128, 128), ppc=16, T_keV=1.0, cells_per_lambda_p=320, steps=4000, courant=0.95,
                    seed=SEED0 + 10, tile=(16, 16, 1)):
    """The self-heating test of Sec. III(b) (Fig. 6): a uniform thermal
    plasma, T = 1 keV, periodic, 320 cells per plasma wavelength (the
    paper's n = 100 n_c sets only the unit: lengths here in c/omega_p, so
    dx = 2 pi / 320 and n = 1); electrons at Philox-uniform positions with
    u ~ N(0, T/mc^2) per component on a fixed neutralising background.  The
    figure reports the relative growth of the total energy against shape
    order and ppc."""
    rng = _rng(seed)
    dx = 2.0 * math.pi / cells_per_lambda_p
    N = n[0] * n[1] * ppc
    theta = T_keV / MEC2_KEV
    x = rng.random(N) * (n[0] * dx)
    y = rng.random(N) * (n[1] * dx)
    s = math.sqrt(theta)
    ux, uy, uz = (rng.standard_normal(N) * s for _ in range(3))
    e = Species("electron", -1.0, 1.0, 1.0 / ppc, x, y, np.zeros(N), ux, uy, uz, capacity=N)
    dt = courant * dx / math.sqrt(2.0)
    return Workload("self_heating_2d", 2, (n[0], n[1], 1), (dx, dx, 1.0), dt, (PERIODIC,) * 3, [e], steps,
                    rho_bg=1.0, tile=tile, notes={"theta": theta, "ppc": ppc, "debye_over_dx": math.sqrt(theta) / dx})


def laser_foil_2d(nx=2048, ny=1024, cells_per_lambda=64, slab=(1024, 1088), n0=10.0, ppc=32,
                  T_keV=1.0, a0=20.0, waist_um=3.0, fwhm_fs=30.0, steps=4000, courant=0.95,
                  seed=SEED0 + 2, tile=(16, 16, 1), x_focus_cell=None):
    """Hydrogen slab n0 n_c over x-cells [slab), all y, ppc electrons and ppc
    protons per cell (Maxwell-Juttner), LP Gaussian laser from x-min.
    Lengths: lambda = 1 um = 2 pi c/omega_L."""
    rng = _rng(seed)
    dx = 2.0 * math.pi / cells_per_lambda
    dt = courant * dx / math.sqrt(2.0)
    theta = T_keV / MEC2_KEV
    sx0, sx1 = slab
    ncell = (sx1 - sx0) * ny
    N = ncell * ppc
    ci = np.repeat(np.arange(ncell), ppc)
    cx = sx0 + ci % (sx1 - sx0)
    cy = ci // (sx1 - sx0)
    species = []
    for name, q, m in (("electron", -1.0, 1.0), ("proton", 1.0, M_PROTON)):
        x = (cx + rng.random(N)) * dx
        y = (cy + rng.random(N)) * dx
        ux, uy, uz = maxwell_juttner_u(rng, N, theta / m)
        species.append(Species(name, q, m, n0 / ppc, x, y, np.zeros(N), ux, uy, uz, capacity=N))
    omega_L = 2.0 * math.pi * 2.99792458e8 / 1.0e-6
    fwhm = fwhm_fs * 1e-15 * omega_L
    waist = waist_um * 2.0 * math.pi
    xf = (sx0 if x_focus_cell is None else x_focus_cell) * dx
    laser = Laser(a0=a0, waist=waist, fwhm=fwhm, t_peak=2.5 * fwhm, x_focus=xf, yc=0.5 * ny * dx)
    return Workload("laser_foil_2d", 2, (nx, ny, 1), (dx, dx, 1.0), dt, (ABSORB, PERIODIC, PERIODIC),
                    species, steps, laser=laser, tile=tile,
                    notes={"theta": theta, "n0": n0, "ppc": ppc, "slab": slab})


def qed_collision_2d(nx=2048, ny=512, cells_per_lambda=32, n_beam=10_000_000, gamma0=1957.0, spread=0.01,
                     sigma_um=1.0, a0=200.0, waist_um=2.0, fwhm_fs=15.0, x_focus_um=6.5, n_peak=0.01,
                     photon_cap=24.0, pair_cap=0.5, photon_emin=2.0, steps=3000, courant=0.95, seed=SEED0 + 7,
                     tile=(16, 16, 1)):
    """Strong-field QED collision (2D3V): a linearly polarised Gaussian laser
    of amplitude a0 enters from x-min and focuses at x_focus; an electron beam
    (Gaussian, sigma in x and y, gamma0 with a relative rms spread, moving
    along -x) is placed so that its centre meets the pulse peak at the focus.
    Species: electrons (beam, QED), positrons (QED), photons.  The beam's
    peak density is n_peak (weight from the macro count); emitted photons
    below photon_emin (m c^2) are tallied, not kept.  Lengths: lambda = 1 um."""
    rng = _rng(seed)
    dx = 2.0 * math.pi / cells_per_lambda
    dt = courant * dx / math.sqrt(2.0)
    lam = 2.0 * math.pi
    sig = sigma_um * lam
    omega_L = 2.0 * math.pi * 2.99792458e8 / 1.0e-6
    fwhm = fwhm_fs * 1e-15 * omega_L
    t_peak = 2.5 * fwhm
    xf = x_focus_um * lam
    yc = 0.5 * ny * dx
    # the pulse peak reaches x_f at t_peak + x_f; the beam centre (speed ~ 1)
    # starts at 2 x_f + t_peak to be there at that time
    xb = 2.0 * xf + t_peak
    x = rng.normal(xb, sig, n_beam)
    y = rng.normal(yc, sig, n_beam)
    x = np.clip(x, 0.5 * dx, (nx - 0.5) * dx)
    y = np.mod(y, ny * dx)
    g = gamma0 * (1.0 + spread * rng.standard_normal(n_beam))
    ux = -np.sqrt(g * g - 1.0)
    zero = np.zeros(n_beam)
    core = n_beam * dx * dx / (2.0 * math.pi * sig * sig)  # macro-particles per cell at the peak
    w = n_peak / core
    e = Species("electron", -1.0, 1.0, w, x, y, zero, ux, zero.copy(), zero.copy(),
                capacity=int(n_beam * (1.0 + pair_cap)), qed=1)
    emp = np.zeros(0)
    npair = int(n_beam * pair_cap)
    po = Species("positron", 1.0, 1.0, w, emp, emp, emp, emp, emp, emp, capacity=max(npair, 1), qed=1)
    ph = Species("photon", 0.0, 0.0, w, emp, emp, emp, emp, emp, emp, capacity=int(n_beam * photon_cap), kind=1)
    laser = Laser(a0=a0, waist=waist_um * lam, fwhm=fwhm, t_peak=t_peak, x_focus=xf, yc=yc)
    t_collide = t_peak + xf
    return Workload("qed_collision_2d", 2, (nx, ny, 1), (dx, dx, 1.0), dt, (ABSORB, PERIODIC, PERIODIC),
                    [e, po, ph], steps, laser=laser, tile=tile,
                    notes={"t_collide": t_collide, "steps_to_collision": int(t_collide / dt), "w": w,
                           "beam_x0": xb, "peak_macros_per_cell": core},
                    qed={"photon_sp": 2, "electron_sp": 0, "positron_sp": 1, "lambda_r_m": 1e-6,
                         "photon_emin": photon_emin})


def qed_foil_3d(n=(1024, 512, 512), cells_per_lambda=32, foil=(512, 576), n0=100.0, ppc=8, T_keV=1.0, a0=300.0,
                waist_um=3.0, fwhm_fs=30.0, t_peak_fwhm=2.5, photon_cap=0.5, pair_cap=0.05, photon_emin=2.0,
                steps=2000, courant=0.95, seed=SEED0 + 8, tile=(4, 4, 4)):
    """3D laser-foil with QED: an electron-proton foil of density n0 n_c over
    x-cells [foil), all y and z, ppc electrons and ppc protons per cell at
    random positions in the cell (Maxwell-Juttner T), a circularly polarised
    Gaussian laser of amplitude a0 per component entering from x-min and
    focused on the foil front, absorbing x, periodic y and z.  Species:
    electrons (QED), protons, positrons (QED, empty), photons (empty);
    capacities for the QED children are fractions of the electron count.
    Lengths: lambda = 1 um = 2 pi c/omega_L."""
    rng = _rng(seed)
    dx = 2.0 * math.pi / cells_per_lambda
    dt = courant * dx / math.sqrt(3.0)
    theta = T_keV / MEC2_KEV
    nx, ny, nz = n
    fx0, fx1 = foil
    fw = fx1 - fx0
    ncell = fw * ny * nz
    N = ncell * ppc
    ci = np.repeat(np.arange(ncell, dtype=np.int64), ppc)
    cx = fx0 + ci % fw
    cy = (ci // fw) % ny
    cz = ci // (fw * ny)
    del ci
    species = []
    for name, q, m, qed in (("electron", -1.0, 1.0, 1), ("proton", 1.0, M_PROTON, 0)):
        x = (cx + rng.random(N)) * dx
        y = (cy + rng.random(N)) * dx
        z = (cz + rng.random(N)) * dx
        ux, uy, uz = maxwell_juttner_u(rng, N, theta / m)
        cap = int(N * (1.0 + pair_cap)) if qed else N
        species.append(Species(name, q, m, n0 / ppc, x, y, z, ux, uy, uz, capacity=cap, qed=qed))
    emp = np.zeros(0)
    w = n0 / ppc
    species.append(Species("positron", 1.0, 1.0, w, emp, emp, emp, emp, emp, emp,
                           capacity=max(int(N * pair_cap), 1), qed=1))
    species.append(Species("photon", 0.0, 0.0, w, emp, emp, emp, emp, emp, emp,
                           capacity=max(int(N * photon_cap), 1), kind=1))
    omega_L = 2.0 * math.pi * 2.99792458e8 / 1.0e-6
    fwhm = fwhm_fs * 1e-15 * omega_L
    lam = 2.0 * math.pi
    laser = Laser(a0=a0, waist=waist_um * lam, fwhm=fwhm, t_peak=t_peak_fwhm * fwhm, x_focus=fx0 * dx,
                  yc=0.5 * ny * dx, zc=0.5 * nz * dx, pol=1)
    t_arrive = laser.t_peak + fx0 * dx
    return Workload("qed_foil_3d", 3, tuple(n), (dx, dx, dx), dt, (ABSORB, PERIODIC, PERIODIC), species, steps,
                    laser=laser, tile=tile,
                    notes={"theta": theta, "n0": n0, "ppc": ppc, "foil": foil, "t_peak_at_foil": t_arrive,
                           "steps_to_peak_at_foil": int(t_arrive / dt)},
                    qed={"photon_sp": 3, "electron_sp": 0, "positron_sp": 2, "lambda_r_m": 1e-6,
                         "photon_emin": photon_emin})


def qed_field_sample(n_e=2048, gamma0=1957.0, spread=0.01, B0=400.0, dt=0.1319, steps=48, seed=SEED0 + 9):
    """The QED regime of ``qed_collision_2d`` in a uniform field, small enough
    for the FP64 oracle: n_e electrons with the beam's energy distribution
    (gamma0 with a relative rms spread) moving in random directions of the
    x-y plane through a uniform B_z = B0 (the caller sets it), which gives
    chi = |u| B0 / E_s ~ 1.9 at gamma0 for lambda_r = 1 um -- the collision's
    peak chi (2 gamma0 a0 hbar omega / m c^2 for a0 = 200); 1D periodic grid
    of 16 cells, the collision's dt, tiny weight (no self-fields).  Species:
    electrons (QED), positrons (QED), photons; photons below 2 m c^2 are
    tallied, as in the collision."""
    rng = _rng(seed)
    g = gamma0 * (1.0 + spread * rng.standard_normal(n_e))
    u = np.sqrt(g * g - 1.0)
    ang = rng.uniform(0.0, 2.0 * math.pi, n_e)
    x = (np.arange(n_e) + rng.random(n_e)) * (16.0 / n_e)
    zero = np.zeros(n_e)
    w = 1e-12
    e = Species("electron", -1.0, 1.0, w, x, zero, zero.copy(), u * np.cos(ang), u * np.sin(ang), zero.copy(),
                capacity=4 * n_e, qed=1)
    emp = np.zeros(0)
    po = Species("positron", 1.0, 1.0, w, emp, emp, emp, emp, emp, emp, capacity=4 * n_e, qed=1)
    ph = Species("photon", 0.0, 0.0, w, emp, emp, emp, emp, emp, emp, capacity=64 * n_e, kind=1)
    return Workload("qed_field_sample", 1, (16, 1, 1), (1.0, 1.0, 1.0), dt, (PERIODIC,) * 3, [e, po, ph], steps,
                    tile=(16, 1, 1), notes={"B0": B0, "gamma0": gamma0},
                    qed={"photon_sp": 2, "electron_sp": 0, "positron_sp": 1, "lambda_r_m": 1e-6, "photon_emin": 2.0})


def b_critical(lambda_r_m=1e-6):
    """the critical field B_cr = m^2 c^2 / (e hbar) in units of m c omega_r / e:
    m c^2 / (hbar omega_r), omega_r = 2 pi c / lambda_r"""
    return MEC2_KEV * 1e3 * lambda_r_m / (2.0 * math.pi * HBARC_EV_M)


def cascade(gamma0=1000.0, b=0.009, replicas=2000, t_end=4.0, dt=None, steps=None, seed=SEED0 + 11,
            lambda_r_m=1e-6, photon_emin=0.0, capacity_per_replica=64):
    """Seed replicas of the single-electron cascade of Sec. IV: each replica
    is one electron of Lorentz factor gamma0 moving along +y across a uniform
    B_z = b B_cr (the caller sets the field, notes["B0"]); chi0 = gamma0 b.
    The replicas share a 16-cell periodic 1D grid at random x, with a tiny
    weight so that they do not interact: every electron's identity starts
    its own Philox stream, so the replicas are independent seeds.  Species:
    electrons (QED), positrons (QED), photons (photons below photon_emin, in
    m c^2, are tallied).  dt defaults to 1 / (8000 b^(2/3)): Method II's
    acceptance per step peaks for leptons near gamma ~ 2, at about
    3400 b^(2/3) dt for lambda_r = 1 um, so this keeps it below one half;
    steps defaults to t_end / dt (t_end in 1/omega_r).
    Paper set-ups: cascade(1000, 0.001), cascade(1000, 0.009) (Fig. 9),
    cascade(2e5, 0.2) (Fig. 10)."""
    rng = _rng(seed)
    B0 = b * b_critical(lambda_r_m)
    chi0 = gamma0 * b
    if dt is None:
        dt = 1.0 / (8000.0 * b ** (2.0 / 3.0)) * (lambda_r_m / 1e-6) ** (2.0 / 3.0)
    if steps is None:
        steps = int(math.ceil(t_end / dt))
    n = int(replicas)
    x = (np.arange(n) + rng.random(n)) * (16.0 / n)
    zero = np.zeros(n)
    u = math.sqrt(gamma0 * gamma0 - 1.0)
    w = 1e-12
    cap = capacity_per_replica * n
    e = Species("electron", -1.0, 1.0, w, x, zero, zero.copy(), zero.copy(), np.full(n, u), zero.copy(),
                capacity=cap, qed=1)
    emp = np.zeros(0)
    po = Species("positron", 1.0, 1.0, w, emp, emp, emp, emp, emp, emp, capacity=cap, qed=1)
    ph = Species("photon", 0.0, 0.0, w, emp, emp, emp, emp, emp, emp, capacity=4 * cap, kind=1)
    return Workload(f"cascade gamma0={gamma0:g} B0={b:g} B_cr", 1, (16, 1, 1), (1.0, 1.0, 1.0), dt,
                    (PERIODIC,) * 3, [e, po, ph], steps, tile=(16, 1, 1),
                    notes={"B0": B0, "gamma0": gamma0, "chi0": chi0, "replicas": n, "t_end": steps * dt},
                    qed={"photon_sp": 2, "electron_sp": 0, "positron_sp": 1, "lambda_r_m": lambda_r_m,
                         "photon_emin": photon_emin})


def vacuum_pulse_1d(n_cells=1024, cells_per_lambda=32, a0=1.0, fwhm=4.0 * 2.0 * math.pi, steps=1500,
                    courant=0.95, pol=0):
    """Laser pulse entering an empty 1D absorbing box (boundary tests)."""
    dx = 2.0 * math.pi / cells_per_lambda
    laser = Laser(a0=a0, waist=1.0, fwhm=fwhm, t_peak=2.5 * fwhm, x_focus=0.0, pol=pol)
    return Workload("vacuum_pulse_1d", 1, (n_cells, 1, 1), (dx, 1.0, 1.0), courant * dx,
                    (ABSORB, PERIODIC, PERIODIC), [], steps, laser=laser, tile=(16, 1, 1))


def random_particles(rng, n, dim, L, umax=0.3):
    """Uniform positions in [0, L_d) and uniform momenta in [-umax, umax]."""
    x = [rng.random(n) * L[d] if d < dim else np.zeros(n) for d in range(3)]
    u = [rng.uniform(-umax, umax, n) for _ in range(3)]
    return x, u
