"""The domain decomposition's host logic (paper_2104_00642_gb300.decomp, the
slabs of Sec. II.F) on CPU ranks: 1 to 5 gloo ranks, each stepping an oracle
sub-domain (bc SLAB along x: ghost layers filled by the exchanges, particles
leaving the slab handed to the neighbour), against one oracle on the whole
periodic grid.  The decomposed run must give the same fields and the same
particles (matched by identity) to round-off: only the order of the
current's summation differs.  No GPU."""
import os
import socket

import numpy as np
import pytest

from paper_2104_00642_gb300 import decomp as D

N, DX, NPPC, STEPS = (30, 8), (0.1, 0.12), 6, 40
G = 4


def _setup():
    """the global state: a 2D periodic plasma with hot electrons and ions
    (|u| up to 0.6, so particles cross slab faces) and smooth random fields"""
    rng = np.random.default_rng(2104)
    dt = 0.9 / np.sqrt(1 / DX[0] ** 2 + 1 / DX[1] ** 2)
    L = (N[0] * DX[0], N[1] * DX[1])
    n = N[0] * N[1] * NPPC
    species = []
    for q, m, umax in ((-1.0, 1.0, 0.6), (1.0, 1836.0, 0.02)):
        x = rng.uniform(0.0, L[0], n)
        y = rng.uniform(0.0, L[1], n)
        u = rng.uniform(-umax, umax, (n, 3))
        species.append((q, m, x, y, u))
    yy, xx = np.meshgrid(np.arange(N[1]), np.arange(N[0]), indexing="ij")
    F = []
    for c in range(6):
        a = rng.uniform(0.2, 0.5)
        kx, ky = rng.integers(1, 3, 2)
        F.append(a * np.sin(2 * np.pi * kx * xx / N[0] + rng.uniform(0, 6)) *
                 np.cos(2 * np.pi * ky * yy / N[1] + rng.uniform(0, 6)))
    return dt, species, F


class OracleSlab:
    """the engine interface of decomp over an oracle sub-domain (SLAB x)"""

    def __init__(self, o):
        self.o = o

    def phase(self, k):
        self.o.step_phase(k)

    def layers(self, c, lo, hi):
        return self.o.field_raw(c)[..., lo + G:hi + G].copy()

    def set_layers(self, c, lo, a):
        f = self.o.field_raw(c)
        f[..., lo + G:lo + G + a.shape[-1]] = a
        self.o.set_field_raw(c, f)

    def add_layers(self, c, lo, a):
        f = self.o.field_raw(c)
        f[..., lo + G:lo + G + a.shape[-1]] += a
        self.o.set_field_raw(c, f)

    def take_leaving(self, isp):
        x, u, ids, tau = self.o.take_outbox(isp)
        return {"x": x, "u": u, "id": ids, "tau": tau}

    def insert(self, isp, p):
        self.o.load_state(isp, p["x"], p["u"], p["id"], p["tau"])


def _state(o, nsp, x_off):
    out = []
    for isp in range(nsp):
        ids, _ = o.qed_state(isp)
        p = o.particles(isp)
        a = p["alive"] == 1
        out.append({"id": ids[a], "x": p["x"][a] + x_off, "y": p["y"][a],
                    "u": np.stack([p["ux"][a], p["uy"][a], p["uz"][a]], axis=1)})
    return out


# the QED case: ultra-relativistic electrons gyrating in a uniform B_z
# (chi ~ 5 at gamma 2000, gyro-radius about 20 cells), emitting photons that
# convert to pairs (Sec. IV, Method I); tiny weights, so the fields stay the
# applied B_z up to round-off.  Emitters, photons and pairs cross slab faces,
# also in the step of their events.
QED_SEED = 0x5EED0F4
QED_B0, QED_GAMMA, QED_N, QED_W, QED_STEPS = 1000.0, 2000.0, 24, 1e-12, 30


def _setup_qed():
    rng = np.random.default_rng(2105)
    dt = 0.9 / np.sqrt(1 / DX[0] ** 2 + 1 / DX[1] ** 2)
    L = (N[0] * DX[0], N[1] * DX[1])
    x = rng.uniform(0.0, L[0], QED_N)
    y = rng.uniform(0.0, L[1], QED_N)
    phi = rng.uniform(0.0, 2 * np.pi, QED_N)
    um = np.sqrt(QED_GAMMA ** 2 - 1.0)
    u = np.stack([um * np.cos(phi), um * np.sin(phi), np.zeros(QED_N)], axis=1)
    tau = rng.exponential(size=QED_N)
    F = [np.zeros((N[1], N[0])) for _ in range(6)]
    F[5][:] = QED_B0
    # (q, m, w, kind, qed, x, y, u, tau): electrons, positrons, photons
    empty = (np.zeros(0), np.zeros(0), np.zeros((0, 3)), np.zeros(0))
    species = [(-1.0, 1.0, QED_W, 0, 1, x, y, u, tau), (1.0, 1.0, QED_W, 0, 1) + empty,
               (0.0, 0.0, QED_W, 1, 0) + empty]
    return dt, species, F


def _build(O, shape, bc, dt, species, cap, sel_fn, x_off):
    o = O.OracleSim(2, shape, DX, dt, bc=bc)
    for isp, sp in enumerate(species):
        q, m, w = sp[:3]
        if len(sp) == 5:  # (q, m, x, y, u): the plasma case
            kind, qed, x, y, u = 0, 0, sp[2], sp[3], sp[4]
            w = 0.01
            tau = np.zeros(len(x))
        else:
            kind, qed, x, y, u, tau = sp[3], sp[4], sp[5], sp[6], sp[7], sp[8]
        o.add_species(q, m, w, cap, kind=kind, qed=qed)
        ids = np.arange(len(x), dtype=np.uint64) + np.uint64(isp << 40)
        sel = sel_fn(x)
        xyz = np.stack([x[sel] - x_off, y[sel], np.zeros(sel.sum())], axis=1)
        o.load_state(isp, xyz, u[sel], ids[sel], tau[sel])
    if len(species[0]) > 5:
        o.set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=1e-6, photon_emin=0.0, seed=QED_SEED)
    return o


def _rank_main(rank, world, port, result_path, case="plasma"):
    import torch.distributed as dist
    from oracle import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dt, species, F = _setup() if case == "plasma" else _setup_qed()
        dec = D.SlabDecomposition(N[0], DX[0], ghost=G, dist=dist)
        cap = 4 * N[0] * N[1] * NPPC if case == "plasma" else 200_000  # (slots of migrated particles stay)
        o = _build(O, (dec.n, N[1]), (O.SLAB, O.PERIODIC), dt, species, cap,
                   lambda x: (x >= dec.x0 * DX[0]) & (x < dec.x1 * DX[0]), dec.x0 * DX[0])
        eng = OracleSlab(o)
        for c in range(6):
            o.set_field(c, F[c][:, dec.x0:dec.x1][None])
        dec.start(eng)
        steps = STEPS if case == "plasma" else QED_STEPS
        for _ in range(steps):
            dec.step(eng, len(species))
        # everything to rank 0
        mine = {"fields": [o.field(c)[0] for c in range(9)], "parts": _state(o, len(species), dec.x0 * DX[0]),
                "x0": dec.x0, "x1": dec.x1}
        got = [None] * world
        dist.all_gather_object(got, mine)
        if rank == 0:
            ref = _build(O, N, (O.PERIODIC, O.PERIODIC), dt, species, cap, lambda x: np.ones(len(x), bool), 0.0)
            for c in range(6):
                ref.set_field(c, F[c][None])
            ref.step(steps)
            worst_f, worst_x, worst_u, moved, counts = 0.0, 0.0, 0.0, 0, []
            for c in range(9):
                whole = np.concatenate([g["fields"][c] for g in sorted(got, key=lambda t: t["x0"])], axis=1)
                r = ref.field(c)[0]
                worst_f = max(worst_f, float(np.max(np.abs(whole - r)) / max(np.max(np.abs(r)), 1e-300)))
            rs = _state(ref, len(species), 0.0)
            for isp in range(len(species)):
                ids = np.concatenate([g["parts"][isp]["id"] for g in got])
                assert len(ids) == len(rs[isp]["id"]) and len(np.unique(ids)) == len(ids)
                order, rorder = np.argsort(ids), np.argsort(rs[isp]["id"])
                assert np.array_equal(ids[order], rs[isp]["id"][rorder])
                x = np.concatenate([g["parts"][isp]["x"] for g in got])[order]
                u = np.concatenate([g["parts"][isp]["u"] for g in got])[order]
                Lx = N[0] * DX[0]
                dxp = (x - rs[isp]["x"][rorder] + 0.5 * Lx) % Lx - 0.5 * Lx
                worst_x = max(worst_x, float(np.max(np.abs(dxp))))
                worst_u = max(worst_u, float(np.max(np.abs(u - rs[isp]["u"][rorder]))))
                # particles that ended on another rank than they started on
                # (the plasma case) / particles of each species (the QED case)
                if case == "plasma":
                    x_start = species[isp][2][(ids[order] - np.uint64(isp << 40)).astype(np.int64)]
                    r_start = np.searchsorted([g["x0"] * DX[0] for g in sorted(got, key=lambda t: t["x0"])][1:],
                                              x_start, side="right")
                    r_end = np.searchsorted([g["x0"] * DX[0] for g in sorted(got, key=lambda t: t["x0"])][1:],
                                            x % Lx, side="right")
                    moved += int(np.sum(r_start != r_end))
                else:
                    counts.append(len(ids))
            with open(result_path, "w") as f:
                f.write(f"{worst_f} {worst_x} {worst_u} {moved} {' '.join(str(c) for c in counts)}\n")
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_slab_decomposition_matches_the_whole_grid(world, tmp_path):
    """fields (interiors side by side) within 1e-12 of their largest value,
    particle positions within 1e-12 and momenta within 1e-12 of the
    single-domain oracle after 40 steps; with more than one rank, particles
    did change slabs"""
    import torch.multiprocessing as mp
    out = tmp_path / "result.txt"
    mp.spawn(_rank_main, args=(world, _free_port(), str(out)), nprocs=world, join=True)
    wf, wx, wu, moved = open(out).read().split()
    print(world, wf, wx, wu, moved)
    assert float(wf) < 1e-12 and float(wx) < 1e-12 and float(wu) < 1e-12
    if world > 1:
        assert int(moved) > 50


@pytest.mark.parametrize("world", [3])
def test_slab_decomposition_with_qed_matches_the_whole_grid(world, tmp_path):
    """the QED case: the same electrons, photons and pairs (matched by
    identity: children's identities come from their parents' Philox
    streams) with the same positions and momenta to round-off, after 30
    steps with events in slabs, at slab faces and in the step of a crossing"""
    import torch.multiprocessing as mp
    out = tmp_path / "result.txt"
    mp.spawn(_rank_main, args=(world, _free_port(), str(out), "qed"), nprocs=world, join=True)
    wf, wx, wu, _, *counts = open(out).read().split()
    counts = [int(c) for c in counts]
    print(world, wf, wx, wu, counts)
    assert float(wf) < 1e-12 and float(wx) < 1e-12 and float(wu) < 1e-9
    assert counts[2] > 100 and counts[1] > 3  # photons and pairs were made


def test_slab_bounds_cover_the_grid():
    for n, r in ((30, 1), (30, 4), (31, 5), (64, 8)):
        b = [D.slab_bounds(n, r, k) for k in range(r)]
        assert b[0][0] == 0 and b[-1][1] == n
        assert all(b[k][1] == b[k + 1][0] for k in range(r - 1))
        assert max(x1 - x0 for x0, x1 in b) - min(x1 - x0 for x0, x1 in b) <= 1
    with pytest.raises(ValueError):
        D.SlabDecomposition(3, 0.1, ghost=4)  # narrower than its ghost layers


def _allreduce_main(rank, world, port, result_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dec = D.SlabDecomposition(N[0], DX[0], ghost=G, dist=dist)
        # a diagnostic that each rank holds a part of: the energy of its own
        # cells, here a value whose sum over ranks is known exactly
        got = dec.allreduce_sum([float(dec.n), 0.1 * (rank + 1), 1e-300])
        if rank == 0:
            with open(result_path, "w") as f:
                f.write(" ".join(repr(float(v)) for v in got) + "\n")
    finally:
        dist.destroy_process_group()


def test_allreduce_sums_the_ranks_diagnostics(tmp_path):
    """the global diagnostics of a decomposed run: FP64 sums over the ranks
    (the cells of the slabs add up to the grid)"""
    import torch.multiprocessing as mp
    out = tmp_path / "sum.txt"
    world = 3
    mp.spawn(_allreduce_main, args=(world, _free_port(), str(out)), nprocs=world, join=True)
    cells, tenths, tiny = (float(v) for v in open(out).read().split())
    assert cells == N[0]
    assert abs(tenths - 0.1 * (1 + 2 + 3)) < 1e-15
    assert tiny == 3e-300
