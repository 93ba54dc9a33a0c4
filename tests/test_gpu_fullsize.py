"""Parity at the full sizes of the throughput workloads, in the launch
configuration the bench times (FP32 cell+offset, tiled push, the bench's
sort interval, so the first step sorts): one step of the whole workload on
the GPU, against outputs the oracle computes one by one.

The particles are loaded ordered by tile (numpy's stable argsort of the tile
of the cell the O6 rule gives), so the GPU's stable sort at the first step
must leave them in place.  Smooth random fields are set on both sides.  The
oracle then steps, on the same grid and fields, a sample of the particles:
about 2000 at random, plus every particle whose deposit window can reach one
of a few sampled nodes.  A particle's push depends only on the fields and
its own state, so the sampled particles' new states must match the GPU's
(tolerances of the one-step parity tests); the current at the sampled nodes
sums every particle that reaches them, so it must match too."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_00642_gb300 import pic, workloads as W
from tests.helpers import boundary_ambiguous, oracle_from_workload

pytestmark = pytest.mark.gpu

TOL = 1e-5
KEYS = ("x", "y", "z")


def _cells(w, s):
    """integer cells as the FP32 load forms them (Sec. II cell + offset): the
    offset rounded to FP32, a rounded 1.0 moving to the next cell"""
    out = []
    for d in range(w.dim):
        X = getattr(s, KEYS[d]) / w.dx[d]
        c = np.floor(X)
        up = (X - c).astype(np.float32) >= np.float32(1.0)
        c = c.astype(np.int64) + up
        if w.bc[d] == W.PERIODIC:
            c %= w.n[d]
        else:
            c = np.minimum(c, w.n[d] - 1)
        out.append(c)
    return out


def _tile_keys(w, cells):
    tl = [int(np.log2(w.tile[d])) for d in range(w.dim)]
    nt = [w.n[d] // w.tile[d] for d in range(w.dim)]
    k = np.zeros_like(cells[0])
    for d in reversed(range(w.dim)):
        k = k * nt[d] + (cells[d] >> tl[d])
    return k


def _smooth_fields(shape, rng, amp=(0.6, 0.6, 0.6, 0.4, 0.4, 0.4)):
    """six components, each a sum of three separable low Fourier modes"""
    nz, ny, nx = shape
    ax = [np.arange(m, dtype=np.float64) for m in (nx, ny, nz)]
    F = []
    for c in range(6):
        f = np.zeros(shape)
        for _ in range(3):
            k = rng.integers(1, 4, 3)
            ph = rng.uniform(0, 2 * np.pi, 3)
            fx = np.sin(2 * np.pi * k[0] * ax[0] / max(nx, 1) + ph[0])
            fy = np.cos(2 * np.pi * k[1] * ax[1] / max(ny, 1) + ph[1]) if ny > 1 else np.ones(1)
            fz = np.cos(2 * np.pi * k[2] * ax[2] / max(nz, 1) + ph[2]) if nz > 1 else np.ones(1)
            f += rng.uniform(0.3, 1.0) * fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
        F.append(amp[c] * f / 3.0)
    return F


def _take(s, idx):
    return W.Species(s.name, s.q, s.m, s.w, s.x[idx], s.y[idx], s.z[idx], s.ux[idx], s.uy[idx], s.uz[idx],
                     capacity=max(len(idx), 1))


def _run(w, seed, sort_interval, n_random=2000, n_nodes=6):
    rng = np.random.default_rng(seed)
    # 1. particles ordered by tile, as the sort must leave them
    cells = []
    for i, s in enumerate(w.species):
        c = _cells(w, s)
        order = np.argsort(_tile_keys(w, c), kind="stable")
        w.species[i] = _take(s, order)
        w.species[i].capacity = s.capacity
        cells.append([a[order] for a in c])
    sim = pic.from_workload(w, precision=pic.FP32_CELLOFF, sort_interval=sort_interval)
    box = sim.box()
    F = _smooth_fields(box, rng)
    for c in range(6):
        sim.pic_set_field(c, F[c])
    sim.pic_step(1)
    # 2. the sample: random particles, and every particle that can reach a sampled node
    nodes = []
    for _ in range(n_nodes):
        s0 = w.species[0]
        p = rng.integers(0, s0.n)
        nodes.append([int(cells[0][d][p]) for d in range(w.dim)])
    picks = []
    for i, s in enumerate(w.species):
        sel = np.zeros(s.n, dtype=bool)
        sel[rng.choice(s.n, size=min(n_random, s.n), replace=False)] = True
        for nd in nodes:
            near = np.ones(s.n, dtype=bool)
            for d in range(w.dim):
                dd = cells[i][d] - nd[d]
                if w.bc[d] == W.PERIODIC:
                    dd = (dd + w.n[d] // 2) % w.n[d] - w.n[d] // 2
                near &= np.abs(dd) <= 4
            sel |= near
        picks.append(np.nonzero(sel)[0])
    sub = W.Workload(w.name, w.dim, w.n, w.dx, w.dt, w.bc, [_take(s, picks[i]) for i, s in enumerate(w.species)],
                     1, rho_bg=w.rho_bg, laser=w.laser, tile=w.tile)
    o = oracle_from_workload(sub, sort_interval=0)
    for c in range(6):
        o.set_field(c, F[c])
    o.step(1)
    # 3. particles: new states of the sample
    namb = 0
    for i, s in enumerate(w.species):
        g = sim.pic_get_particles(i)
        po = o.particles(i)
        idx = picks[i]
        assert sim.pic_particle_count(i) == s.n
        for d in range(w.dim):
            assert np.max(np.abs(g[KEYS[d]][idx] - po[KEYS[d]])) <= 10 * TOL * w.dx[d], (s.name, d)
        umag = np.sqrt(po["ux"] ** 2 + po["uy"] ** 2 + po["uz"] ** 2)
        for k in ("ux", "uy", "uz"):
            assert np.all(np.abs(g[k][idx] - po[k]) <= TOL * umag + 1e-7), (s.name, k)
        cg, bits = sim.pic_get_cells(i)
        for d in range(w.dim):
            ref = np.floor(po[KEYS[d]] / w.dx[d]).astype(np.int64) % w.n[d]
            got = (cg[idx].astype(np.int64) >> sum(bits[:d])) & ((1 << bits[d]) - 1)
            a = boundary_ambiguous(po[KEYS[d]], w.dx[d])
            namb += int(a.sum())
            assert np.array_equal(got[~a], ref[~a]), (s.name, d)
    assert namb <= max(3, 1e-3 * sum(len(p) for p in picks))
    # 4. current at the sampled nodes (all contributing particles are in the sample)
    for c, ax in ((pic.JX, 0), (pic.JY, 1), (pic.JZ, 2)):
        jg, jo = sim.pic_fields(c), o.field(c)
        for nd in nodes:
            ijk = tuple(reversed(nd + [0] * (3 - w.dim)))
            cnt = 0.0
            for i, s in enumerate(w.species):
                near = np.ones(s.n, dtype=bool)
                for d in range(w.dim):
                    dd = cells[i][d] - nd[d]
                    if w.bc[d] == W.PERIODIC:
                        dd = (dd + w.n[d] // 2) % w.n[d] - w.n[d] // 2
                    near &= np.abs(dd) <= 3
                f = abs(s.q * s.w) * (w.dx[ax] / w.dt if ax < w.dim else 1.0)
                cnt += f * near.sum()
            assert abs(jg[ijk] - jo[ijk]) <= TOL * cnt + 1e-30, (c, nd, jg[ijk], jo[ijk], cnt)
        assert np.any(jo[tuple(zip(*[tuple(reversed(nd + [0] * (3 - w.dim))) for nd in nodes]))] != 0.0)
    sim.close()


def test_laser_foil_2d_full_size_one_step():
    """2048 x 1024 cells, 4,194,304 electrons and protons (the bench's default workload)"""
    _run(W.laser_foil_2d(), seed=11, sort_interval=16)


def test_thermal_3d_full_size_one_step():
    """256^3 cells, 134,217,728 electrons at 8 per cell (the 3D throughput workload)"""
    _run(W.thermal_3d(), seed=12, sort_interval=4, n_random=1000, n_nodes=4)
