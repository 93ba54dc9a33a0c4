"""Parity at the full sizes of the throughput workloads, in the launch
configuration the bench times (FP32 cell+offset, tiled push, the bench's
sort interval, so the first step sorts): one step of the whole workload on
the GPU, against outputs the oracle computes one by one.

The particles are loaded in the sort's order (numpy's stable argsort of the
key (tile, cell within the tile) of the cell the O6 rule gives), so the
GPU's stable sort at the first step must leave them in place.  Smooth random fields are set on both sides.  The
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
    """the sort key: tile index (x fastest), then the cell within the tile
    (x fastest)"""
    tl = [int(np.log2(w.tile[d])) for d in range(w.dim)]
    nt = [w.n[d] // w.tile[d] for d in range(w.dim)]
    k = np.zeros_like(cells[0])
    for d in reversed(range(w.dim)):
        k = k * nt[d] + (cells[d] >> tl[d])
    loc = np.zeros_like(cells[0])
    for d in reversed(range(w.dim)):
        loc = loc * w.tile[d] + (cells[d] & (w.tile[d] - 1))
    return k * int(np.prod([w.tile[d] for d in range(w.dim)])) + loc


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


B_QED = 3000.0  # chi ~ 15 for the 1 GeV beam: most sampled electrons emit in one step


@pytest.fixture(scope="module")
def qed_collision_sample():
    """the 10^7-electron beam of the QED collision workload in a strong,
    smooth B_z; the oracle steps 300 of its electrons (with their full-load
    identities, hence the same Philox streams) once"""
    w = W.qed_collision_2d()
    rng = np.random.default_rng(21)
    e = w.species[0]
    idx = np.sort(rng.choice(e.n, size=300, replace=False))
    nz, ny, nx = 1, w.n[1], w.n[0] + 1
    yy = np.arange(ny)[:, None] / ny
    xx = np.arange(nx)[None, :] / nx
    bz = B_QED * (1.0 + 0.1 * np.sin(2 * np.pi * (xx + 2 * yy)))[None, :, :]
    sub = W.Workload(w.name, w.dim, w.n, w.dx, w.dt, w.bc,
                     [_take(e, idx)] + [W.Species(s.name, s.q, s.m, s.w, s.x, s.y, s.z, s.ux, s.uy, s.uz,
                                                  capacity=4 * len(idx), kind=s.kind, qed=s.qed)
                                        for s in w.species[1:]],
                     1, laser=w.laser, tile=w.tile, qed=w.qed)
    sub.species[0].qed = 1
    sub.species[0].capacity = 4 * len(idx)
    o = oracle_from_workload(sub, sort_interval=0, seed=SEED_QED)
    o.set_ids(0, idx.astype(np.uint64))
    o.set_field(O.BZ, bz)
    tau0 = o.qed_state(0)[1].copy()
    o.step(1)
    return w, idx, bz, o, tau0


SEED_QED = 0x5EED0001


@pytest.mark.parametrize("prec", [pic.FP32_CELLOFF, pic.FP64_PLAIN])
def test_qed_collision_2d_full_size_events(prec, qed_collision_sample):
    """The whole beam steps once on the GPU (tables, the bench's sort
    interval, so the first step sorts): for the 300 sampled electrons the
    emission events are the oracle's (photon identities derived from the
    parent's Philox stream; a decision may differ only where the optical
    depth ended the step within the table-vs-quadrature rate difference of
    zero), with the oracle's photon energies (1e-3), and the non-emitters'
    optical depths (the rate difference) and momenta agree."""
    w, idx, bz, o, tau0 = qed_collision_sample
    sim = pic.from_workload(w, precision=prec, sort_interval=8, seed=SEED_QED)
    sim.pic_set_field(pic.BZ, bz)
    sim.pic_step(1)
    iph = w.qed["photon_sp"]
    key = np.array([SEED_QED & 0xFFFFFFFF, SEED_QED >> 32], dtype=np.uint32)

    def draw(pid):  # the parent's emission draw of step 0: photon identity, restarted depth
        r = O.philox4x32_10(np.array([pid & 0xFFFFFFFF, pid >> 32, 0, 0], dtype=np.uint32), key)
        return (int(r[3]) << 32) | int(r[2]), -np.log(O.uniform24(int(r[1])))

    gid, gtau = sim.pic_get_qed_state(0)
    ge = sim.pic_get_particles(0)
    where = {int(v): k for k, v in enumerate(gid.tolist())}
    gpos = np.array([where[int(i)] for i in idx])
    oid, otau = o.qed_state(0)
    assert np.array_equal(oid, idx.astype(np.uint64))
    oe = o.particles(0)
    gph_id, _ = sim.pic_get_qed_state(iph)
    oph_id, _ = o.qed_state(iph)
    gph, oph = set(gph_id.tolist()), set(oph_id.tolist())
    cand, restart = zip(*[draw(int(i)) for i in idx])
    restart = np.array(restart)
    # an event (kept photon or one below photon_emin) restarts the optical
    # depth from -ln r (the FP32 form takes the logarithm in FP32: 5e-7)
    rtol = 1e-12 if prec == pic.FP64_PLAIN else 5e-7
    g_ev = np.abs(gtau[gpos] - restart) <= rtol * np.maximum(restart, 1.0)
    o_ev = np.abs(otau - restart) <= 1e-12 * restart
    assert o_ev.sum() >= 60, (g_ev.sum(), o_ev.sum())
    # decisions differ only where the depth ended the step within the band the
    # rate difference explains (tables vs quadrature, FP32 chi and rate)
    delta = 3e-5 if prec == pic.FP64_PLAIN else 5e-5
    for k in np.nonzero(g_ev != o_ev)[0]:
        left, dec = (otau[k], tau0[k] - otau[k]) if g_ev[k] else (gtau[gpos][k], tau0[k] - gtau[gpos][k])
        assert 0.0 < left <= 2.0 * delta * dec + 1e-12, (k, g_ev[k], left, dec)
    g_em = np.array([c in gph for c in cand])
    o_em = np.array([c in oph for c in cand])
    assert np.all(o_em <= o_ev) and np.all(g_em <= g_ev)
    assert o_em.sum() >= 30 and np.all((g_em != o_em) <= (g_ev != o_ev)), (g_em.sum(), o_em.sum())
    # photon energies of the common events
    gk, ok = sim.pic_get_particles(iph), o.particles(iph)
    gmap = dict(zip(gph_id.tolist(), np.sqrt(gk["ux"] ** 2 + gk["uy"] ** 2 + gk["uz"] ** 2).tolist()))
    omap = dict(zip(oph_id.tolist(), np.sqrt(ok["ux"] ** 2 + ok["uy"] ** 2 + ok["uz"] ** 2).tolist()))
    both = [c for c, a, b in zip(cand, g_em, o_em) if a and b]
    rel = np.array([abs(gmap[c] / omap[c] - 1.0) for c in both])
    assert np.max(rel) <= 1e-3, np.max(rel)
    # electrons without an event on either side: momenta and depth decrements
    quiet = (~g_ev) & (~o_ev)
    assert quiet.sum() >= 10
    q = np.nonzero(quiet)[0]
    umag = np.sqrt(oe["ux"] ** 2 + oe["uy"] ** 2 + oe["uz"] ** 2)
    tol = 1e-10 if prec == pic.FP64_PLAIN else TOL
    for k in ("ux", "uy", "uz"):
        assert np.all(np.abs(ge[k][gpos][q] - oe[k][q]) <= tol * umag[q] + 1e-7), k
    dg, do = tau0[q] - gtau[gpos][q], tau0[q] - otau[q]
    assert np.all(np.abs(dg - do) <= delta * do), np.max(np.abs(dg - do) / do)
    sim.close()
