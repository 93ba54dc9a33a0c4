"""Shared test helpers: build matching oracle / GPU simulations from one
seeded input and compare them with the tolerances of the parity contract."""
from __future__ import annotations

import math

import numpy as np

from oracle import oracle as O
from paper_2104_00642_gb300 import workloads as W


def oracle_from_workload(w: W.Workload, sort_interval=0, tile=None, seed=0):
    """the oracle on a workload's grid, species, laser and (QED workloads)
    Monte Carlo set-up; seed: the Philox key, as the simulation's"""
    t = tile if tile is not None else w.tile
    o = O.OracleSim(w.dim, w.n[: w.dim], w.dx[: w.dim], w.dt, bc=w.bc[: w.dim], rho_bg=w.rho_bg,
                    sort_interval=sort_interval, tile=t[: w.dim])
    for s in w.species:
        o.add_species(s.q, s.m, s.w, s.capacity, kind=s.kind, qed=s.qed)
    if w.qed is not None:  # before the load: the initial optical depths draw from the seed
        o.set_qed(seed=seed, **w.qed)
    for i, s in enumerate(w.species):
        if s.n:
            o.load(i, s.x, s.y if w.dim > 1 else None, s.z if w.dim > 2 else None, s.ux, s.uy, s.uz)
    if w.laser is not None:
        L = w.laser
        o.set_laser(L.a0, L.waist, L.fwhm, L.t_peak, L.x_focus, L.yc, L.zc, L.pol)
    return o


def random_state(dim, n, dx, dt, nppc, seed, umax=0.5, fields=True, bc=None, q=-1.0, m=1.0):
    """random particles and random smooth-ish fields (as a Workload)"""
    rng = np.random.default_rng(seed)
    nn = tuple(list(n) + [1] * (3 - len(n)))
    dd = tuple(list(dx) + [1.0] * (3 - len(dx)))
    N = int(np.prod(nn[:dim])) * nppc
    L = [nn[d] * dd[d] for d in range(3)]
    x, u = W.random_particles(rng, N, dim, L, umax)
    sp = W.Species("e", q, m, 0.1, x[0], x[1], x[2], u[0], u[1], u[2], capacity=N)
    bcs = bc if bc is not None else (W.PERIODIC,) * 3
    w = W.Workload("random", dim, nn, dd, dt, tuple(list(bcs) + [0] * (3 - len(bcs))), [sp], 1,
                   tile=(8, 8, 8) if dim == 3 else ((16, 16, 1) if dim == 2 else (16, 1, 1)))
    F = None
    if fields:
        shape = [1, 1, 1]
        for d in range(dim):
            shape[2 - d] = nn[d] + (1 if w.bc[d] == W.ABSORB else 0)
        F = [rng.uniform(-1.0, 1.0, shape) * (0.3 if c >= 6 else 1.0) for c in range(9)]
    return w, F


def boundary_ambiguous(x, dx, tol=2.0 ** -18):
    """particles whose position lies within tol cells of a cell face"""
    X = x / dx
    f = X - np.floor(X)
    return (f < tol) | (f > 1 - tol)


def window_scale(o_parts, w, dim, comp_axis, reach=3):
    """per-node scale of the summed current terms: |q w| dx_d/dt times the
    number of particles whose deposit window (2 reach + 1 cells around the
    particle's cell; 3 covers the order-2 window) covers the node"""
    s = w.species[0]
    shape = [1, 1, 1]
    for d in range(dim):
        shape[2 - d] = w.n[d] + (1 if w.bc[d] == W.ABSORB else 0)
    cnt = np.zeros(shape)
    keys = ("x", "y", "z")
    idx = []
    for d in range(3):
        if d < dim:
            c = np.floor(o_parts[keys[d]] / w.dx[d]).astype(np.int64)
            idx.append(c)
        else:
            idx.append(np.zeros_like(o_parts["ux"], dtype=np.int64))
    for d0 in range(-reach, reach + 1):
        for d1 in (range(-reach, reach + 1) if dim > 1 else [0]):
            for d2 in (range(-reach, reach + 1) if dim > 2 else [0]):
                ii = np.mod(idx[0] + d0, shape[2])
                jj = np.mod(idx[1] + d1, shape[1])
                kk = np.mod(idx[2] + d2, shape[0])
                np.add.at(cnt, (kk, jj, ii), 1.0)
    f = abs(s.q * s.w) * (w.dx[comp_axis] / w.dt if comp_axis < dim else 1.0)
    return cnt * f


def energy(d):
    return d["U_E"] + d["U_B"] + sum(d["U_kin"])


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


__all__ = ["oracle_from_workload", "random_state", "boundary_ambiguous", "window_scale", "energy", "rel", "math"]
