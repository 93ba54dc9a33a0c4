"""Spatial domain decomposition of the split step (Sec. II.F: the paper's code
runs MPI sub-domains): slabs along x, one rank per device, and the host
logic that keeps them one simulation -- which rank owns which cells, the
ghost-layer exchange of E and B between the phases of the step, the sum of
the current deposited into ghost layers into the neighbours' cells, and the
migration of particles whose position left the slab -- over
torch.distributed point-to-point messages (gloo on CPU ranks; NCCL sends on
a multi-GPU machine).

The grid is periodic along x (rank R-1's right neighbour is rank 0).  A
rank's engine holds its slab -- cells [x0, x1) of the global grid, in
slab-local coordinates (x_local = x - x0 dx) -- with G ghost layers on each
side.  The engine interface (duck-typed):

  phase(k)             phase k of the split step: 0 E^{n+1/2} (with J^n),
                       1 B^{n+1/2}, 2 push and deposit J^{n+1}, 3 B^{n+1},
                       4 E^{n+1} (with J^{n+1}); the engine updates only its
                       own cells [0, n) and may deposit into the ghosts
  layers(c, lo, hi)    component c's x-layers [lo, hi) (slab-local index,
                       ghosts at -G..-1 and n..n+G-1), an array (..., hi - lo)
  set_layers(c, lo, a) overwrite layers [lo, lo + a.shape[-1])
  add_layers(c, lo, a) add into them
  take_leaving(isp)    the particles that left the slab in the last push:
                       a dict of arrays with 'x' (n, 3) slab-local positions
                       and any other per-particle state the engine carries
  insert(isp, parts)   append particles (the same dict, positions local)

Exchange schedule of one step, from the stencils (Eqs. (9)-(12) take
backward differences of B for E and forward differences of E for B; the
gather of Eq. (19) reads up to two layers beyond the particle's cell; the
Esirkepov window of Eqs. (20)-(22) reaches two layers beyond the slab):

  phase 0 -> E ghosts -> phase 1 -> B ghosts -> phase 2 -> J ghost sum,
  migration -> phase 3 -> B ghosts -> phase 4

(phase 3 needs E ghosts, unchanged since after phase 0; phase 0 of the next
step needs B ghosts, exchanged after phase 3, and the summed J).  start()
exchanges E and B once before the first step.
"""
from __future__ import annotations

import numpy as np

EX, EY, EZ, BX, BY, BZ, JX, JY, JZ = range(9)
E_COMPS = (EX, EY, EZ)
B_COMPS = (BX, BY, BZ)
J_COMPS = (JX, JY, JZ)

_TAG_TO_LEFT, _TAG_TO_RIGHT = 11, 12


def slab_bounds(n_x: int, ranks: int, rank: int) -> tuple[int, int]:
    """cells [x0, x1) of rank `rank` when n_x cells are split into `ranks`
    slabs as evenly as possible (the first n_x % ranks slabs one cell
    wider)"""
    if ranks < 1 or not 0 <= rank < ranks:
        raise ValueError("bad rank")
    base, extra = divmod(int(n_x), int(ranks))
    x0 = rank * base + min(rank, extra)
    return x0, x0 + base + (1 if rank < extra else 0)


class SlabDecomposition:
    """One rank's view of the decomposition: its slab, its neighbours, and the
    exchanges of the split step (see the module docstring).

    n_x: global cells along x; dx: cell size along x; ghost: ghost layers
    per side (at least the reach of the widest stencil: 4 for the order-2
    and order-4 shapes); dist: torch.distributed (initialised), or None for
    a single rank (every exchange is then the periodic self-copy)."""

    def __init__(self, n_x: int, dx: float, ghost: int = 4, dist=None):
        self.dist = dist
        self.rank = dist.get_rank() if dist is not None else 0
        self.ranks = dist.get_world_size() if dist is not None else 1
        self.n_x = int(n_x)
        self.dx = float(dx)
        self.G = int(ghost)
        self.x0, self.x1 = slab_bounds(self.n_x, self.ranks, self.rank)
        self.n = self.x1 - self.x0
        if self.n < self.G:
            raise ValueError(f"slab of {self.n} cells is narrower than its {self.G} ghost layers")
        self.left = (self.rank - 1) % self.ranks
        self.right = (self.rank + 1) % self.ranks
        lx0, lx1 = slab_bounds(self.n_x, self.ranks, self.left)
        self.n_left = lx1 - lx0

    # -------------------------------------------------------------------
    # messages: every exchange sends one array to each neighbour and receives
    # one from each (tags tell them apart when both neighbours are one rank)
    # -------------------------------------------------------------------
    def _swap(self, to_left: np.ndarray, to_right: np.ndarray):
        """send to_left to the left neighbour and to_right to the right one;
        return (from_left, from_right), shaped like what they sent"""
        if self.ranks == 1:
            return to_right, to_left  # periodic self-neighbour
        import torch
        sl, sr = torch.from_numpy(np.ascontiguousarray(to_left)), torch.from_numpy(np.ascontiguousarray(to_right))
        rl, rr = torch.empty_like(sr), torch.empty_like(sl)
        reqs = [self.dist.isend(sl, self.left, tag=_TAG_TO_LEFT), self.dist.isend(sr, self.right, tag=_TAG_TO_RIGHT),
                self.dist.irecv(rl, self.left, tag=_TAG_TO_RIGHT), self.dist.irecv(rr, self.right, tag=_TAG_TO_LEFT)]
        for r in reqs:
            r.wait()
        return rl.numpy(), rr.numpy()

    def _swap_var(self, to_left: np.ndarray, to_right: np.ndarray):
        """as _swap for arrays whose first dimension differs per message
        (particles): the lengths go first"""
        if self.ranks == 1:
            return to_right, to_left
        nl, nr = self._swap(np.array([len(to_left)], dtype=np.int64), np.array([len(to_right)], dtype=np.int64))
        import torch
        shape = to_left.shape[1:]
        sl, sr = torch.from_numpy(np.ascontiguousarray(to_left)), torch.from_numpy(np.ascontiguousarray(to_right))
        rl = torch.empty((int(nl[0]),) + shape, dtype=sl.dtype)
        rr = torch.empty((int(nr[0]),) + shape, dtype=sl.dtype)
        reqs = []
        if len(to_left):
            reqs.append(self.dist.isend(sl, self.left, tag=_TAG_TO_LEFT))
        if len(to_right):
            reqs.append(self.dist.isend(sr, self.right, tag=_TAG_TO_RIGHT))
        if len(rl):
            reqs.append(self.dist.irecv(rl, self.left, tag=_TAG_TO_RIGHT))
        if len(rr):
            reqs.append(self.dist.irecv(rr, self.right, tag=_TAG_TO_LEFT))
        for r in reqs:
            r.wait()
        return rl.numpy(), rr.numpy()

    # -------------------------------------------------------------------
    # the three exchanges
    # -------------------------------------------------------------------
    def exchange_ghosts(self, engine, comps) -> None:
        """fill the G ghost layers of each component on both sides with the
        neighbours' own layers: my [0, G) become the left neighbour's right
        ghosts [n_left, n_left + G), my [n - G, n) the right neighbour's left
        ghosts [-G, 0)"""
        G, n = self.G, self.n
        send_l = np.stack([engine.layers(c, 0, G) for c in comps])
        send_r = np.stack([engine.layers(c, n - G, n) for c in comps])
        from_l, from_r = self._swap(send_l, send_r)
        for i, c in enumerate(comps):
            engine.set_layers(c, -G, from_l[i])
            engine.set_layers(c, n, from_r[i])

    def sum_ghost_current(self, engine) -> None:
        """add the current deposited into my ghost layers to the neighbours'
        cells they overlap (my [-G, 0) -> left's [n_left - G, n_left), my
        [n, n + G) -> right's [0, G)), and receive theirs into mine"""
        G, n = self.G, self.n
        send_l = np.stack([engine.layers(c, -G, 0) for c in J_COMPS])
        send_r = np.stack([engine.layers(c, n, n + G) for c in J_COMPS])
        from_l, from_r = self._swap(send_l, send_r)
        for i, c in enumerate(J_COMPS):
            engine.add_layers(c, 0, from_l[i])       # the left neighbour's right ghosts are my first cells
            engine.add_layers(c, n - G, from_r[i])   # the right neighbour's left ghosts are my last cells

    def migrate(self, engine, n_species: int) -> int:
        """hand every particle that left the slab to the neighbour it entered,
        shifted into that neighbour's frame; returns how many left"""
        L = self.n * self.dx
        moved = 0
        for isp in range(n_species):
            out = engine.take_leaving(isp)
            x = out["x"]
            moved += len(x)
            go_left = x[:, 0] < 0.0
            keys = sorted(out.keys())
            packs = {}
            for side, sel in (("l", go_left), ("r", ~go_left)):
                cols = []
                for k in keys:
                    a = np.asarray(out[k])[sel]
                    if k == "x":
                        a = a.copy()
                        a[:, 0] += self.n_left * self.dx if side == "l" else -L
                    per = int(np.prod(a.shape[1:], dtype=np.int64))  # elements per particle
                    cols.append(np.ascontiguousarray(a.reshape(len(a), per)).view(np.uint8))
                packs[side] = np.concatenate(cols, axis=1)
            from_l, from_r = self._swap_var(packs["l"], packs["r"])
            for got in (from_l, from_r):
                if len(got) == 0:
                    continue
                parts, off = {}, 0
                for k in keys:
                    proto = np.asarray(out[k])
                    width = int(np.prod(proto.shape[1:], dtype=np.int64)) * proto.dtype.itemsize
                    raw = np.ascontiguousarray(got[:, off:off + width])
                    parts[k] = raw.view(proto.dtype).reshape((len(got),) + proto.shape[1:])
                    off += width
                engine.insert(isp, parts)
        return moved

    # -------------------------------------------------------------------
    # the step
    # -------------------------------------------------------------------
    def start(self, engine) -> None:
        """ghosts of E and B from the neighbours, before the first step"""
        self.exchange_ghosts(engine, E_COMPS + B_COMPS)

    def step(self, engine, n_species: int) -> None:
        """one split step on every rank (all ranks call it together)"""
        engine.phase(0)
        self.exchange_ghosts(engine, E_COMPS)
        engine.phase(1)
        self.exchange_ghosts(engine, B_COMPS)
        engine.phase(2)
        self.sum_ghost_current(engine)
        self.migrate(engine, n_species)
        engine.phase(3)
        self.exchange_ghosts(engine, B_COMPS)
        engine.phase(4)

    def allreduce_sum(self, values) -> np.ndarray:
        """FP64 sum over ranks (global diagnostics: energies, counts)"""
        v = np.asarray(values, dtype=np.float64)
        if self.ranks == 1:
            return v
        import torch
        t = torch.from_numpy(v.copy())
        self.dist.all_reduce(t)
        return t.numpy()
