"""Sharded level solve: one multigrid level split over ranks (GPUs).

The paper's multi-GPU path (Sec. 9.5, App. G) runs the V-cycle on every rank
over the octs it owns and exchanges the values of boundary octs with its
neighbours before each smoothing sweep, with an allreduce of the residual
norm; its domains come from a recursive k-section of space (Sec. 2).  This
module is that driver, owner-computes style:

* ``ksection`` splits a level's octs into one domain per rank: the rank count
  is factored into primes taken largest first (Sec. 2, Eq. split sequence),
  and each node of the tree is cut into k slabs along the longest axis of its
  box, with walls placed so that every slab holds octs in proportion to its
  ranks (Sec. 2, load-balanced wall placement; here by an exact sort of the
  octs' coordinates instead of a histogram search, as one host holds them).
* every rank builds a replica of the level from the same keys, sorted so that
  each rank's octs form one contiguous range (``owner_order``); the octs of
  each coarser multigrid level are owned by the owner of their first child,
  which keeps every level's ranges contiguous.
* ``ShardPlan`` lists, per multigrid level, which cells each rank must
  receive from which other rank: the colour-c cells of face-neighbour octs
  after a colour-c pass, the father cells restricted by another rank's
  children, and the coarse octs a rank's prolongation reads.
* ``ShardedSolver`` runs the V-cycle through a backend that executes every
  operation on the rank's range only (``CmgBackend``: the C-ABI range calls of
  libcmg.so), moving the listed cells with gather / scatter between the
  operations through a communicator (``TorchComm``: torch.distributed
  point-to-point and all-reduce; ``LocalHub``: ranks as threads of one
  process).

Since the range operations run the whole-level kernels' per-oct bodies and
every cell a rank reads is either its own or an exact copy of its owner's,
a sharded V-cycle computes the single-rank result cell for cell; only the
order of the norm sums (stopping test, periodic mean) differs.  Storage is
replicated (each rank holds the whole level): the exchange pattern is the
distributed one, the memory footprint is not.
"""
import threading

import numpy as np

# ------------------------------------------------------------ Morton keys
# Sec. 4.2 Eq. (morton_encode): bit b of i, j, k at key bits 3b, 3b+1, 3b+2.
_M = [np.uint64(x) for x in (0x1249249249249249, 0x10c30c30c30c30c3, 0x100f00f00f00f00f,
                             0x001f0000ff0000ff, 0x001f00000000ffff, 0x00000000001fffff)]


def _compact3(x):
    x = x & _M[0]
    x = (x ^ (x >> np.uint64(2))) & _M[1]
    x = (x ^ (x >> np.uint64(4))) & _M[2]
    x = (x ^ (x >> np.uint64(8))) & _M[3]
    x = (x ^ (x >> np.uint64(16))) & _M[4]
    x = (x ^ (x >> np.uint64(32))) & _M[5]
    return x


def _spread3(x):
    x = x.astype(np.uint64) & _M[5]
    x = (x | (x << np.uint64(32))) & _M[4]
    x = (x | (x << np.uint64(16))) & _M[3]
    x = (x | (x << np.uint64(8))) & _M[2]
    x = (x | (x << np.uint64(4))) & _M[1]
    x = (x | (x << np.uint64(2))) & _M[0]
    return x


def morton_decode(keys):
    """[n] uint64 keys -> [n, 3] int64 oct coordinates."""
    k = np.asarray(keys, dtype=np.uint64)
    return np.stack([_compact3(k), _compact3(k >> np.uint64(1)), _compact3(k >> np.uint64(2))],
                    axis=1).astype(np.int64)


def morton_encode(ijk):
    ijk = np.asarray(ijk, dtype=np.int64)
    return _spread3(ijk[:, 0]) | (_spread3(ijk[:, 1]) << np.uint64(1)) | (_spread3(ijk[:, 2]) << np.uint64(2))


# -------------------------------------------------------------- k-section

def split_sequence(n_ranks):
    """Prime factors of n_ranks, largest first (Sec. 2, Eq. split sequence)."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    f, n, p = [], n_ranks, 2
    while p * p <= n:
        while n % p == 0:
            f.append(p)
            n //= p
        p += 1
    if n > 1:
        f.append(n)
    return sorted(f, reverse=True)


def ksection(coords, n_ranks, box=None):
    """Owner rank of every oct (coords [n, 3] integer oct coordinates) by the
    recursive k-section of Sec. 2: at tree level l every node's box is cut into
    k_l slabs along its longest axis, the walls at whole oct coordinates chosen
    so that slab j holds the share of octs of its ranks.  box: (lo[3], hi[3])
    of the root, default the octs' bounding box."""
    coords = np.asarray(coords, dtype=np.int64)
    n = len(coords)
    owner = np.zeros(n, dtype=np.int32)
    if n == 0 or n_ranks == 1:
        return owner
    if box is None:
        box = (coords.min(axis=0), coords.max(axis=0) + 1)
    seq = split_sequence(n_ranks)

    def cut(idx, lo, hi, depth, rank0, ranks):
        if depth == len(seq):
            owner[idx] = rank0
            return
        k = seq[depth]
        per = ranks // k
        axis = int(np.argmax(np.asarray(hi) - np.asarray(lo)))
        x = coords[idx, axis]
        xs = np.sort(x)
        walls = [lo[axis]]
        for j in range(1, k):
            t = int(round(len(idx) * j / k))
            w = int(xs[t]) if t < len(xs) else int(hi[axis])
            walls.append(max(w, walls[-1]))
        walls.append(hi[axis])
        for j in range(k):
            sel = idx[(x >= walls[j]) & (x < walls[j + 1])]
            clo, chi = np.array(lo), np.array(hi)
            clo[axis], chi[axis] = walls[j], walls[j + 1]
            cut(sel, clo, chi, depth + 1, rank0 + j * per, per)

    cut(np.arange(n), np.asarray(box[0]), np.asarray(box[1]), 0, 0, n_ranks)
    return owner


def owner_order(owner):
    """Permutation that lists the octs rank by rank, each rank's octs in their
    original order: build every replica of the level from keys[perm]."""
    owner = np.asarray(owner)
    return np.lexsort((np.arange(len(owner)), owner))


# ------------------------------------------------------------------- plan

def _parity(c):
    return ((c & 1) + ((c >> 1) & 1) + ((c >> 2) & 1)) & 1


_COLOUR_CELLS = [np.array([c for c in range(8) if _parity(c) == p], dtype=np.int64) for p in (0, 1)]


class _Lookup:
    """Index of a key in one level's key array (-1 if absent)."""

    def __init__(self, keys):
        self.keys = np.asarray(keys, dtype=np.uint64)
        self.order = np.argsort(self.keys, kind="stable")
        self.sorted = self.keys[self.order]

    def __call__(self, q):
        q = np.asarray(q, dtype=np.uint64)
        if len(self.sorted) == 0:
            return np.full(q.shape, -1, dtype=np.int64)
        pos = np.clip(np.searchsorted(self.sorted, q), 0, len(self.sorted) - 1)
        hit = self.sorted[pos] == q
        return np.where(hit, self.order[pos], -1).astype(np.int64)


class ShardPlan:
    """Ownership ranges and the cells every rank receives from every other,
    for each multigrid level of one level's hierarchy.  Computed identically
    on every rank from the hierarchy's keys and cell masks.

    ranges[m][r] = (lo, hi): rank r owns octs lo..hi-1 of MG level m.
    colour[m][c][(src, dst)]: cells (oct * 8 + child) of colour c on MG level m
        that rank dst reads from rank src's octs (face neighbours).
    restrict[m][(src, dst)]: cells of MG level m + 1 that rank src's children
        write (father cells) and rank dst owns.
    prolong[m][(src, dst)]: cells of MG level m + 1 that rank dst's
        prolongation on level m reads from rank src's octs."""

    def __init__(self, n_ranks, ranges, colour, restrict, prolong):
        self.n_ranks = n_ranks
        self.ranges = ranges
        self.colour = colour
        self.restrict = restrict
        self.prolong = prolong

    @classmethod
    def build(cls, mg_keys, mg_active, mg_levs, owner0, n_ranks, nx=1, periodic_mask=7):
        depth = len(mg_keys)
        owners = [np.asarray(owner0, dtype=np.int64)]
        looks = [_Lookup(k) for k in mg_keys]
        full = [np.all(np.asarray(a) != 0, axis=1) for a in mg_active]
        for m in range(1, depth):
            f = np.nonzero(full[m - 1])[0]
            parent = looks[m](np.asarray(mg_keys[m - 1], dtype=np.uint64)[f] >> np.uint64(3))
            first = np.full(len(mg_keys[m]), np.iinfo(np.int64).max, dtype=np.int64)
            np.minimum.at(first, parent[parent >= 0], f[parent >= 0])
            if np.any(first == np.iinfo(np.int64).max):
                raise ValueError("a coarse oct without a fully active child")
            owners.append(owners[m - 1][first])
        ranges = []
        for m, o in enumerate(owners):
            if np.any(np.diff(o) < 0):
                raise ValueError("MG level %d: octs are not ordered by owner (build the level from keys in "
                                 "owner_order)" % m)
            ranges.append([(int(np.searchsorted(o, r, "left")), int(np.searchsorted(o, r, "right")))
                           for r in range(n_ranks)])

        def pairs(src_owner, dst_owner, cells):
            out = {}
            x = src_owner != dst_owner
            if not np.any(x):
                return out
            key = src_owner[x] * n_ranks + dst_owner[x]
            cl = cells[x]
            order = np.lexsort((cl, key))
            key, cl = key[order], cl[order]
            for k in np.unique(key):
                sel = cl[key == k]
                out[(int(k // n_ranks), int(k % n_ranks))] = np.unique(sel).astype(np.int32)
            return out

        colour, restrict, prolong = [], [], []
        for m in range(depth):
            keys = np.asarray(mg_keys[m], dtype=np.uint64)
            n = len(keys)
            npd = nx << (mg_levs[m] - 1)
            xyz = morton_decode(keys)
            src_l, dst_l = [], []
            for d in range(6):
                a, step = d >> 1, (1 if d & 1 else -1)
                q = xyz.copy()
                q[:, a] += step
                if (periodic_mask >> a) & 1:
                    q[:, a] %= npd
                    ok = np.ones(n, dtype=bool)
                else:
                    ok = (q[:, a] >= 0) & (q[:, a] < npd)
                nb = np.full(n, -1, dtype=np.int64)
                if np.any(ok):
                    nb[ok] = looks[m](morton_encode(q[ok]))
                hit = nb >= 0
                src_l.append(nb[hit])
                dst_l.append(np.nonzero(hit)[0])
            src_oct = np.concatenate(src_l) if src_l else np.zeros(0, np.int64)
            dst_oct = np.concatenate(dst_l) if dst_l else np.zeros(0, np.int64)
            per_c = []
            for c in (0, 1):
                cc = _COLOUR_CELLS[c]
                so = np.repeat(src_oct, 4)
                do = np.repeat(dst_oct, 4)
                cells = (so * 8 + np.tile(cc, len(src_oct))).astype(np.int64)
                per_c.append(pairs(owners[m][so], owners[m][do], cells))
            colour.append(per_c)
            if m + 1 < depth:
                # restriction: fully active children write their father cell
                f = np.nonzero(full[m])[0]
                p = looks[m + 1](keys[f] >> np.uint64(3))
                cells = p * 8 + (keys[f] & np.uint64(7)).astype(np.int64)
                restrict.append(pairs(owners[m][f], owners[m + 1][p], cells))
                # prolongation: the 2x2x2 coarse octs around the father cell,
                # toward its octant (absent ones read zero)
                pk = keys >> np.uint64(3)
                oc = (keys & np.uint64(7)).astype(np.int64)
                pxyz = morton_decode(pk)
                cnpd = nx << (mg_levs[m + 1] - 1)
                src_l, dst_l = [], []
                for t in range(8):
                    q = pxyz.copy()
                    ok = np.ones(n, dtype=bool)
                    for a in range(3):
                        if (t >> a) & 1:
                            q[:, a] += np.where((oc >> a) & 1, 1, -1)
                            if (periodic_mask >> a) & 1:
                                q[:, a] %= cnpd
                            else:
                                ok &= (q[:, a] >= 0) & (q[:, a] < cnpd)
                    nb = np.full(n, -1, dtype=np.int64)
                    if np.any(ok):
                        nb[ok] = looks[m + 1](morton_encode(q[ok]))
                    hit = nb >= 0
                    src_l.append(nb[hit])
                    dst_l.append(np.nonzero(hit)[0])
                so = np.concatenate(src_l)
                do = np.concatenate(dst_l)
                cells = np.repeat(so, 8) * 8 + np.tile(np.arange(8), len(so))
                prolong.append(pairs(owners[m + 1][np.repeat(so, 8)], owners[m][np.repeat(do, 8)], cells))
        return cls(n_ranks, ranges, colour, restrict, prolong)

    def sends(self, table, rank):
        return {dst: cells for (src, dst), cells in table.items() if src == rank}

    def recvs(self, table, rank):
        return {src: cells for (src, dst), cells in table.items() if dst == rank}


# ---------------------------------------------------------- communicators

class TorchComm:
    """Point-to-point exchanges and all-reduce over torch.distributed (gloo
    or nccl); buffers move on `device` (CPU for gloo)."""

    def __init__(self, device="cpu", group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)
        self.device = device

    def exchange(self, sends, recv_sizes):
        import torch
        reqs, out = [], {}
        for q, n in sorted(recv_sizes.items()):
            out[q] = torch.empty(int(n), dtype=torch.float64, device=self.device)
            reqs.append(self.dist.irecv(out[q], src=q, group=self.group))
        for q, t in sorted(sends.items()):
            reqs.append(self.dist.isend(t.to(self.device).contiguous(), dst=q, group=self.group))
        for r in reqs:
            r.wait()
        return out

    def allreduce_sum(self, x):
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, group=self.group)
        return float(t.item())


class LocalHub:
    """Ranks as threads of one process (each driving its own replica): a
    barrier-synchronised mailbox.  The ranks' GPU work never waits on another
    rank's kernels; every exchange goes through the host between operations."""

    def __init__(self, n):
        self.n = n
        self.box = {}
        self.vals = [0.0] * n
        self.barrier = threading.Barrier(n)
        self.lock = threading.Lock()

    def comm(self, rank):
        return _LocalComm(self, rank)


class _LocalComm:
    def __init__(self, hub, rank):
        self.hub, self.rank, self.size = hub, rank, hub.n

    def exchange(self, sends, recv_sizes):
        h = self.hub
        with h.lock:
            for q, t in sends.items():
                h.box[(self.rank, q)] = t.clone()
        h.barrier.wait()
        with h.lock:
            out = {q: h.box.pop((q, self.rank)) for q in recv_sizes}
        h.barrier.wait()
        return out

    def allreduce_sum(self, x):
        h = self.hub
        h.vals[self.rank] = float(x)
        h.barrier.wait()
        s = 0.0
        for v in h.vals:  # rank order on every rank
            s += v
        h.barrier.wait()
        return s


# ----------------------------------------------------------------- solver

class ShardedSolver:
    """The V-cycle of one level on this rank's octs (App. G), exchanging the
    plan's cells between operations; norms by all-reduce.  The level's phi
    must be zero on entry (the relative residual is measured against the
    residual of the initial guess, ||f - L 0|| including coarse-fine values,
    as in the single-rank solve)."""

    def __init__(self, backend, plan, comm):
        self.b, self.plan, self.comm = backend, plan, comm
        self.rank = comm.rank
        self._cells = {}
        self.exchanges = 0
        self.exchanged_cells = 0

    def _dev_cells(self, cells):
        key = id(cells)
        if key not in self._cells:
            self._cells[key] = (cells, self.b.cells(cells))
        return self._cells[key][1]

    def _exchange(self, m, table, fields):
        sends = self.plan.sends(table, self.rank)
        recvs = self.plan.recvs(table, self.rank)
        for field in fields:
            out = {q: self.b.gather(m, field, self._dev_cells(c)) for q, c in sends.items()}
            got = self.comm.exchange(out, {q: len(c) for q, c in recvs.items()})
            for q, c in recvs.items():
                self.b.scatter(m, field, self._dev_cells(c), got[q])
            self.exchanges += 1
            self.exchanged_cells += sum(len(c) for c in sends.values())

    def _range(self, m):
        return self.plan.ranges[m][self.rank]

    def _pass(self, m, colour, zero_other=False):
        lo, hi = self._range(m)
        self.b.sweep(m, colour, zero_other, lo, hi)
        self._exchange(m, self.plan.colour[m][colour], (0,))

    def _coarse(self, m, p):
        if self.b.exact_coarse:
            lo, hi = self._range(m)
            if hi > lo:
                self.b.coarse_exact()
            return
        for k in range(p["coarse_sweeps"]):
            self._pass(m, 0, zero_other=(k == 0 and m > 0))
            self._pass(m, 1)

    def _vcycle(self, m, p):
        depth = self.b.depth
        if m == depth - 1:
            self._coarse(m, p)
            return
        lo, hi = self._range(m)
        for s in range(p["n_pre"]):
            self._pass(m, 0, zero_other=(m > 0 and s == 0))
            self._pass(m, 1)
        self.b.restrict(m, p["n_pre"] > 0, lo, hi)
        # father cells written by other ranks' children: their source, and
        # phi = 0 as the restriction left it
        self._exchange(m + 1, self.plan.restrict[m], (1, 0))
        if p["n_pre"] == 0 and m + 1 < depth - 1:
            # the coarse level's residual comes first there and reads the
            # neighbours' (zeroed) phi
            self._exchange(m + 1, self.plan.colour[m + 1][0], (0,))
            self._exchange(m + 1, self.plan.colour[m + 1][1], (0,))
        self._vcycle(m + 1, p)
        self._exchange(m + 1, self.plan.prolong[m], (0,))
        c0_dead = p["n_post"] > 0
        self.b.prolong(m, c0_dead, lo, hi)
        # the corrected cells of the neighbours' octs (colour 1 only when a
        # colour-0 pass comes next)
        self._exchange(m, self.plan.colour[m][1], (0,))
        if not c0_dead:
            self._exchange(m, self.plan.colour[m][0], (0,))
        for s in range(p["n_post"]):
            self._pass(m, 0)
            self._pass(m, 1)

    def _norm2(self, c1_swept):
        lo, hi = self._range(0)
        return self.comm.allreduce_sum(self.b.residual(0, c1_swept, lo, hi))

    def solve(self, tol=1e-10, max_cycles=100, fixed_cycles=0, n_pre=2, n_post=2, coarse_sweeps=4):
        p = {"n_pre": n_pre, "n_post": n_post, "coarse_sweeps": coarse_sweeps}
        self.b.ghosts()
        n0 = self._norm2(False)
        hist = []
        rel = 1.0 if n0 > 0 else 0.0
        cycles = 0
        target = fixed_cycles if fixed_cycles > 0 else max_cycles
        if n0 > 0:
            while cycles < target and (fixed_cycles > 0 or rel > tol):
                self._vcycle(0, p)
                cycles += 1
                rel = float(np.sqrt(self._norm2(n_post > 0) / n0))
                hist.append(rel)
                if not np.isfinite(rel):
                    break
        if self.b.periodic_full:
            lo, hi = self._range(0)
            total = self.comm.allreduce_sum(self.b.sum_phi(lo, hi))
            self.b.shift_phi(lo, hi, total / (8.0 * self.b.n_octs))
        return {"cycles": cycles, "rel_final": rel, "rel_history": hist, "norm0": float(np.sqrt(n0)),
                "exchanges": self.exchanges, "exchanged_cells": self.exchanged_cells}

    def replicate(self):
        """Make every replica's level-0 phi whole (each rank sends its own
        cells to every other rank), e.g. before the level serves as the parent
        whose phi gives a refined level's coarse-fine values."""
        lo, hi = self._range(0)
        mine = np.arange(lo * 8, hi * 8, dtype=np.int32)
        table = {}
        for q in range(self.plan.n_ranks):
            if q != self.rank:
                table[(self.rank, q)] = mine
                qlo, qhi = self.plan.ranges[0][q]
                table[(q, self.rank)] = np.arange(qlo * 8, qhi * 8, dtype=np.int32)
        self._exchange(0, table, (0,))


# ----------------------------------------------------------- GPU backend

class CmgBackend:
    """Range operations on a libcmg.so level (FP64), for ShardedSolver."""

    def __init__(self, level, periodic_mask=7, nx=1, refined=None):
        from . import cmg
        self.cmg = cmg
        self.L = level
        self.depth = cmg.cmg_level_mg_depth(level)
        self.n_octs = cmg.cmg_level_n_octs(level)
        info = [cmg.cmg_level_mg_info(level, m) for m in range(self.depth)]
        self.mg_n = [i[0] for i in info]
        self.mg_levs = [i[1] for i in info]
        self.refined = (level.parent is not None) if refined is None else refined
        self.periodic_full = (not self.refined and periodic_mask == 7 and self.n_octs == (nx << (self.mg_levs[0] - 1)) ** 3)
        self.exact_coarse = self.periodic_full and nx == 1 and self.mg_levs[-1] == 1 and self.mg_n[-1] == 1

    def hierarchy(self):
        c = self.cmg
        return ([c.cmg_level_mg_keys(self.L, m) for m in range(self.depth)],
                [c.cmg_level_mg_active(self.L, m) for m in range(self.depth)], self.mg_levs)

    def cells(self, cells):
        import torch
        return torch.from_numpy(np.ascontiguousarray(cells, dtype=np.int32)).cuda()

    def sweep(self, m, colour, zero_other, lo, hi):
        self.cmg.cmg_level_mg_step_range(self.L, m, self.cmg.CMG_OPR_SWEEP, colour | (2 if zero_other else 0), lo, hi)

    def residual(self, m, c1_swept, lo, hi):
        return self.cmg.cmg_level_mg_step_range(self.L, m, self.cmg.CMG_OPR_RESIDUAL, int(c1_swept), lo, hi)

    def restrict(self, m, c1_swept, lo, hi):
        self.cmg.cmg_level_mg_step_range(self.L, m, self.cmg.CMG_OPR_RESTRICT, int(c1_swept), lo, hi)

    def prolong(self, m, c0_dead, lo, hi):
        self.cmg.cmg_level_mg_step_range(self.L, m, self.cmg.CMG_OPR_PROLONG, int(c0_dead), lo, hi)

    def coarse_exact(self):
        self.cmg.cmg_level_mg_step(self.L, self.depth - 1, self.cmg.CMG_OP_COARSE, self.cmg.CMG_PREC_FP64, 0)

    def ghosts(self):
        if self.refined:
            self.cmg.cmg_level_mg_step(self.L, 0, self.cmg.CMG_OP_GHOSTS)

    def sum_phi(self, lo, hi):
        return self.cmg.cmg_level_mg_step_range(self.L, 0, self.cmg.CMG_OPR_SUM_PHI, 0, lo, hi)

    def shift_phi(self, lo, hi, v):
        self.cmg.cmg_level_mg_step_range(self.L, 0, self.cmg.CMG_OPR_SHIFT_PHI, 0, lo, hi, value=v)

    def gather(self, m, field, cells):
        return self.cmg.cmg_level_mg_gather(self.L, m, field, cells)

    def scatter(self, m, field, cells, values):
        self.cmg.cmg_level_mg_scatter(self.L, m, field, cells, values.to(cells.device))
