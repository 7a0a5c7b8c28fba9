"""Test infrastructure: the oracle as a ShardedSolver backend, so that the
sharded driver (partition, exchange schedule, norms) runs on CPU ranks.

Each rank holds a whole oracle level (a replica).  An operation on the octs
[lo, hi) is the oracle's whole-level operation followed by restoring every
cell outside the range (the cells this rank does not own keep the values the
exchanges gave them).  A red-black colour pass reads only the other colour,
the residual and prolongation of an oct read only other octs' values, and the
restriction writes each father cell from its own child, so the restored
whole-level step equals the step on the range alone."""
import numpy as np
import torch

import oracle as O


class OracleBackend:
    def __init__(self, level, refined, periodic_full):
        self.L = level
        self.depth = level.mg_depth
        self.n_octs = level.n
        self.mg_levs = [level.mg_lev(m) for m in range(self.depth)]
        self.refined = refined
        self.periodic_full = periodic_full
        self.exact_coarse = periodic_full and self.mg_levs[-1] == 1 and level.mg_n_octs(self.depth - 1) == 1
        keys = [np.asarray(level.mg_keys(m), dtype=np.uint64) for m in range(self.depth)]
        act = [level.mg_active(m) for m in range(self.depth)]
        # father cell (coarse oct * 8 + octant) of every fully active oct, per MG level
        self._father = []
        for m in range(self.depth - 1):
            order = np.argsort(keys[m + 1])
            sk = keys[m + 1][order]
            pk = keys[m] >> np.uint64(3)
            pos = np.clip(np.searchsorted(sk, pk), 0, max(len(sk) - 1, 0))
            p = np.where(sk[pos] == pk, order[pos], -1)
            full = np.all(act[m] != 0, axis=1)
            fa = np.where(full & (p >= 0), p * 8 + (keys[m] & np.uint64(7)).astype(np.int64), -1)
            self._father.append(fa)
        self._keys, self._act = keys, act

    def hierarchy(self):
        return self._keys, self._act, self.mg_levs

    def cells(self, cells):
        return np.asarray(cells, dtype=np.int64)

    def _keep_range(self, m, field, before, lo, hi):
        after = self.L.mg_get(m, field)
        after[:lo] = before[:lo]
        after[hi:] = before[hi:]
        self.L.mg_set(m, field, after)

    def _ghost(self, m):
        return m == 0 and self.refined

    def sweep(self, m, colour, zero_other, lo, hi):
        before = self.L.mg_get(m, "phi")
        if zero_other:
            # the pass that follows a restriction reads an all-zero other
            # colour (the single-rank restriction zeroed every coarse cell);
            # this replica's other-colour cells of octs it does not own may
            # be stale, and are overwritten or exchanged before any later read
            z = before.copy()
            z[:, [c for c in range(8) if (bin(c).count("1") & 1) != colour]] = 0.0
            self.L.mg_set(m, "phi", z)
            before = z
        if self._ghost(m):
            self.L.ghosts()
        O.lib().or_rb_colour_pass(self.L._h, m, colour, int(self._ghost(m)))
        self._keep_range(m, "phi", before, lo, hi)

    def residual(self, m, c1_swept, lo, hi):
        if self._ghost(m):
            self.L.ghosts()
        O.lib().or_residual(self.L._h, m, int(self._ghost(m)))
        r = self.L.mg_get(m, "r")[lo:hi].ravel()
        return float(np.sum(r * r))

    def restrict(self, m, c1_swept, lo, hi):
        if self._ghost(m):
            self.L.ghosts()
        O.lib().or_residual(self.L._h, m, int(self._ghost(m)))
        f_before = self.L.mg_get(m + 1, "f").ravel().copy()
        p_before = self.L.mg_get(m + 1, "phi").ravel().copy()
        self.L.restrict(m)
        f_after = self.L.mg_get(m + 1, "f").ravel()
        p_after = self.L.mg_get(m + 1, "phi").ravel()
        mine = np.zeros(len(f_after), dtype=bool)
        fa = self._father[m][lo:hi]
        mine[fa[fa >= 0]] = True
        f_after[~mine] = f_before[~mine]
        p_after[~mine] = p_before[~mine]
        self.L.mg_set(m + 1, "f", f_after)
        self.L.mg_set(m + 1, "phi", p_after)

    def prolong(self, m, c0_dead, lo, hi):
        before = self.L.mg_get(m, "phi")
        self.L.prolong(m)
        self._keep_range(m, "phi", before, lo, hi)

    def coarse_exact(self):
        self.L.coarse_solve(0)

    def ghosts(self):
        if self.refined:
            self.L.ghosts()

    def sum_phi(self, lo, hi):
        return float(np.sum(self.L.mg_get(0, "phi")[lo:hi]))

    def shift_phi(self, lo, hi, v):
        p = self.L.mg_get(0, "phi")
        p[lo:hi] -= v
        self.L.mg_set(0, "phi", p)

    def gather(self, m, field, cells):
        f = self.L.mg_get(m, "phi" if field == 0 else "f").ravel()
        return torch.from_numpy(f[cells].copy())

    def scatter(self, m, field, cells, values):
        name = "phi" if field == 0 else "f"
        f = self.L.mg_get(m, name).ravel()
        f[cells] = values.cpu().numpy()
        self.L.mg_set(m, name, f)
