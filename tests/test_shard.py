"""The sharded level solve (paper Sec. 9.5 and App. G: the V-cycle on each
rank's octs with halo exchanges and an all-reduced residual norm; Sec. 2: the
recursive k-section partition) on CPU ranks, with the FP64 oracle as every
rank's compute backend (tests/shard_oracle_backend.py).

* the k-section follows Sec. 2: prime factors largest first, cuts along the
  longest axis, balanced slabs;
* the exchange plan equals a brute-force list of the cells each rank reads
  from other ranks (neighbour table of the oracle);
* two gloo ranks (separate processes) and three thread ranks reproduce the
  single-rank oracle: bit for bit on a refined level (no reductions touch phi
  there), to rounding on a periodic level (whose mean is removed once, from
  all-reduced sums, instead of after every cycle)."""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_2604_06035_gb300 import inputs
from paper_2604_06035_gb300 import shard as S

HERE = os.path.dirname(os.path.abspath(__file__))


def test_split_sequence_is_the_prime_factorisation_largest_first():
    assert S.split_sequence(1) == []
    assert S.split_sequence(2) == [2]
    assert S.split_sequence(8) == [2, 2, 2]
    assert S.split_sequence(12) == [3, 2, 2]
    assert S.split_sequence(7) == [7]
    assert S.split_sequence(90) == [5, 3, 3, 2]


@pytest.mark.parametrize("n_ranks", [2, 3, 4, 6, 12])
def test_ksection_balances_disjoint_boxes(n_ranks):
    coords = inputs.uniform_oct_coords(5)  # 16^3 octs
    owner = S.ksection(coords, n_ranks)
    counts = np.bincount(owner, minlength=n_ranks)
    assert counts.sum() == len(coords) and np.all(counts > 0)
    # slabs are cut on whole oct planes: the imbalance is below one plane of the node
    assert counts.max() - counts.min() <= 16 * 16
    # every rank's octs fill an axis-aligned box, and the boxes are disjoint
    boxes = []
    for r in range(n_ranks):
        c = coords[owner == r].astype(np.int64)
        lo, hi = c.min(axis=0), c.max(axis=0) + 1
        assert np.prod(hi - lo) == len(c)
        boxes.append((lo, hi))
    for a in range(n_ranks):
        for b in range(a + 1, n_ranks):
            (l1, h1), (l2, h2) = boxes[a], boxes[b]
            assert np.any((h1 <= l2) | (h2 <= l1))
    # the first cut of 12 = 3 x 2 x 2 makes three slabs along the first (longest) axis
    if n_ranks == 12:
        first = [boxes[r][0][0] for r in range(0, 12, 4)]
        assert sorted(first) == [0, 5, 11] or len(set(first)) == 3


def _levels(cfg, owner0, parent_phi=None):
    """Oracle levels of a two-level workload built from keys in owner order."""
    perm = S.owner_order(owner0)
    B = O.Level(cfg["levels"][0], O.morton_encode(cfg["coords"][0]))
    B.set_density(cfg["rho"][0], 1.0)
    kf = O.morton_encode(cfg["coords"][1])[perm]
    F = O.Level(cfg["levels"][1], kf, parent=B)
    F.set_density(cfg["rho"][1][perm], 1.0)
    if parent_phi is not None:
        B.set_phi(parent_phi)
    return B, F, perm


def _plan_for(level, owner_sorted, n_ranks, refined):
    from shard_oracle_backend import OracleBackend
    b = OracleBackend(level, refined=refined, periodic_full=not refined)
    keys, act, levs = b.hierarchy()
    return b, S.ShardPlan.build(keys, act, levs, owner_sorted, n_ranks)


def test_plan_matches_brute_force_neighbour_reads():
    cfg = inputs.two_level_amr(base_level=5, seed=2)
    owner = S.ksection(cfg["coords"][1], 3)
    B, F, perm = _levels(cfg, owner)
    own = owner[perm]
    _, plan = _plan_for(F, own, 3, True)
    nbr = F.neighbors()[:, 1:]  # [n][6], -1 = coarse-fine ghost
    for c in (0, 1):
        want = {}
        for i in range(F.n):
            for d in range(6):
                j = nbr[i, d]
                if j >= 0 and own[j] != own[i]:
                    want.setdefault((int(own[j]), int(own[i])), set()).update(
                        8 * j + cc for cc in range(8) if S._parity(cc) == c)
        got = {k: set(v.tolist()) for k, v in plan.colour[0][c].items()}
        assert got == want
    # ranges tile every MG level in owner order
    for m, rg in enumerate(plan.ranges):
        assert rg[0][0] == 0 and rg[-1][1] == F.mg_n_octs(m)
        for r in range(2):
            assert rg[r][1] == rg[r + 1][0]


def _single_rank(cfg, owner, cycles, parent_phi):
    B, F, perm = _levels(cfg, owner, parent_phi)
    if parent_phi is None:
        B.solve(fixed_cycles=cycles)
        return B.get_phi(), None
    F.solve(fixed_cycles=cycles)
    return None, F.get_phi()


def _sharded_rank(rank, comm, cfg, owner, cycles, parent_phi, base):
    """One rank's sharded solve; returns (lo, hi, its phi rows)."""
    from shard_oracle_backend import OracleBackend
    n_ranks = comm.size
    if base:
        B = O.Level(cfg["levels"][0], O.morton_encode(cfg["coords"][0][S.owner_order(owner)]))
        B.set_density(cfg["rho"][0][S.owner_order(owner)], 1.0)
        be, plan = _plan_for(B, owner[S.owner_order(owner)], n_ranks, False)
        st = S.ShardedSolver(be, plan, comm).solve(fixed_cycles=cycles)
        lo, hi = plan.ranges[0][rank]
        return lo, hi, B.get_phi()[lo:hi], st
    B, F, perm = _levels(cfg, owner, parent_phi)
    be, plan = _plan_for(F, owner[perm], n_ranks, True)
    st = S.ShardedSolver(be, plan, comm).solve(fixed_cycles=cycles)
    lo, hi = plan.ranges[0][rank]
    return lo, hi, F.get_phi()[lo:hi], st


def _worker(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, HERE)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = inputs.two_level_amr(base_level=5, seed=2)
    comm = S.TorchComm("cpu")
    owner_b = S.ksection(cfg["coords"][0], world)
    lo, hi, phi_b, st_b = _sharded_rank(rank, comm, cfg, owner_b, 3, None, True)
    owner_f = S.ksection(cfg["coords"][1], world)
    rng = np.random.default_rng(5)
    pphi = rng.standard_normal((len(cfg["coords"][0]), 8))
    lo2, hi2, phi_f, st_f = _sharded_rank(rank, comm, cfg, owner_f, 3, pphi, False)
    np.savez(os.path.join(out_dir, "rank%d.npz" % rank), lo=lo, hi=hi, phi_b=phi_b, lo2=lo2, hi2=hi2,
             phi_f=phi_f, ex=st_f["exchanges"], cells=st_f["exchanged_cells"], rel=st_f["rel_final"])
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_gloo_ranks_reproduce_the_single_rank_oracle(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    cfg = inputs.two_level_amr(base_level=5, seed=2)
    # periodic base: phi to rounding of the single-rank oracle (same oct order)
    owner_b = S.ksection(cfg["coords"][0], world)
    pb = S.owner_order(owner_b)
    Bs = O.Level(cfg["levels"][0], O.morton_encode(cfg["coords"][0][pb]))
    Bs.set_density(cfg["rho"][0][pb], 1.0)
    Bs.solve(fixed_cycles=3)
    ref_b = Bs.get_phi()
    # refined level with a given parent phi: bit for bit
    owner_f = S.ksection(cfg["coords"][1], world)
    pphi = np.random.default_rng(5).standard_normal((len(cfg["coords"][0]), 8))
    _, ref_f = _single_rank(cfg, owner_f, 3, pphi)
    got_b = np.zeros_like(ref_b)
    got_f = np.zeros_like(ref_f)
    for r in range(world):
        z = np.load(os.path.join(tmp_path, "rank%d.npz" % r))
        got_b[int(z["lo"]):int(z["hi"])] = z["phi_b"]
        got_f[int(z["lo2"]):int(z["hi2"])] = z["phi_f"]
        assert int(z["ex"]) > 0 and int(z["cells"]) > 0
    assert np.max(np.abs(got_b - ref_b)) <= 1e-13 * np.max(np.abs(ref_b))
    assert np.array_equal(got_f, ref_f)


def test_three_thread_ranks_reproduce_the_single_rank_oracle():
    import threading
    cfg = inputs.two_level_amr(base_level=5, seed=2)
    world = 3
    owner_f = S.ksection(cfg["coords"][1], world)
    pphi = np.random.default_rng(7).standard_normal((len(cfg["coords"][0]), 8))
    hub = S.LocalHub(world)
    res = [None] * world
    err = []

    def run(r):
        try:
            res[r] = _sharded_rank(r, hub.comm(r), cfg, owner_f, 2, pphi, False)
        except Exception as e:  # surfaced below
            err.append(e)
            hub.barrier.abort()

    ts = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not err, err
    _, ref_f = _single_rank(cfg, owner_f, 2, pphi)
    got = np.zeros_like(ref_f)
    for lo, hi, phi, st in res:
        got[lo:hi] = phi
    assert np.array_equal(got, ref_f)
    # all ranks saw the same all-reduced residual history
    assert len({tuple(r[3]["rel_history"]) for r in res}) == 1
