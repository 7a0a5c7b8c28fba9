"""The oracle's threaded loops (or_set_threads) compute the same bits as one
thread: every parallel loop writes disjoint cells and reads only values no
other iteration writes (one colour of a red-black pass reads only the other
colour), and every sum over cells stays serial in the same order.  The CPU
baseline of the benchmark times the oracle on all host cores on this
premise."""
import numpy as np
import pytest

import oracle as O
from paper_2604_06035_gb300 import inputs


def _solve_all(threads):
    O.set_threads(threads)
    try:
        cfg = inputs.two_level_amr(base_level=5, seed=2)
        B = O.Level(5, O.morton_encode(cfg["coords"][0]))
        F = O.Level(6, O.morton_encode(cfg["coords"][1]), parent=B)
        B.set_density(cfg["rho"][0], 1.0)
        F.set_density(cfg["rho"][1], 1.0)
        out = {"nbr_f": F.neighbors()}
        _, sb = B.solve(tol=1e-11)
        _, sf = F.solve(fixed_cycles=3)
        out["phi_b"], out["phi_f"] = B.get_phi(), F.get_phi()
        out["hist"] = np.array(sb["rel_history"] + sf["rel_history"])
        F.set_phi(np.zeros_like(out["phi_f"]))
        _, sm = F.solve_mixed(fixed_cycles=2)
        out["phi_f_mixed"], out["hist_mixed"] = F.get_phi(), np.array(sm["rel_history"])
        F.set_phi(np.zeros_like(out["phi_f"]))
        _, sp = F.solve_pcg(fixed_cycles=3)
        out["phi_f_pcg"], out["hist_pcg"] = F.get_phi(), np.array(sp["rel_history"])
        out["ghosts"] = F.ghosts()
        return out
    finally:
        O.set_threads(1)


def test_threads_are_bit_identical():
    n = O.set_threads(4)
    O.set_threads(1)
    if n == 1:
        pytest.skip("oracle built without OpenMP")
    one, four = _solve_all(1), _solve_all(4)
    for k in one:
        a, b = one[k], four[k]
        assert a.dtype == b.dtype and a.shape == b.shape, k
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8)), k


def test_thread_count_is_reported():
    assert O.set_threads(1) == 1
    assert O.get_threads() == 1
    n = O.set_threads(3)
    assert n in (1, 3)
    O.set_threads(1)
