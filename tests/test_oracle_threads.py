"""The oracle's OpenMP loops (used only to time the all-cores CPU baseline) give
the same bits as one thread: every node's collision is independent and the push
writes each target slot exactly once."""
import numpy as np

from paper_2101_03055_gb300 import inputs as I


def test_thread_count_does_not_change_results(oracle_mod):
    pb = I.chemotaxis_plume(61, 37, seed=4)
    try:
        oracle_mod.set_threads(1)
        a = oracle_mod.OracleSim(pb)
        a.step(40)
        used = oracle_mod.set_threads(4)
        b = oracle_mod.OracleSim(pb)
        b.step(40)
    finally:
        oracle_mod.set_threads(1)
    assert used in (1, 4)
    assert np.array_equal(a.moments(), b.moments())
