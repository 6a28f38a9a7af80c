"""Seeded input generators (shared by both sides; no method arithmetic)."""
import numpy as np

from paper_2112_07075_b300 import inputs


def test_batch_problem_generator_is_seeded_and_balanced():
    a = inputs.batch_problems(4)
    b = inputs.batch_problems(4)
    assert a == b and len(a) == 256
    assert {p["order"] for p in a} == {1, 2, 3, 4}
    assert all(8 <= p["n"] <= 64 for p in a)
    assert sum(p["kind"] == "gresho" for p in a) == 128


def test_uniform01_is_counter_based_and_in_range():
    u = inputs.uniform01(7, np.arange(1000, dtype=np.uint64))
    assert np.all((u >= 0) & (u < 1)) and abs(u.mean() - 0.5) < 0.05
    assert np.array_equal(u[10:20], inputs.uniform01(7, np.arange(10, 20, dtype=np.uint64)))
    assert not np.array_equal(u, inputs.uniform01(8, np.arange(1000, dtype=np.uint64)))
