"""Seeded synthetic inputs: the many-solute batch recipe (uneven grids, 20-120 atoms)."""
import numpy as np

from paper_2403_01039_gb300 import synth


def _five_smooth(k):
    for p in (2, 3, 5):
        while k % p == 0:
            k //= p
    return k == 1


def test_smooth_even_is_smallest_valid_size():
    for n in range(2, 300):
        m = synth.smooth_even(n)
        assert m >= n and m % 2 == 0 and _five_smooth(m // 2)
        assert all(not (c % 2 == 0 and _five_smooth(c // 2)) for c in range(n, m))


def test_batch_workload_recipe():
    a = synth.batch_workload()
    b = synth.batch_workload()
    assert len(a) == 64 and [w["seed"] for w in a] == list(range(4000, 4064))
    for w, v in zip(a, b):
        n = w["grid"]["n"][0]
        assert w["grid"]["n"] == (n, n, n) and 64 <= n <= 128 and n == synth.smooth_even(n)
        atoms = len(w["solute"]["q"])
        assert 20 <= atoms <= 120
        xyz = w["solute"]["xyz"]
        r = 10.0 * (atoms / 50.0) ** (1.0 / 3.0)
        assert np.all(np.linalg.norm(xyz - xyz.mean(axis=0), axis=1) <= 2 * r)
        assert abs(np.sum(w["solute"]["q"])) < 1e-12
        assert np.array_equal(xyz, v["solute"]["xyz"])          # seeded
