"""The seeded input generators (the one module the oracle and the CUDA path
share): shapes, the distributions' support, determinism per seed, and the
workload table."""
import numpy as np
import pytest

from paper_2308_00292_gb300 import inputs


@pytest.mark.parametrize("gen", ["uniform_cube", "clustered", "sphere"])
def test_3d_generators(gen):
    x, q = inputs.make(gen, 2000, 5)
    assert x.shape == (2000, 3) and q.shape == (2000,)
    x2, q2 = inputs.make(gen, 2000, 5)
    assert np.array_equal(x, x2) and np.array_equal(q, q2)
    assert not np.array_equal(x, inputs.make(gen, 2000, 6)[0])


def test_2d_generators():
    x, q = inputs.make("disk2d", 5000, 3)
    assert x.shape == (5000, 2) and np.all(np.hypot(x[:, 0], x[:, 1]) <= 1.0)
    assert np.all(np.abs(q) <= 1.0)
    x, q = inputs.make("circle2d", 5000, 3)
    assert np.allclose(np.hypot(x[:, 0], x[:, 1]), 1.0, atol=1e-15)
    x, q = inputs.make("circle_disk2d", 5001, 3)
    r = np.hypot(x[:, 0], x[:, 1])
    assert np.allclose(r[:2500], 1.0, atol=1e-15) and np.all(r[2500:] <= 1.0)
    assert np.array_equal(x, inputs.make("circle_disk2d", 5001, 3)[0])


def test_workload_table():
    for name, cfg in inputs.CONFIGS.items():
        assert cfg["eps"] > 0 and cfg["seed"] >= 0, name
    c = inputs.CONFIGS["log2d_circle_disk_n8e6"]
    assert c["gen"] == "circle_disk2d" and c["n"] == 8_000_000 and c["eps"] == 1e-8
