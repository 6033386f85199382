"""The seeded input generator: SplitMix64 constants and the workload recipes' shapes."""
import numpy as np

import synthetic


def test_splitmix64_reference_value():
    # The SplitMix64 sequence started from state 0 begins 0xE220A8397B1DCDAF
    # (the published generator's first output for seed 0).
    z = synthetic._mix(np.array([synthetic.GAMMA], dtype=np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF
    assert synthetic._mix_int(synthetic.GAMMA) == 0xE220A8397B1DCDAF


def test_uniform_is_deterministic_and_in_range():
    a = synthetic.uniform(7, 0, 10000, -0.1, 0.1)
    b = synthetic.uniform(7, 0, 10000, -0.1, 0.1)
    np.testing.assert_array_equal(a, b)
    assert a.min() >= -0.1 and a.max() < 0.1
    assert abs(a.mean()) < 0.01
    c = synthetic.uniform(7, 1, 10000, -0.1, 0.1)
    assert not np.array_equal(a, c)


def test_recipes():
    phi = synthetic.allen_cahn_init((128, 128))
    assert phi.dtype == np.float32 and phi.shape == (128, 128)
    assert np.abs(phi).max() <= 0.1
    ch = synthetic.cahn_hilliard_init((64, 64))
    assert abs(ch.astype(np.float64).mean()) < 1e-8
    u, v = synthetic.gray_scott_init((32, 32, 32), seed=3, n_seeds=4, side=8)
    assert u.dtype == np.float32 and v.dtype == np.float32
    # outside the seeds the state is exactly the fixed point (noise is multiplicative)
    outside = v == 0
    assert outside.any() and np.all(u[outside] >= 0.99) and np.all(u[outside] <= 1.01)
    assert np.all(v >= 0) and np.all(v <= 0.25 * 1.01 + 1e-7)
    specs = synthetic.batch_instances()
    sides = np.array([s["n"] for s in specs])
    assert len(specs) == 512 and sides.min() >= 64 and sides.max() <= 512
    assert all(0.02 <= s["F"] < 0.06 and 0.045 <= s["k"] < 0.07 for s in specs)
