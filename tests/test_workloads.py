"""The shared input generators: the C generator equals the numpy one, and
the value recipes and configuration shapes hold."""
import numpy as np

import workloads as wl


def test_c_generator_matches_numpy():
    for seed in (0, 1, 12345):
        np.testing.assert_array_equal(wl.draws(seed, 1000, start=17), wl.draws_numpy(seed, 1000, start=17))
        np.testing.assert_array_equal(wl.uniform(seed, (10, 7)).reshape(-1, order="F"),
                                      wl.uniform_numpy(seed, 70))
        np.testing.assert_array_equal(wl.integers(seed, (70,)), wl.integers_numpy(seed, 70))


def test_value_ranges():
    u = wl.uniform(0, (100000,))
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.02
    k = wl.integers(0, (100000,))
    assert set(np.unique(k)) == set(range(-3, 4))


def test_counter_based_offsets():
    full = wl.uniform(3, (1000,))
    np.testing.assert_array_equal(full[400:], wl.uniform(3, (600,), start=400))


def test_random_coefficients():
    for d in (3, 4):
        c = wl.random_coef(d, 100)
        assert c.shape == (1, 6 if d == 3 else 24)
        assert set(np.unique(c)) <= {-2.0, -1.0, 1.0, 2.0, 4.0}


def test_table2_shapes():
    for r in wl.TABLE2_ROWS:
        c = wl.table2(r)
        d = wl.table2_dim(r)
        assert c.shape[1] == (6 if d == 3 else 24)
        for f in c:
            assert f[0] == 2.0 and set(np.unique(f[1:])) <= {0.0, -1.0}
    assert wl.table2(1).shape == (2, 6) and wl.table2(5).shape == (3, 24)


def test_config_shapes():
    assert wl.config2().spec == (48, 48, 48) and wl.config2().O == 16
    blocks = wl.config4_blocks()
    assert len(blocks) == 64
    assert all(16 <= b.spec[0] <= 40 and 6 <= b.O <= 14 for b in blocks)
