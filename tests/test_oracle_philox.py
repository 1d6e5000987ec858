"""Pins of the oracle's Philox4x64-10 against numpy's independent
implementation of the same published generator (Salmon et al., SC'11)."""
import numpy as np
import pytest


def numpy_block(ctr, key):
    # numpy's bit generator advances its 256-bit counter by one before it
    # produces a block, so start it one below the counter we want
    c = int(ctr[0]) | (int(ctr[1]) << 64) | (int(ctr[2]) << 128) | (int(ctr[3]) << 192)
    c = (c - 1) % (1 << 256)
    words = [(c >> (64 * i)) & ((1 << 64) - 1) for i in range(4)]
    bg = np.random.Philox(counter=np.array(words, dtype=np.uint64),
                          key=np.array([int(k) for k in key], dtype=np.uint64))
    return [int(v) for v in bg.random_raw(4)]


@pytest.mark.parametrize("seed", range(8))
def test_philox_matches_numpy(oracle_mod, seed):
    rng = np.random.default_rng(1000 + seed)
    ctr = [int(v) for v in rng.integers(0, 2 ** 63, size=4, dtype=np.uint64)]
    key = [int(v) for v in rng.integers(0, 2 ** 63, size=2, dtype=np.uint64)]
    assert oracle_mod.philox(ctr, key) == numpy_block(ctr, key)


def test_philox_counter_layout_examples(oracle_mod):
    # the counters the method uses: (id, substep, step, stream) under (seed, 0)
    for ctr in ([0, 0, 0, 3], [12345, 9, 3599, 1], [2 ** 40 + 7, 0, 0, 3]):
        assert oracle_mod.philox(ctr, [42, 0]) == numpy_block(ctr, [42, 0])


def test_u01_open_interval(oracle_mod):
    lo = oracle_mod.u01(0)
    hi = oracle_mod.u01(2 ** 64 - 1)
    assert 0.0 < lo < 1e-15
    assert 1.0 - 1e-15 < hi < 1.0
    # 52 random bits plus one half: evenly spaced, exactly representable
    assert oracle_mod.u01(1 << 12) - lo == pytest.approx(2.0 ** -52, rel=0, abs=0)
