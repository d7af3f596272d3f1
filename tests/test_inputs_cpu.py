"""The seeded input generators shared by the oracle and the CUDA path (no GPU).

The generator is SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014) used as a counter-based stream: output i of stream (seed, field) is the SplitMix64
finaliser of key + i * 0x9E3779B97F4A7C15, the i-th output of SplitMix64 started at state `key`.
The pins below check the finaliser against SplitMix64's published reference outputs, then the
properties the workloads rely on: the mapping to [0, 1), counter addressing, uniformity, the
truncated normal, and the documented ranges of the benchmark's run mixes.
"""
import numpy as np
import pytest

from paper_2312_05410_gb300 import inputs as I

# The first five outputs of SplitMix64 started at state 1234567, as printed by the algorithm's public
# reference implementation.
SPLITMIX64_1234567 = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
                      16408922859458223821]


def test_finaliser_reproduces_the_splitmix64_reference_outputs():
    state = 1234567
    scalar = [I._mix64_scalar(state + i * I.GOLDEN_GAMMA) for i in range(1, 6)]
    assert scalar == SPLITMIX64_1234567
    z = np.array([(state + i * I.GOLDEN_GAMMA) & I.MASK64 for i in range(1, 6)], dtype=np.uint64)
    assert [int(v) for v in I._mix64(z)] == SPLITMIX64_1234567


def test_uniform01_is_the_top_53_bits_of_the_stream():
    key = I.stream_key(7, 2)
    u = I.uniform01(7, 2, 4)
    for i, x in enumerate(u, start=1):
        bits = I._mix64_scalar(key + i * I.GOLDEN_GAMMA) >> 11
        assert x == bits / 2.0 ** 53
    assert np.all((u >= 0.0) & (u < 1.0))


def test_counters_address_one_stream_and_streams_differ():
    full = I.uniform01(3, 5, 1000)
    np.testing.assert_array_equal(I.uniform01(3, 5, 400, offset=600), full[600:])
    np.testing.assert_array_equal(I.uniform01(3, 5, 1000), full)  # deterministic
    assert not np.array_equal(I.uniform01(3, 6, 1000), full)      # another field
    assert not np.array_equal(I.uniform01(4, 5, 1000), full)      # another seed


def test_uniform01_is_uniform():
    from scipy import stats
    u = I.uniform01(11, 1, 200000)
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    assert abs(u.mean() - 0.5) < 3 * (1 / np.sqrt(12 * u.size)) * 2
    # no lag-one correlation
    assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 0.01


def test_truncated_normal_stays_in_bounds_and_is_symmetric():
    from scipy import stats
    g = I.truncated_normal(I.uniform01(2, 2, 100000), bound=2.0)
    assert g.min() >= -2.0 and g.max() <= 2.0
    assert abs(g.mean()) < 0.02
    # variance of the standard normal truncated to [-2, 2]
    a, b = -2.0, 2.0
    var = stats.truncnorm(a, b).var()
    assert abs(g.var() - var) < 0.02


def test_ensemble_mix_has_the_documented_ranges():
    ms = I.ensemble_members(64, seed=3)
    assert len(ms) == 64
    sides = {m["spec"].nx for m in ms}
    assert sides <= {128, 192, 256, 384, 512} and len(sides) == 5
    assert all(m["spec"].nx == m["spec"].ny for m in ms)
    assert all(0.1 <= m["v_mag"] <= 0.9 for m in ms)
    assert all(0.3 <= m["spec"].c_inc <= 0.7 for m in ms)
    again = I.ensemble_members(64, seed=3)
    assert [(m["spec"].nx, m["v_mag"]) for m in again] == [(m["spec"].nx, m["v_mag"]) for m in ms]


@pytest.mark.parametrize("seed", [5, 11])
def test_hybrid_batch_has_the_documented_ranges(seed):
    ms = I.hybrid_members(16, 256, seed=seed)
    assert len(ms) == 16
    assert all(m["spec"].nx == 256 and m["spec"].ny == 256 for m in ms)
    assert all(0.1 <= m["v_mag"] <= 0.9 for m in ms)
    assert all(0.3 <= m["c_inc"] <= 0.7 for m in ms)
    # the surrogate's training batch (seed 11) and the benchmark's batch (seed 5) are different runs
    other = I.hybrid_members(16, 256, seed=16 - seed)
    assert [m["v_mag"] for m in other] != [m["v_mag"] for m in ms]
