"""The seeded input generators (paper_2104_07146_gb300/synth.py) on the CPU:
the stream is SplitMix64 (its published first output for state 0 and a
pure-integer restatement), it is counter-based (any slice without the
prefix), and the point sets have the stated shapes: uniform points in the
unit cube, the uniform / Gaussian-blob mixture clipped to [0, 1]^d with the
uniform points first, and sorted collinear points."""
import numpy as np

from paper_2104_07146_gb300 import synth

_M = (1 << 64) - 1


def _mix(z):
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M
    return z ^ (z >> 31)


def test_splitmix64_published_first_output():
    # SplitMix64 from state 0: first output 0xe220a8397b1dcdaf; seed 0 has mix(0) = 0
    assert int(synth.uint64_stream(0, 1)[0]) == 0xE220A8397B1DCDAF


def test_stream_matches_an_integer_restatement_and_is_counter_based():
    for seed in (1, 1001, 2 ** 40 + 7):
        base = _mix(seed & _M)
        ref = [_mix((base + (i + 1) * 0x9E3779B97F4A7C15) & _M) for i in range(50)]
        assert [int(v) for v in synth.uint64_stream(seed, 50)] == ref
        assert np.array_equal(synth.uniform(seed, 20, offset=30), synth.uniform(seed, 50)[30:])


def test_uniform_and_normal_moments():
    u = synth.uniform(3, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.005
    z = synth.normal(4, 200001)
    assert z.shape == (200001,)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.01
    assert abs(np.mean(z ** 4) - 3.0) < 0.05                    # Gaussian kurtosis


def test_point_set_shapes():
    p = synth.locations_uniform(1000, 3, seed=5)
    assert p.shape == (1000, 3) and p.min() >= 0.0 and p.max() < 1.0
    n = 10000
    b = synth.locations_blobs(n, 2, 0.3, 8, 0.03, seed=6)
    nb = 3000
    assert b.shape == (n, 2) and b.min() >= 0.0 and b.max() <= 1.0
    assert np.array_equal(b[:n - nb], synth.locations_uniform(n - nb, 2, seed=6))
    # the blob points gather around 8 centres in [0.1, 0.9]^2 with sd 0.03
    centres = 0.1 + 0.8 * synth.uniform(6 + 0x1000, 16).reshape(8, 2)
    dist = np.min(np.linalg.norm(b[n - nb:, None, :] - centres[None], axis=2), axis=1)
    assert np.mean(dist < 0.15) > 0.999
    assert 0.025 < np.sqrt(np.mean(dist ** 2) / 2) < 0.035
    c = synth.locations_collinear(500, seed=7)
    assert np.all(np.diff(c[:, 0]) >= 0) and np.all(c[:, 1] == 0.5)


def test_workload_recipes():
    m = synth.MEDIUM
    assert (m["n"], m["leaf"], m["aca_eps"], m["frac_blob"]) == (65536, 64, 1e-6, 0.3)
    assert synth.medium_locations(1000).shape == (1000, 2)
