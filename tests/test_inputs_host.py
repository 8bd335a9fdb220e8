"""The seeded input generators (no GPU): SplitMix64 against its published
output for seed 0, the ranges and determinism of the drop and sweep draws, and
the non-overlap rule of the multi-drop workload."""
import itertools

import numpy as np

from paper_0710_5470_gb300 import inputs


def test_splitmix64_reference_outputs():
    # the first outputs of SplitMix64 (Steele, Lea & Flood 2014) from state 0
    r = inputs.SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_and_integer_ranges():
    r = inputs.SplitMix64(7)
    u = [r.uniform(-2.0, 3.0) for _ in range(20000)]
    assert min(u) >= -2.0 and max(u) < 3.0 and abs(np.mean(u) - 0.5) < 0.05
    k = [r.integer(3, 6) for _ in range(4000)]
    assert set(k) == {3, 4, 5, 6}


def test_random_drops_do_not_overlap():
    for seed in range(20):
        shape = (512, 512)
        c, R, rejects = inputs.random_drops(seed, shape)
        assert 1 <= len(R) <= 8 and all(20.0 <= x <= 80.0 for x in R)
        for (c1, r1), (c2, r2) in itertools.combinations(zip(c, R), 2):
            d = [min(abs(a - b), n - abs(a - b)) for a, b, n in zip(c1, c2, shape)]
            assert np.hypot(*d) >= r1 + r2 + 4 * 2.0
        assert inputs.random_drops(seed, shape) == (c, R, rejects)


def test_sweep_instances_ranges_and_determinism():
    s = inputs.sweep_instances(seed=0, count=256)
    assert s == inputs.sweep_instances(seed=0, count=256)
    assert s != inputs.sweep_instances(seed=1, count=256)
    for d in s:
        assert 64 <= d["n"] <= 384 and isinstance(d["n"], int)
        assert 0.50 <= d["T"] < 0.56 and 0.002 <= d["kappa"] < 0.03 and 0.6 <= d["tau"] < 1.5
        assert 0.15 * d["n"] <= d["R"] < 0.35 * d["n"]
    assert sum(d["n"] ** 2 for d in s) == 15578749
