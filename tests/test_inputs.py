"""Seeded input generators: SplitMix64 against its published outputs."""
import os

import numpy as np

import vx_inputs as vi

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")


def test_splitmix64_reference_vectors():
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        seed, *words = line.split()
        got = vi.SplitMix64(int(seed)).next_u64(3)
        assert [int(w, 16) for w in words] == [int(x) for x in got]


def test_uniform_range_and_streams():
    u = vi.SplitMix64(7).uniform(10000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01
    a = vi.SplitMix64(7)
    first = a.uniform(5)
    second = a.uniform(5)
    both = vi.SplitMix64(7).uniform(10)
    assert np.array_equal(np.concatenate([first, second]), both)
    assert not np.array_equal(vi.substream(3, 0).uniform(4), vi.substream(3, 1).uniform(4))


def test_workload_shapes():
    c1 = vi.tissue_c1()
    assert c1["seeds"].shape == (100, 2) and c1["lam"].shape == (300,)
    assert c1["seeds"].min() >= 0 and c1["seeds"].max() < 1
    b = vi.batch_c3(8)
    assert all(200 <= t["n"] <= 5000 for t in b)
    assert all(3.5 <= t["P0"] <= 4.0 for t in b)
