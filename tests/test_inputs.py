"""Seeded descriptor generator: published SplitMix64 vector and workload shapes."""
import numpy as np

from paper_2412_01138_gb300 import inputs as I


def test_splitmix64_published_vector():
    r = I.SplitMix64(1234567)
    assert [r.next_u64() for _ in range(5)] == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                                                4593380528125082431, 16408922859458223821]


def test_random_nodes_sorted_distinct():
    for seed in range(50):
        c = I.draw_random_nodes(4, seed)
        assert list(c) == sorted(c) and min(np.diff(c)) >= I.MIN_NODE_GAP and 0 <= c[0] and c[-1] < 1


def test_workload_shapes():
    c1, c2, c3, c5 = I.config1(), I.config2(), I.config3(), I.config5()
    assert (c1.ndof, c1.N, c1.M, c1.q, c1.p) == (63, 8, 16, 2, 2)
    assert (c2.ndof, c2.N, c2.M, c2.q, c2.p, c2.R) == (255 ** 2, 32, 64, 4, 2, 9)
    assert (c3.ndof, c3.N, c3.M, c3.R) == (127 ** 3, 64, 32, 17)
    assert (c5.ndof, c5.N, c5.M, c5.R, c5.T) == (511 ** 2, 128, 32, 12, 2.0)
    batch = I.config4()
    assert len(batch) == 512
    assert all(31 <= v <= 511 for p in batch for v in p.n)
    assert all(16 <= p.N <= 64 and 5 <= p.R <= 17 for p in batch)
