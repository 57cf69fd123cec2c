"""Host logic of the autotuner: cache keys bucket the problem shape, and a
stored entry round-trips to launch options (no GPU needed)."""
from paper_2607_25388_b300 import autotune as A


def test_keys_bucket_horizon_and_opponents():
    info = (148, "B300")
    assert A.key(10, 60, 16384, 5, info) == A.key(10, 50, 16384, 5, info)     # T 49..64 share a bucket
    assert A.key(10, 60, 16384, 5, info) != A.key(10, 65, 16384, 5, info)
    assert A.key(5, 60, 4096, 3, info) == A.key(8, 60, 4096, 3, info)         # 4..9 opponents share one
    assert A.key(3, 60, 4096, 3, info) != A.key(5, 60, 4096, 3, info)
    assert A.key(10, 60, 16384, 5, info) != A.key(10, 60, 16384, 5, (132, "B300"))


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    info = (148, "B300")
    assert A.lookup(10, 60, 16384, 5, path, info) is None
    A.store(10, 60, 16384, 5, dict(block=128, samples_per_thread=2, ctas_per_sm=3, ms=0.8), path, info)
    o = A.lookup(10, 60, 16384, 5, path, info)
    assert (o.block, o.samples_per_thread, o.ctas_per_sm) == (128, 2, 3)
    A.store(2, 30, 4096, 3, dict(block=256, samples_per_thread=1, ctas_per_sm=0, ms=0.1), path, info)
    assert A.lookup(10, 60, 16384, 5, path, info).block == 128


class _FakeBatch:
    def __init__(self, races, K=4096, L=3):
        self.races = races
        self.agents = sum(r["n_v"] for r in races)
        self.K, self.L = K, L


def test_batch_keys_and_round_trip(tmp_path):
    info = (148, "B300")
    a = _FakeBatch([dict(n_v=2, T=30), dict(n_v=10, T=80)])
    b = _FakeBatch([dict(n_v=2, T=31), dict(n_v=10, T=79)])
    c = _FakeBatch([dict(n_v=3, T=30), dict(n_v=10, T=80)])
    assert A.key_batch(a, info) == A.key_batch(b, info)      # same size, vehicles and extremes
    assert A.key_batch(a, info) != A.key_batch(c, info)      # one more vehicle
    path = str(tmp_path / "tune.json")
    assert A.lookup_batch(a, path, info) is None
    A._store(A.key_batch(a, info), dict(block=128, samples_per_thread=3, ctas_per_sm=0, schedule=2, ms=1.0), path)
    o = A.lookup_batch(b, path, info)
    assert (o.block, o.samples_per_thread, o.ctas_per_sm, o.schedule) == (128, 3, 0, 2)


def test_search_space_and_tiles_per_response():
    c = list(A._candidates())
    assert len(c) == len(set(c)) == len(A.SHAPES) * len(A.CTAS) * len(A.SCHEDULES)
    assert {s for *_, s in c} == {1, 2}
    assert A._tiles(4096, 128, 3) == 11 and A._tiles(4096, 128, 2) == 16 and A._tiles(4096, 256, 1) == 16
    assert A._tiles(1000, 128, 1) == 8 and A._tiles(4096, 128, 0) is None and A._tiles(4096, 0, 0) is None
