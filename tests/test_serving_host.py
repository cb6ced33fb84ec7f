"""Host logic of the serving loop, without a GPU: the admission arena (the
first-fit sub-allocator that decides whether a request's device block fits)
against an independent model, and the server's config validation."""
import numpy as np
import pytest

from paper_2201_02309_b300 import build, native


@pytest.fixture(scope="module")
def lib():
    build.build()
    return native


class ModelArena:
    """First fit over a sorted free list, blocks rounded up to 256, merge on free."""

    def __init__(self, size):
        self.size = size
        self.free = [(0, size)]  # sorted (offset, length)
        self.used = {}

    def alloc(self, n):
        n = max(n, 1)
        n = -(-n // 256) * 256
        for i, (o, l) in enumerate(self.free):
            if l >= n:
                if l == n:
                    del self.free[i]
                else:
                    self.free[i] = (o + n, l - n)
                self.used[o] = n
                return o
        return -1

    def release(self, o):
        n = self.used.pop(o)
        self.free.append((o, n))
        self.free.sort()
        merged = []
        for a, l in self.free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1] = (merged[-1][0], merged[-1][1] + l)
            else:
                merged.append((a, l))
        self.free = merged

    def largest(self):
        return max((l for _, l in self.free), default=0)


def test_arena_matches_model_on_random_traffic(lib):
    rng = np.random.default_rng(11)
    size = 1 << 20
    a = lib.katsevich_arena_create(size)
    m = ModelArena(size)
    live = []
    try:
        for step in range(4000):
            if live and (rng.random() < 0.45 or len(live) > 60):
                o = live.pop(int(rng.integers(len(live))))
                lib.katsevich_arena_free(a, o)
                m.release(o)
            else:
                n = int(rng.choice([1, 255, 256, 257, 1000, 4096, 30000, 100000, 300000]))
                got, want = lib.katsevich_arena_alloc(a, n), m.alloc(n)
                assert got == want, (step, n, got, want)
                if got >= 0:
                    live.append(got)
            assert lib.katsevich_arena_largest_free(a) == m.largest()
            assert lib.katsevich_arena_in_use(a) == sum(m.used.values())
        for o in live:
            lib.katsevich_arena_free(a, o)
        # everything merged back into one block
        assert lib.katsevich_arena_largest_free(a) == size
        assert lib.katsevich_arena_in_use(a) == 0
    finally:
        lib.katsevich_arena_destroy(a)


def test_arena_blocks_are_disjoint_and_aligned(lib):
    a = lib.katsevich_arena_create(10_000)
    try:
        offs = [lib.katsevich_arena_alloc(a, n) for n in (1, 300, 2000, 5000)]
        assert all(o % 256 == 0 for o in offs)
        spans = sorted((o, o + -(-max(n, 1) // 256) * 256) for o, n in zip(offs, (1, 300, 2000, 5000)))
        assert all(e <= s for (_, e), (s, _) in zip(spans, spans[1:]))
        assert lib.katsevich_arena_alloc(a, 10_000) == -1  # does not fit: the request waits
        with pytest.raises(native.KatsevichError):
            lib.katsevich_arena_free(a, 128)  # not a block
        lib.katsevich_arena_free(a, offs[1])
        with pytest.raises(native.KatsevichError):
            lib.katsevich_arena_free(a, offs[1])  # double free
    finally:
        lib.katsevich_arena_destroy(a)


def test_server_config_is_validated_before_any_device_call(lib):
    for bad in [dict(arena_bytes=0, plan_cache_bytes=1, slots=2),
                dict(arena_bytes=1 << 20, plan_cache_bytes=-1, slots=2),
                dict(arena_bytes=1 << 20, plan_cache_bytes=1, slots=0),
                dict(arena_bytes=1 << 20, plan_cache_bytes=1, slots=65),
                dict(arena_bytes=1 << 20, plan_cache_bytes=1, slots=2, max_bypass=-1)]:
        with pytest.raises(native.KatsevichError) as e:
            native.katsevich_server_create(**bad)
        assert e.value.status == native.KATS_EINVAL
