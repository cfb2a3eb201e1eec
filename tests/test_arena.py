"""Host logic of the batch arena (include/lbdp_batch.h): first fit over
256-byte granules with coalescing frees, checked against an independent
brute-force model of the same policy on random alloc/free sequences.  No GPU:
the arena is host bookkeeping only."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def lbdp():
    from paper_2202_01631_gb300 import build
    build.build()
    from paper_2202_01631_gb300 import lbdp as mod
    return mod


class GranuleModel:
    """A bitmap of 256-byte granules; allocation takes the lowest run of free
    granules long enough (first fit)."""

    def __init__(self, cap):
        self.n = cap // 256
        self.used = np.zeros(self.n, dtype=bool)
        self.held = {}

    def alloc(self, nbytes):
        g = -(-nbytes // 256)
        run = 0
        for i in range(self.n):
            run = run + 1 if not self.used[i] else 0
            if run == g:
                start = i - g + 1
                self.used[start:i + 1] = True
                self.held[start * 256] = g
                return start * 256
        return None

    def free(self, off):
        g = self.held.pop(off)
        self.used[off // 256:off // 256 + g] = False

    def stats(self):
        runs, run, big = 0, 0, 0
        for u in self.used:
            if not u:
                run += 1
                big = max(big, run)
            else:
                runs += run > 0
                run = 0
        runs += run > 0
        return int(self.used.sum()) * 256, big * 256, runs


def test_first_fit_and_coalescing(lbdp):
    a = lbdp.lb_arena_create(10 * 256 + 100)   # rounded down to 10 granules
    try:
        assert lbdp.lb_arena_stats(a) == (0, 2560, 1)
        o = [lbdp.lb_arena_alloc(a, n) for n in (256, 300, 256)]
        assert o == [0, 256, 768]
        lbdp.lb_arena_free(a, 256)                # hole of 2 granules at 256
        assert lbdp.lb_arena_stats(a) == (512, 1536, 2)
        assert lbdp.lb_arena_alloc(a, 200) == 256  # first fit takes the hole
        lbdp.lb_arena_free(a, 0)
        lbdp.lb_arena_free(a, 256)                # merges with the range at 0
        assert lbdp.lb_arena_stats(a) == (256, 1536, 2)
        with pytest.raises(lbdp.LbError) as e:
            lbdp.lb_arena_alloc(a, 1537)
        assert e.value.status == -2               # LB_ERR_NOMEM, nothing changed
        assert lbdp.lb_arena_stats(a) == (256, 1536, 2)
        lbdp.lb_arena_free(a, 768)
        assert lbdp.lb_arena_stats(a) == (0, 2560, 1)
        with pytest.raises(lbdp.LbError):
            lbdp.lb_arena_free(a, 768)            # not held
        with pytest.raises(lbdp.LbError):
            lbdp.lb_arena_alloc(a, 0)
    finally:
        lbdp.lb_arena_destroy(a)
    with pytest.raises(lbdp.LbError):
        lbdp.lb_arena_create(255)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_matches_brute_force_model(lbdp, seed):
    rng = np.random.default_rng(seed)
    cap = 64 * 256
    a = lbdp.lb_arena_create(cap)
    m = GranuleModel(cap)
    live = []
    try:
        for _ in range(400):
            if live and rng.random() < 0.45:
                off = live.pop(int(rng.integers(len(live))))
                lbdp.lb_arena_free(a, off)
                m.free(off)
            else:
                n = int(rng.integers(1, 9 * 256))
                want = m.alloc(n)
                if want is None:
                    with pytest.raises(lbdp.LbError):
                        lbdp.lb_arena_alloc(a, n)
                else:
                    assert lbdp.lb_arena_alloc(a, n) == want
                    live.append(want)
            assert lbdp.lb_arena_stats(a) == m.stats()
    finally:
        lbdp.lb_arena_destroy(a)
