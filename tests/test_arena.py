"""The workspace arena's bookkeeping (host only, no GPU): first-fit
placement, alignment, coalescing of freed neighbours, refusal when no free
range fits, and agreement with a plain interval model over a long random
sequence of allocations and frees."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def G():
    from paper_2404_16322_gb300 import build
    build.build()
    import paper_2404_16322_gb300 as G
    return G


def test_first_fit_alignment_and_coalescing(G):
    a = G.Arena(1000, 64)  # usable: 960 bytes
    assert a.size == 960 and a.largest_free == 960
    x = a.alloc(1)
    y = a.alloc(65)
    z = a.alloc(200)
    assert (x, y, z) == (0, 64, 192)  # 1 -> 64, 65 -> 128
    assert a.used == 64 + 128 + 256
    assert a.alloc(960) == -1  # does not fit any more
    a.free(y)
    assert a.alloc(100) == 64  # first fit reuses the hole
    a.free(64)
    a.free(x)
    a.free(z)  # x, the hole and z merge back into one range
    assert a.used == 0 and a.largest_free == 960
    with pytest.raises(Exception):
        a.free(12345)
    a.close()


def _model_alloc(free, need):
    for i, (o, n) in enumerate(free):
        if n >= need:
            if n == need:
                free.pop(i)
            else:
                free[i] = (o + need, n - need)
            return o
    return -1


def _model_free(free, o, n):
    free.append((o, n))
    free.sort()
    out = []
    for f in free:
        if out and out[-1][0] + out[-1][1] == f[0]:
            out[-1] = (out[-1][0], out[-1][1] + f[1])
        else:
            out.append(f)
    free[:] = out


def test_random_sequence_matches_an_interval_model(G):
    rng = np.random.default_rng(5)
    align, size = 256, 1 << 20
    a = G.Arena(size, align)
    free = [(0, size)]
    live = {}
    for _ in range(3000):
        if live and rng.random() < 0.45:
            o = int(rng.choice(sorted(live)))
            a.free(o)
            _model_free(free, o, live.pop(o))
        else:
            nb = int(rng.integers(1, 1 << 16))
            need = -(-nb // align) * align
            got = a.alloc(nb)
            want = _model_alloc(free, need)
            assert got == want
            if got >= 0:
                live[got] = need
        assert a.used == sum(live.values())
        assert a.largest_free == max([n for _, n in free], default=0)
    a.close()
