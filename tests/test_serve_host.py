"""Host-side pieces of the serving loop that need no GPU."""
import pytest

torch = pytest.importorskip("torch")


def test_arena_first_fit_and_coalescing():
    from paper_1509_03838_gb300.serve import Arena
    a = Arena(4096, "cpu")
    x = a.alloc(1000)          # rounds up to 1024
    y = a.alloc(1000)
    z = a.alloc(2048)
    assert x == (0, 1024) and y == (1024, 1024) and z == (2048, 2048)
    assert a.alloc(1) is None and a.used == 4096 == a.peak
    a.release(*y)
    assert a.alloc(2048) is None     # only 1024 contiguous bytes are free
    a.release(*x)
    assert a.free == [(0, 2048)]     # neighbours coalesce
    assert a.alloc(2048) == (0, 2048)
    a.release(0, 2048)
    a.release(*z)
    assert a.free == [(0, 4096)] and a.used == 0


def test_serve_spec_is_seeded_and_shaped():
    from paper_1509_03838_gb300 import synth
    s1 = synth.serve_spec(seed=3, n_jobs=5000)
    s2 = synth.serve_spec(seed=3, n_jobs=5000)
    assert (s1.arrival_s == s2.arrival_s).all()
    gaps = s1.arrival_s[1:] - s1.arrival_s[:-1]
    assert abs(gaps.mean() - 1 / 20000.0) < 0.1 / 20000.0   # Poisson, 20k/s
    b = s1.batch
    assert b.M.min() >= 3 and b.M.max() <= 6
    assert b.N.min() >= 1 << 12 and b.N.max() <= 1 << 20
    assert b.K.min() >= 16 and b.K.max() <= 512
    assert ((b.failed >= 0) == s1.inject).all()
    assert 0.08 < s1.inject.mean() < 0.12
