"""GPU parity of the further LSB operations and of corruption detection:
circular convolution and cross-correlation (Eq. 2), the inner product, and
detection of a corrupted stream with all M outputs present (Remark 4)."""
import numpy as np
import pytest

from paper_1509_03838_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ne():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_03838_gb300 import build, ne as nemod
    build.build()
    return nemod


def dev(a, dtype=torch.int64):
    return torch.from_numpy(np.asarray(a, dtype=np.int64)).to(dtype).cuda()


KIND_CASES = [
    # kind, w, M, N, K, data bits, declared
    ("circular", 64, 4, 5000, 64, 15, True),
    ("circular", 64, 3, 1600, 1600, 10, False),   # K = N
    ("circular", 32, 3, 777, 16, 7, True),
    ("xcorr", 64, 4, 4000, 100, 15, True),
    ("xcorr", 64, 5, 9, 200, 12, False),          # N < K
    ("xcorr", 32, 3, 3100, 33, 7, True),
]


@pytest.mark.parametrize("case", KIND_CASES)
def test_conv_kinds_match_oracle(ne, orc, case):
    kind, w, M, N, K, bits, declared = case
    gen = synth.rng(N + K + M)
    x = synth.uniform_int(gen, (M, N), -(1 << bits), 1 << bits)
    g = synth.uniform_int(gen, (K,), -(1 << 15), 1 << 15)
    dt = torch.int32 if w == 32 else torch.int64
    op = orc.conv_circular if kind == "circular" else orc.xcorr
    code = ne.NE_CONV_CIRCULAR if kind == "circular" else ne.NE_CONV_XCORR
    expect = op(x, g, w, strict=False)
    y = torch.zeros(expect.shape, dtype=dt, device="cuda")
    ne.ne_conv_kind(dev(x, dt), dev(g, torch.int32), y, kind=code,
                    x_range=(-(1 << bits), (1 << bits) - 1) if declared else None)
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy().astype(np.int64), expect)


@pytest.mark.parametrize("kind", ["circular", "xcorr"])
def test_conv_kinds_on_entangled_streams_recover(ne, orc, kind):
    M, w = 4, 64
    p = ne.ne_params(M, w)
    gen = synth.rng(3)
    c = synth.uniform_int(gen, (M, 3000), -(1 << 15), 1 << 15)
    g = synth.uniform_int(gen, (64,), -(1 << 15), 1 << 15)
    op = orc.conv_circular if kind == "circular" else orc.xcorr
    code = ne.NE_CONV_CIRCULAR if kind == "circular" else ne.NE_CONV_XCORR
    plain = op(c, g, w)
    eps = dev(c)
    ne.ne_entangle(eps, l=p.l)
    f = (1 << p.l) + 1
    for r in range(M):
        delta = torch.zeros(plain.shape, dtype=torch.int64, device="cuda")
        ne.ne_conv_kind(eps, dev(g, torch.int32), delta, kind=code,
                        x_range=(-(1 << 15) * f, ((1 << 15) - 1) * f),
                        live_mask=((1 << M) - 1) & ~(1 << r))
        d = torch.empty_like(delta)
        ne.ne_recover(delta, d, l=p.l, failed=r)
        torch.cuda.synchronize()
        assert np.array_equal(d.cpu().numpy(), plain), r


@pytest.mark.parametrize("w,M,N", [(64, 4, 1 << 20), (64, 6, 12345), (32, 3, 5000)])
def test_inner_product_protected(ne, orc, w, M, N):
    p = ne.ne_params(M, w)
    gen = synth.rng(N)
    bits = 3 if w == 32 else 12  # N * 2^(2 bits) within the exact range
    assert N * (1 << (2 * bits)) <= p.d_max_exact
    c = synth.uniform_int(gen, (M, N), -(1 << bits), 1 << bits)
    g = synth.uniform_int(gen, (N,), -(1 << bits), 1 << bits)
    dt = torch.int32 if w == 32 else torch.int64
    eps = dev(c, dt)
    ne.ne_entangle(eps, l=p.l)
    for r in range(M):
        y = torch.full((M, 1), 7, dtype=dt, device="cuda")
        ne.ne_dot(eps, dev(g, dt), y, live_mask=((1 << M) - 1) & ~(1 << r))
        torch.cuda.synchronize()
        e_or = orc.dot(orc.entangle(c, w, p.l), g, w)
        got = y.cpu().numpy().astype(np.int64)[:, 0]
        for m in range(M):
            if m != r:
                assert got[m] == e_or[m]
        d = torch.empty_like(y)
        ne.ne_recover(y, d, l=p.l, failed=r)
        torch.cuda.synchronize()
        assert d.cpu().numpy().astype(np.int64)[:, 0].tolist() == orc.dot(c, g, w).tolist()


@pytest.mark.parametrize("w,M", [(64, 3), (64, 4), (64, 8), (32, 4), (64, 11)])
def test_detect_matches_oracle(ne, orc, w, M):
    p = ne.ne_params(M, w)
    gen = synth.rng(w * M + 1)
    Nout = 50000
    d_true = synth.uniform_int(gen, (M, Nout), -p.d_max_paper, p.d_max_paper + 1)
    delta = orc.entangle(d_true, w, p.l)
    dt = torch.int32 if w == 32 else torch.int64
    # clean: nothing flagged, outputs recovered
    out = torch.empty((M, Nout), dtype=dt, device="cuda")
    count, pos = ne.ne_detect(dev(delta, dt), l=p.l, d_max=p.d_max_paper,
                              d=out, max_positions=16)
    torch.cuda.synchronize()
    assert int(count.item()) == 0
    assert np.array_equal(out.cpu().numpy().astype(np.int64), d_true)
    # corrupt one stream at seeded columns (every stream gets some)
    bad_cols = np.sort(gen.choice(Nout, size=40, replace=False))
    corrupted = delta.copy()
    for i, n in enumerate(bad_cols):
        q = i % M
        flip = int(gen.integers(1, 1 << (w - 1)))
        v = (int(corrupted[q, n]) ^ flip) & ((1 << w) - 1)
        corrupted[q, n] = v - (1 << w) if v >> (w - 1) else v
    flags, _ = orc.detect(corrupted, w, p.l, p.d_max_paper)
    assert np.flatnonzero(flags).tolist() == bad_cols.tolist()
    count, pos = ne.ne_detect(dev(corrupted, dt), l=p.l, d_max=p.d_max_paper,
                              max_positions=64)
    torch.cuda.synchronize()
    assert int(count.item()) == len(bad_cols)
    assert sorted(pos.cpu().numpy()[:len(bad_cols)].tolist()) == bad_cols.tolist()
