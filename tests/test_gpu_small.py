"""Small jobs (config 1 shape: M = 3 int32 streams, N = 4096, K = 16): the
prepared call (ne.ProtectedConvCall, arguments converted once) gives the
oracle's convolution of the raw inputs under every failure, on consecutive
calls that change only the failure; and the dispatch that sends small jobs
to the multiply-add kernels gives the same outputs as the tensor-core forms
(Eq. 9, Eq. 16-19)."""
import numpy as np
import pytest

from oracle_par import conv_par
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


def _modes(ne, M):
    return [(ne.NE_FAIL_NONE, -1)] + [(fm, r) for fm in (ne.NE_FAIL_SKIP,
                                                         ne.NE_FAIL_DROP)
                                      for r in range(M)]


def test_prepared_call_every_failure(ne, orc):
    j = synth.small_job(seed=1)
    p = ne.ne_choose_width(j.M, j.K, j.bound_c, j.bound_g)
    assert p.w == 32
    expect = conv_par(orc, j.c, j.g, 32)
    c = torch.from_numpy(j.c.astype(np.int32)).cuda()
    g = torch.from_numpy(j.g.astype(np.int32)).cuda()
    d = torch.full((j.M, j.N + j.K - 1), 9, dtype=torch.int32, device="cuda")
    call = ne.ProtectedConvCall(c, g, d, l=p.l, c_range=j.c_range,
                                max_abs_g=j.bound_g)
    for fm, r in _modes(ne, j.M) * 2:
        d.fill_(9)
        call(failed=r, fail_mode=fm)
        torch.cuda.synchronize()
        assert np.array_equal(d.cpu().numpy().astype(np.int64), expect), (fm, r)


@pytest.mark.parametrize("case", [
    # M, N, K, data bits, w
    (3, 4096, 16, 7, 32),
    (4, 3000, 64, 15, 64),
    (5, 700, 33, 12, 64),
])
def test_small_dispatch_matches_tensor_cores(ne, orc, case):
    """The same small job with the small-job rule (multiply-add kernels)
    and with the tensor-core forms forced: both equal the oracle."""
    M, N, K, bc, w = case
    p = ne.ne_params(M, w)
    gen = synth.rng(N + K + M)
    c = synth.uniform_int(gen, (M, N), -(1 << bc), 1 << bc)
    g = synth.uniform_int(gen, (K,), -(1 << bc) + 1, 1 << bc)
    expect = conv_par(orc, c, g, w)
    dt = torch.int32 if w == 32 else torch.int64
    cd = torch.from_numpy(c.astype(np.int32 if w == 32 else np.int64)).cuda()
    gd = torch.from_numpy(g.astype(np.int32)).cuda()
    rng_c = (-(1 << bc), (1 << bc) - 1)
    try:
        for always in (False, True):
            ne.ne_debug_set_dispatch(always)
            for fm, r in _modes(ne, M):
                d = torch.full((M, N + K - 1), 3, dtype=dt, device="cuda")
                ne.ne_protected_conv(cd, gd, d, l=p.l, c_range=rng_c,
                                     max_abs_g=(1 << bc) - 1, failed=r,
                                     fail_mode=fm)
                y = torch.full((M, N + K - 1), 3, dtype=dt, device="cuda")
                ne.ne_conv(cd, gd, y, x_range=rng_c, max_abs_g=(1 << bc) - 1)
                torch.cuda.synchronize()
                assert np.array_equal(d.cpu().numpy().astype(np.int64), expect), (always, fm, r)
                assert np.array_equal(y.cpu().numpy().astype(np.int64), expect), always
    finally:
        ne.ne_debug_set_dispatch(False)
