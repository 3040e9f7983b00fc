"""Serving with continuous batching: every result equals the job run alone
(bit for bit, tolerance 0) and the oracle's plain convolution, the memory
budget holds, and injected fail-stops are recovered on the device."""
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


def test_serve_results_equal_alone_and_in_the_mix(ne, orc):
    from paper_1509_03838_gb300 import serve
    spec = synth.serve_spec(seed=21, n_jobs=800, rate_hz=20000.0,
                            N_range=(1 << 12, 1 << 16), K_range=(16, 512))
    gen = synth.rng(5)
    failing = np.flatnonzero(spec.inject)
    keep = set(gen.choice(len(spec.batch), size=10, replace=False).tolist())
    keep |= set(failing[:6].tolist())
    budget = 96 << 20  # small budget: admission has to wait for memory
    res = serve.serve(spec, budget_bytes=budget, streams=3, keep=keep, seed=9)
    assert np.all(res.latency_ms > 0) and len(res.latency_ms) == 800
    assert res.peak_bytes <= budget and res.batches > 3
    assert 0.04 < spec.inject.mean() < 0.2
    assert ne.ne_get_device_error() == 0
    for n_checked, (i, (c, g, d, failed, mode)) in enumerate(sorted(res.kept.items())):
        M, N = c.shape
        K = g.numel()
        p = ne.ne_params(M, 64)
        alone = torch.full((M, N + K - 1), 9, dtype=torch.int64, device="cuda")
        ne.ne_protected_conv(c, g, alone, l=p.l, c_range=(-(1 << 15), (1 << 15) - 1),
                             max_abs_g=1 << 15, failed=failed, fail_mode=mode)
        torch.cuda.synchronize()
        assert torch.equal(alone, d), i           # alone == in the mix
        if n_checked < 6:
            assert np.array_equal(d.cpu().numpy(),
                                  orc.conv(c.cpu().numpy(), g.cpu().numpy(), 64)), i
