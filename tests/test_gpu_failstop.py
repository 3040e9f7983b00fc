"""Failures beyond the injected index: a mask of failed streams (two or more
are unrecoverable, Sec. I), fail-stop detection by a host deadline (a core
that misses a predetermined deadline has failed, Sec. I; the outputs are
disentangled once any M - 1 are available, Sec. V), and bounded device
waits that run out on purpose (a kernel role that the host tells never to
run).  Late cores are made on the host: their launch is held back until the
deadline has passed.  Nothing here faults, traps or hangs a GPU."""
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


def _job(seed=31, M=4, N=50000, K=64, b=15):
    j = synth.stream_job(seed, M, N, K, b, b, 64)
    c = torch.from_numpy(j.c).cuda()
    g = torch.from_numpy(j.g.astype(np.int32)).cuda()
    return j, c, g


def test_recover_mask(ne, orc):
    M, w = 4, 64
    j, c, g = _job()
    p = ne.ne_params(M, w)
    eps = torch.empty_like(c)
    ne.ne_entangle(c, eps, l=p.l)
    delta = torch.empty((M, j.N + j.K - 1), dtype=torch.int64, device="cuda")
    ne.ne_conv(eps, g, delta)
    plain = conv_par(orc, j.c, j.g, w)
    for mask in [0] + [1 << m for m in range(M)]:
        d = torch.full_like(delta, 5)
        ne.ne_recover_mask(delta, d, l=p.l, failed_mask=mask)
        torch.cuda.synchronize()
        assert np.array_equal(d.cpu().numpy(), plain), mask
    for mask in (0b11, 0b1010, 0b1111):
        d = torch.full_like(delta, 5)
        with pytest.raises(ne.NEError) as ei:
            ne.ne_recover_mask(delta, d, l=p.l, failed_mask=mask)
        assert ei.value.status == ne.NE_ERR_UNRECOVERABLE
        torch.cuda.synchronize()
        assert (d == 5).all()  # nothing written


def _fs_call(ne, fs, j, c, g, inject, deadline_ms):
    M, N, K = j.M, j.N, j.K
    p = ne.ne_params(M, 64)
    eps = torch.empty_like(c)
    delta = torch.full((M, N + K - 1), 9, dtype=torch.int64, device="cuda")
    d = torch.full((M, N + K - 1), 7, dtype=torch.int64, device="cuda")
    err = None
    try:
        fs.protected_conv(c, g, eps, delta, d, l=p.l, c_range=j.c_range,
                          max_abs_g=j.bound_g, deadline_ms=deadline_ms,
                          inject_late=inject)
    except ne.NEError as e:
        err = e
    torch.cuda.synchronize()
    fs.sync()
    return d, fs.last_late, err


def test_deadline_every_core_in_time(ne, orc):
    j, c, g = _job()
    fs = ne.FailStop(8)
    d, late, err = _fs_call(ne, fs, j, c, g, 0, 10000.0)
    assert err is None and late == 0
    assert np.array_equal(d.cpu().numpy(), conv_par(orc, j.c, j.g, 64))


@pytest.mark.parametrize("r", [0, 2, 3])
def test_deadline_one_late_core_is_recovered(ne, orc, r):
    """Core r is held back past the deadline: the host declares it failed
    and recovers all M outputs from the other M - 1 products."""
    j, c, g = _job(seed=40 + r)
    fs = ne.FailStop(4)
    d, late, err = _fs_call(ne, fs, j, c, g, 1 << r, 150.0)
    assert err is None and late == 1 << r
    assert np.array_equal(d.cpu().numpy(), conv_par(orc, j.c, j.g, 64))


def test_deadline_two_late_cores_are_unrecoverable(ne):
    j, c, g = _job(seed=50, M=5, K=33, b=12)
    fs = ne.FailStop(5)
    d, late, err = _fs_call(ne, fs, j, c, g, 0b10010, 100.0)
    assert err is not None and err.status == ne.NE_ERR_UNRECOVERABLE
    assert late == 0b10010
    assert (d == 7).all()  # d not written


def _expire(ne, orc, role, conv_plain=False):
    """Run a tensor-core launch with `role` never running and a short wait
    limit: the kernel must end (its waits give up), report NE_ERR_TIMEOUT,
    and leave the context usable for a correct run afterwards."""
    M, N, K = 4, 1 << 20, 64
    j, c, g = _job(seed=60 + role, M=M, N=N, K=K)
    p = ne.ne_params(M, 64)
    d = torch.zeros((M, N + K - 1), dtype=torch.int64, device="cuda")
    ne.ne_get_device_error(clear=True)
    ne.ne_debug_set_fault(role, 64)
    try:
        if conv_plain:
            ne.ne_conv(c, g, d, x_range=j.c_range, max_abs_g=j.bound_g)
        else:
            ne.ne_protected_conv(c, g, d, l=p.l, c_range=j.c_range,
                                 max_abs_g=j.bound_g, failed=1,
                                 fail_mode=ne.NE_FAIL_DROP)
        with pytest.raises(ne.NEError) as ei:
            ne.ne_get_device_error(clear=True)
        assert ei.value.status == ne.NE_ERR_TIMEOUT
    finally:
        ne.ne_debug_set_fault(0, 0)
    # the context is intact: the same job now runs correctly
    d.zero_()
    ne.ne_protected_conv(c, g, d, l=p.l, c_range=j.c_range,
                         max_abs_g=j.bound_g, failed=2, fail_mode=ne.NE_FAIL_SKIP)
    torch.cuda.synchronize()
    assert ne.ne_get_device_error(clear=True) == 0
    assert np.array_equal(d.cpu().numpy(), conv_par(orc, j.c, j.g, 64))


@pytest.mark.parametrize("role", [1, 2])
def test_bounded_waits_expire_and_report_timeout(ne, orc, role):
    """Role 1: the loader never copies (the staging warps' wait runs out);
    role 2: the MMA warp never issues (the staging and epilogue waits run
    out).  Runs on the kernel the library picks for the job."""
    _expire(ne, orc, role)


def test_bounded_waits_expire_in_the_plain_kernel(ne, orc):
    _expire(ne, orc, 1, conv_plain=True)


def _child_run(env_extra, select):
    import os
    import subprocess
    import sys
    env = dict(os.environ, **env_extra)
    out = subprocess.run(
        [sys.executable, "-m", "pytest", __file__, "-q", "-x", "-m", "gpu",
         "-p", "no:cacheprovider", "-k", select],
        env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout[-3000:] + out.stderr[-2000:]
    assert " passed" in out.stdout


def test_bounded_waits_expire_on_the_entangled_digit_kernel(ne):
    """NE_CONV_TCR=0: the same expiring waits in the tcgen05 kernel whose
    digits are those of the entangled words; its teardown drains the bulk
    copies and products in flight before freeing tensor memory."""
    _child_run({"NE_CONV_TCR": "0"}, "bounded_waits_expire_and_report")
