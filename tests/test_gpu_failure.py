"""Failure detection without a GPU fault: the bounded grid barrier of the cooperative
Lanczos step gives up, raises its error flag and returns, and the host reads DM_ETIMEOUT.

The wait is made to run out by a barrier target that counts one arrival more than there
are blocks (nothing can complete it); the device must stay usable afterwards.
"""
import time

import numpy as np
import pytest

import synth


def test_selftest_rejects_bad_arguments():
    import paper_2311_06115_gb300 as dm

    lib = dm.load()
    assert lib.dm_selftest_wait_timeout(0, 0, 100, None) == dm.DM_EINVAL
    assert lib.dm_selftest_wait_timeout(9, 0, 100, None) == dm.DM_EINVAL
    assert lib.dm_selftest_wait_timeout(2, -1, 100, None) == dm.DM_EINVAL
    assert lib.dm_selftest_wait_timeout(2, 1, 0, None) == dm.DM_EINVAL
    assert lib.dm_selftest_wait_timeout(2, 1, (1 << 24) + 1, None) == dm.DM_EINVAL


@pytest.mark.gpu
def test_grid_barrier_times_out_and_the_device_stays_usable():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2311_06115_gb300 as dm

    # complete count: every block passes
    st, passed = dm.dm_selftest_wait_timeout(4, 0, 1 << 20)
    assert st == dm.DM_OK and passed == 4
    # one arrival missing: every block gives up after its bounded wait
    t0 = time.perf_counter()
    st, passed = dm.dm_selftest_wait_timeout(4, 1, 1 << 14)
    dt = time.perf_counter() - t0
    assert st == dm.DM_ETIMEOUT and passed == 0
    assert "gave up" in dm.dm_last_error()
    assert dt < 5.0, dt
    # the context is intact: a solve runs and converges afterwards
    X = synth.as_f32(synth.s_curve(1500, 2))
    h = dm.dm_create(X, eps=-1.0)
    dm.dm_compress(h, 1e-5, 128, 48)
    ev, _, conv = dm.dm_eigs(h, 5, evecs=False)
    assert conv and abs(ev[0] - 1.0) < 1e-4
    dm.dm_destroy(h)
    st, passed = dm.dm_selftest_wait_timeout(2, 0, 1 << 20)
    assert st == dm.DM_OK and passed == 2
