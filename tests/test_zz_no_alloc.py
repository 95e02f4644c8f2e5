"""dm_degrees_noalloc, the entry point that allocates no device memory.

It exists for callers that cannot let a library allocate: a framework that owns
all device memory, a fixed memory budget, or a hot path that must not take
cudaMalloc's implicit synchronisation. It must return what the allocating path
(dm_create + dm_get_degrees) returns, on consecutive calls that share its one
scratch array. This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2311_06115_gb300 as m

    m.load()
    return m


def _noalloc(dm, X, eps, alpha):
    import torch

    n = X.shape[0]
    Xd = torch.from_numpy(X).cuda()
    q, dg, s = (torch.full((n,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(3))
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    dm.dm_degrees_noalloc(Xd, eps, alpha, q, dg, s, stream=stream)
    stream.synchronize()
    return q.cpu().numpy(), dg.cpu().numpy(), s.cpu().numpy()


def test_noalloc_matches_allocating_path_on_two_calls(dm):
    # two calls in a row with different sizes: the second sees the first call's scratch contents
    for n, seed, alpha in [(3000, 5, 1.0), (1777, 6, 0.5)]:
        X = synth.as_f32(synth.s_curve(n, seed))
        h = dm.dm_create(X, eps=-1.0, alpha=alpha)
        eps = dm.dm_get_eps(h)
        q_ref, dg_ref, s_ref = dm.dm_get_degrees(h)
        dm.dm_destroy(h)
        q, dg, s = _noalloc(dm, X, eps, alpha)
        np.testing.assert_allclose(q, q_ref, rtol=2e-6)
        np.testing.assert_allclose(dg, dg_ref, rtol=2e-6)
        np.testing.assert_allclose(s, s_ref, rtol=2e-6)


def test_noalloc_rejects_bad_arguments(dm):
    import torch

    lib = dm.load()
    x = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
    o = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = [x.data_ptr(), o.data_ptr(), o.data_ptr(), o.data_ptr()]
    # beyond the 16 MiB scratch limit: rejected before any work is enqueued
    assert lib.dm_degrees_noalloc(p[0], 2_000_000, 3, 1.0, 1.0, p[1], p[2], p[3], None) == dm.DM_EINVAL
    assert "16 MiB" in dm.dm_last_error()
    assert lib.dm_degrees_noalloc(p[0], 4, 3, 0.0, 1.0, p[1], p[2], p[3], None) == dm.DM_EINVAL
    host = np.zeros(4)
    assert lib.dm_degrees_noalloc(p[0], 4, 3, 1.0, 1.0, host.ctypes.data, p[2], p[3], None) == dm.DM_EINVAL
