"""dm_degrees_noalloc, the entry point that allocates no device memory.

It exists for callers that cannot let a library allocate: a framework that owns
all device memory, a fixed memory budget, or a hot path that must not take
cudaMalloc's implicit synchronisation. It must return what the allocating path
(dm_create + dm_get_degrees) returns, on consecutive calls that share its one
scratch array, and it must leave the device's free memory unchanged. This file
is named so that pytest collects it last.
"""
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


def _outputs(n):
    import torch

    return tuple(torch.full((n,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(3))


def _noalloc(dm, X, eps, alpha):
    import torch

    n = X.shape[0]
    Xd = torch.from_numpy(X).cuda()
    q, dg, s = _outputs(n)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    dm.dm_degrees_noalloc(Xd, eps, alpha, q, dg, s, stream=stream)
    stream.synchronize()
    return q.cpu().numpy(), dg.cpu().numpy(), s.cpu().numpy()


def _reference(dm, X, alpha):
    h = dm.dm_create(X, eps=-1.0, alpha=alpha)
    eps = dm.dm_get_eps(h)
    deg = dm.dm_get_degrees(h)
    path = dm.dm_get_stats(h)["degree_path"]
    dm.dm_destroy(h)
    return eps, deg, path


def test_noalloc_matches_allocating_path_on_two_calls(dm):
    # two calls in a row with different sizes: the second sees the first call's scratch contents
    for n, seed, alpha in [(3000, 5, 1.0), (1777, 6, 0.5)]:
        X = synth.as_f32(synth.s_curve(n, seed))
        eps, (q_ref, dg_ref, s_ref), _ = _reference(dm, X, alpha)
        q, dg, s = _noalloc(dm, X, eps, alpha)
        np.testing.assert_allclose(q, q_ref, rtol=2e-6)
        np.testing.assert_allclose(dg, dg_ref, rtol=2e-6)
        np.testing.assert_allclose(s, s_ref, rtol=2e-6)


@pytest.mark.parametrize("kind,n,d", [("mixture", 2500, 17), ("mixture", 2049, 64), ("mnist", 1500, 784),
                                      ("mixture", 1000, 6)])
def test_noalloc_matches_allocating_path_higher_dimensions(dm, kind, n, d):
    # dm_create takes the tensor-core Gram path at d >= 16 (exact BF16 for the 8-bit
    # MNIST-shaped data, TF32 split otherwise); this entry point keeps the FP32 difference form
    X = synth.as_f32(synth.mnist_like(n, seed=2, d=d) if kind == "mnist" else synth.gaussian_mixture(n, d=d, seed=3))
    eps, (q_ref, dg_ref, s_ref), path = _reference(dm, X, 1.0)
    assert (path != 0) == (d >= 16)
    rtol = 5e-6 if d >= 16 else 2e-6
    for _ in range(2):
        q, dg, s = _noalloc(dm, X, eps, 1.0)
        np.testing.assert_allclose(q, q_ref, rtol=rtol)
        np.testing.assert_allclose(dg, dg_ref, rtol=rtol)
        np.testing.assert_allclose(s, s_ref, rtol=rtol)


def test_noalloc_allocates_nothing(dm):
    import torch

    X = synth.as_f32(synth.s_curve(4000, 9))
    Xd = torch.from_numpy(X).cuda()
    q, dg, s = _outputs(4000)
    dm.dm_degrees_noalloc(Xd, 0.5, 1.0, q, dg, s)  # warm-up: module load, scratch lookup
    q0 = q.clone()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(3):
        dm.dm_degrees_noalloc(Xd, 0.5, 1.0, q, dg, s)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.memory_reserved() == reserved0
    assert torch.equal(q, q0)


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


def test_noalloc_binding_rejects_wrong_tensors(dm):
    import torch

    n = 64
    X = torch.rand((n, 3), dtype=torch.float32, device="cuda")
    q, dg, s = _outputs(n)
    bad = [
        (X.double(), q, dg, s),                                  # float64 points
        (X.t().contiguous().t(), q, dg, s),                      # column-major points
        (X.cpu(), q, dg, s),                                     # host points
        (X, q.float(), dg, s),                                   # float32 output: would be overrun
        (X, q, dg[: n - 1], s),                                  # short output
        (X, q, dg, s.cpu()),                                     # host output
        (X.reshape(-1), q, dg, s),                               # not (N, d)
    ]
    for args in bad:
        with pytest.raises(ValueError):
            dm.dm_degrees_noalloc(args[0], 0.5, 1.0, *args[1:])
    assert torch.isnan(q).all() and torch.isnan(dg).all() and torch.isnan(s).all()
