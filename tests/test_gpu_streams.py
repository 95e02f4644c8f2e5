"""Concurrency inside one solve: the tree build on its own stream (overlapping the degree
passes) and the stream-ordered device allocator must give what the single-stream path and
torch's caching allocator give."""
import math

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


def _angle(A, B):
    sv = np.linalg.svd(A.astype(np.float64).T @ B.astype(np.float64), compute_uv=False)
    return math.acos(min(1.0, float(sv.min())))


def _solve(dm, X, k, **kw):
    cfg = dm.dm_config_default(**{k_: v for k_, v in kw.items() if k_ != "use_torch_allocator"})
    h = dm.dm_create(X, eps=-1.0, cfg=cfg, use_torch_allocator=kw.get("use_torch_allocator", False))
    dm.dm_compress(h, 1e-5, 256, 64)
    perm, L = dm.dm_get_tree(h)
    q, dg, s = dm.dm_get_degrees(h)
    ev, V, conv = dm.dm_eigs(h, k)
    st = dm.dm_get_stats(h)
    dm.dm_destroy(h)
    assert conv
    return perm, q, ev, V, st


def test_overlapped_tree_build_matches_single_stream(dm):
    """shared_device = 0 builds the tree on a side stream while the degree passes run;
    shared_device = 1 runs every phase on the handle's stream. The tree is an exact FP64
    construction: identical permutations; the rest within FP64-atomics reordering."""
    X = synth.as_f32(synth.s_curve(30000, 7))
    p0, q0, ev0, V0, st0 = _solve(dm, X, 12, shared_device=0)
    p1, q1, ev1, V1, st1 = _solve(dm, X, 12, shared_device=1)
    np.testing.assert_array_equal(p0, p1)
    np.testing.assert_allclose(q0, q1, rtol=1e-12)
    np.testing.assert_allclose(ev0, ev1, rtol=1e-6, atol=1e-9)
    assert _angle(V0, V1) < 2e-3
    # the deferred phase timers resolve to positive times
    assert st0["ms_create"] > 0 and st0["ms_skeleton"] > 0 and st0["ms_pack"] > 0


def test_stream_ordered_allocator_matches_torch_allocator(dm):
    X = synth.as_f32(synth.swiss_roll(20000, 8))
    pa, qa, eva, Va, _ = _solve(dm, X, 8, use_torch_allocator=False)
    pb, qb, evb, Vb, _ = _solve(dm, X, 8, use_torch_allocator=True)
    np.testing.assert_array_equal(pa, pb)
    np.testing.assert_allclose(qa, qb, rtol=1e-12)
    np.testing.assert_allclose(eva, evb, rtol=1e-6, atol=1e-9)
    assert _angle(Va, Vb) < 2e-3
