"""dm_eigs_batch: many uneven point clouds solved together, every Lanczos step of every
cloud in the same launches. Each cloud's eigenpairs must be those of the oracle's FP64
Lanczos on the same (replayed) structure and of its own solo dm_eigs, and the launches per
step must not grow with the number of clouds."""
import math

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

SIZES = [1500, 3001, 800, 2048, 5000, 1234]


@pytest.fixture(scope="module")
def dm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2311_06115_gb300 as m

    m.load()
    return m


@pytest.fixture(scope="module")
def clouds():
    out = []
    for i, n in enumerate(SIZES):
        X = synth.as_f32(synth.s_curve(n, 20 + i) if i % 2 == 0 else synth.swiss_roll(n, 20 + i))
        eps = O.median_sqdist(X)
        _, _, s = O.degrees(X, eps, 1.0)
        leaf = 128 if n > 1000 else 64
        H = O.compress(X, eps, s, leaf, 1e-5, 48)
        out.append(dict(X=X, eps=eps, s=s, H=H))
    return out


def _handles(dm, clouds, seed0=0):
    hs = []
    for i, c in enumerate(clouds):
        H = c["H"]
        h = dm.dm_create(c["X"], eps=c["eps"], cfg=dm.dm_config_default(seed=seed0 + i))
        dm.dm_load_hmatrix(h, H.L, H.max_rank, H.perm, H.ranks, H.skel, H.P.astype(np.float32))
        hs.append(h)
    return hs


def test_batch_matches_oracle_and_solo(dm, clouds):
    k = 6
    hs = _handles(dm, clouds)
    ev, vecs, status = dm.dm_eigs_batch(hs, k)
    assert list(status) == [dm.DM_OK] * len(hs)
    for i, c in enumerate(clouds):
        evo, Vo, _, sto = O.lanczos_hmat(c["X"], c["eps"], c["s"], c["H"], k + 1, conv_tol=1e-10)
        assert sto == 0
        np.testing.assert_allclose(ev[i], evo[:k], rtol=2e-5, atol=2e-7)
        V = vecs[i].astype(np.float64)
        np.testing.assert_allclose(V.T @ V, np.eye(k), atol=2e-5)
        for t in range(k):
            gap = min(abs(evo[t] - evo[u]) for u in range(k + 1) if u != t)
            if gap > 1e-3:
                cth = abs(float(np.dot(V[:, t], Vo[:, t])))
                assert math.acos(min(1.0, cth)) < 2e-3, (i, t)
            assert V[np.argmax(np.abs(V[:, t])), t] > 0  # sign rule
    # the same handles solved one by one
    for i, h in enumerate(hs):
        evs, _, conv = dm.dm_eigs(h, k, evecs=False)
        assert conv
        np.testing.assert_allclose(ev[i], evs, rtol=2e-5, atol=2e-7)
        dm.dm_destroy(h)


def test_batch_launches_per_step_do_not_grow_with_count(dm, clouds):
    k = 5
    counts = {}
    for sub in (clouds[:2], clouds):
        hs = _handles(dm, sub)
        l0 = dm.dm_kernel_launches()
        ev, _, status = dm.dm_eigs_batch(hs, k, evecs=False)
        launches = dm.dm_kernel_launches() - l0
        steps = max(dm.dm_get_stats(h)["lanczos_iters"] for h in hs)
        for h in hs:
            dm.dm_destroy(h)
        # shared by all clouds: start vectors (3 launches per joining group) and Ritz vectors (6
        # per finishing group); per step: 3 (H-matvec) + 3 (Gram-Schmidt) launches, one more at
        # each check. Neither grows with the number of clouds.
        per_step = (launches - 9 * len(sub)) / steps
        counts[len(sub)] = per_step
        assert per_step <= 7.0, (len(sub), launches, steps)
    print("launches per step:", counts)


def test_batch_mixed_schedules_and_basis_caps(dm, clouds):
    """Handles with their own check_every, and some whose basis cap (m_max) is reached before
    they converge: those leave the step list at the cap and report DM_ENOCONV with the Ritz
    pairs of the full basis, exactly as their solo solve does; the others converge as alone."""
    k = 6
    capped = {1, 4}
    hs = []
    for i, c in enumerate(clouds):
        H = c["H"]
        cfg = dm.dm_config_default(seed=i, check_every=1 + (i % 3), m_max=12 if i in capped else 300)
        h = dm.dm_create(c["X"], eps=c["eps"], cfg=cfg)
        dm.dm_load_hmatrix(h, H.L, H.max_rank, H.perm, H.ranks, H.skel, H.P.astype(np.float32))
        hs.append(h)
    ev, vecs, status = dm.dm_eigs_batch(hs, k)
    for i, h in enumerate(hs):
        st = dm.dm_get_stats(h)
        if i in capped:
            assert status[i] == dm.DM_ENOCONV and st["lanczos_iters"] == 12, (i, status[i], st["lanczos_iters"])
        else:
            assert status[i] == dm.DM_OK, i
        evs, Vs, conv = dm.dm_eigs(h, k)
        assert conv == (i not in capped)
        if i in capped:
            # the same 12-step basis: the same Ritz values up to the summation order
            np.testing.assert_allclose(ev[i], evs, rtol=1e-5, atol=1e-7)
        else:
            np.testing.assert_allclose(ev[i], evs, rtol=2e-5, atol=2e-7)
        V = vecs[i].astype(np.float64)
        np.testing.assert_allclose(V.T @ V, np.eye(k), atol=2e-5)
        dm.dm_destroy(h)


def test_batch_argument_errors(dm, clouds):
    hs = _handles(dm, clouds[:2])
    lib = dm.load()
    import ctypes as C

    arr = (C.c_void_p * 2)(hs[0].ptr, hs[0].ptr)
    ev = np.empty(20)
    assert lib.dm_eigs_batch(arr, 2, 5, ev.ctypes.data, None, None) == dm.DM_EINVAL  # repeated handle
    arr = (C.c_void_p * 2)(hs[0].ptr, hs[1].ptr)
    assert lib.dm_eigs_batch(arr, 2, 0, ev.ctypes.data, None, None) == dm.DM_EINVAL  # k = 0
    h3 = dm.dm_create(clouds[2]["X"], eps=clouds[2]["eps"])
    arr = (C.c_void_p * 2)(hs[0].ptr, h3.ptr)
    assert lib.dm_eigs_batch(arr, 2, 5, ev.ctypes.data, None, None) == dm.DM_ESTATE  # not compressed
    for h in hs + [h3]:
        dm.dm_destroy(h)
