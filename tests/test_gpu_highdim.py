"""Parity at the high-dimensional workload's shape: MNIST-shaped synthetic data (10 Gaussian
clusters on a random 10-dimensional subspace of R^784, ReLU-shifted to ~80% zeros, 8-bit
grid), N = 20,000, leaf 256, max rank 128, tol 1e-4.

The degree passes take the tensor-core Gram path (exact BF16 products of the 8-bit codes);
the tree takes FP64 decisions on both sides (bit-exact permutation); the eigensolve runs on
the oracle's own compression loaded through dm_load_hmatrix, so the CUDA evaluation of
Eq. 2.18 at d = 784 (near blocks and sibling blocks filled by the coordinate-tiled entry
kernel) is compared with the oracle's FP64 Lanczos on the same structure.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N = 20_000
K = 10


@pytest.fixture(scope="module")
def dm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2311_06115_gb300 as m

    m.load()
    return m


@pytest.fixture(scope="module")
def mref():
    X = synth.as_f32(synth.mnist_like(N, seed=5))
    eps = O.median_sqdist(X)
    q, dg, s = O.degrees(X, eps, 1.0)
    H = O.compress(X, eps, s, 256, 1e-4, 128)
    ev, V, it, st = O.lanczos_hmat(X, eps, s, H, K + 1, conv_tol=1e-9)
    assert st == 0
    return dict(X=X, eps=eps, q=q, dg=dg, s=s, H=H, ev=ev, V=V)


def test_mnist_shaped_bandwidth_degrees_and_tree(dm, mref):
    X = mref["X"]
    h = dm.dm_create(X, eps=-1.0)
    assert dm.dm_get_eps(h) == mref["eps"]
    st = dm.dm_get_stats(h)
    assert st["degree_path"] == 2  # exact BF16 Gram matrix of the 8-bit codes
    q, dg, s = dm.dm_get_degrees(h)
    rows = np.random.default_rng(8).choice(N, 500, replace=False)
    np.testing.assert_allclose(q[rows], mref["q"][rows], rtol=5e-6)
    np.testing.assert_allclose(dg[rows], mref["dg"][rows], rtol=5e-6)
    np.testing.assert_allclose(s[rows], mref["s"][rows], rtol=5e-6)
    dm.dm_compress(h, 1e-4, 256, 128)
    perm, L = dm.dm_get_tree(h)
    assert L == mref["H"].L and np.array_equal(perm, mref["H"].perm)
    dm.dm_destroy(h)


def test_mnist_shaped_eigs_on_replayed_structure(dm, mref):
    H = mref["H"]
    h = dm.dm_create(mref["X"], eps=mref["eps"])
    dm.dm_load_hmatrix(h, H.L, H.max_rank, H.perm, H.ranks, H.skel, H.P.astype(np.float32))
    x = synth.random_rhs(N, 2, seed=12).astype(np.float32)
    y = dm.dm_matvec(h, np.asfortranarray(x))
    yr = O.hmatvec(mref["X"], mref["eps"], mref["s"], H, x.astype(np.float64))
    err = np.abs(y - yr).max() / np.abs(x).max()
    print(f"d=784 replay: max |y - y_oracle| / max|x| = {err:.3e}")
    assert err < 1e-5, err
    ev, V, conv = dm.dm_eigs(h, K)
    assert conv
    evo, Vo = mref["ev"][:K], mref["V"][:, :K]
    rel = np.abs(ev - evo) / np.abs(evo)
    print(f"d=784 eigenvalues: max rel {rel.max():.3e}")
    np.testing.assert_allclose(ev, evo, rtol=2e-5, atol=2e-7)
    gap = np.abs(np.diff(mref["ev"][:K + 1]))
    for i in range(K):
        c = abs(float(np.dot(V[:, i].astype(np.float64), Vo[:, i])))
        g = min(gap[i - 1] if i > 0 else np.inf, gap[i])
        # per-vector angles where the spectrum separates the pair; the subspace as a whole always
        if g > 1e-3:
            assert math.acos(min(1.0, c)) < 2e-3, (i, g)
    sv = np.linalg.svd(Vo.T @ V.astype(np.float64), compute_uv=False)
    assert math.acos(min(1.0, sv.min())) < 2e-3
    dm.dm_destroy(h)
