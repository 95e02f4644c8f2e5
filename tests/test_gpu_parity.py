"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP32 device arithmetic against FP64): unit roundoff u = 6e-8; an
entry exp2(-r^2) from pre-scaled FP32 coordinates carries ~3u relative error
plus the MUFU ex2 error (~2 ulp); sums of up to a few hundred such terms in FP32
tiles grow that to ~1e-6 relative at most, so degree vectors are held to 2e-6
and matvec outputs to 1e-5 of max|x| per element (>= 100 u of headroom).
Integer work (bandwidth median, tree permutation) is bit-exact.
"""
import math

import numpy as np
import pytest

import oracle as O
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


def _scurve(n, seed=0):
    return synth.as_f32(synth.s_curve(n, seed))


def _rel_inf(a, b, scale):
    return float(np.max(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64))) / scale)


# ------------------------------------------------------------------ bandwidth and degrees

@pytest.mark.parametrize("n", [1000, 1449, 3000])
def test_bandwidth_median_bit_exact(dm, n):
    X = _scurve(n, 5)
    h = dm.dm_create(X, eps=-1.0)
    assert dm.dm_get_eps(h) == O.median_sqdist(X, seed=0)


@pytest.mark.parametrize("n,alpha,eps_scale", [(2048, 1.0, 1.0), (1537, 1.0, 1.0), (999, 0.5, 1.0), (600, 0.0, 1.0),
                                                (3001, 1.0, 1.0), (5000, 0.5, 0.05)])
def test_degrees_match_oracle(dm, n, alpha, eps_scale):
    """Degree vectors; from N = 2048 on the d = 3 passes evaluate only the upper tiles of the
    symmetric W (row and column sums). eps_scale 0.05 shrinks the kernel so that the scaled
    squared norms exceed the dot form's limit: the difference form runs."""
    X = _scurve(n, 1)
    eps = O.median_sqdist(X) * eps_scale
    h = dm.dm_create(X, eps=eps, alpha=alpha)
    q, dg, s = dm.dm_get_degrees(h)
    oq, odg, os_ = O.degrees(X, eps, alpha)
    np.testing.assert_allclose(q, oq, rtol=2e-6)
    np.testing.assert_allclose(dg, odg, rtol=2e-6)
    np.testing.assert_allclose(s, os_, rtol=2e-6)


def test_degrees_on_generic_dimension(dm):
    X = synth.as_f32(synth.gaussian_mixture(700, d=64, seed=2))
    eps = O.median_sqdist(X)
    h = dm.dm_create(X, eps=eps)
    q, dg, s = dm.dm_get_degrees(h)
    oq, odg, os_ = O.degrees(X, eps, 1.0)
    np.testing.assert_allclose(q, oq, rtol=5e-6)
    np.testing.assert_allclose(s, os_, rtol=5e-6)


@pytest.mark.parametrize("kind,n,d", [("mnist", 3001, 784), ("mnist", 700, 200), ("mixture", 1537, 17),
                                       ("mixture", 2000, 64), ("mixture", 999, 128)])
def test_degrees_tensor_core_gram(dm, kind, n, d):
    """Degree passes of d >= 16 on the tensor cores: 8-bit quantised data (MNIST-shaped) as an
    exact BF16 Gram matrix, other data as the TF32 three-term split (relative Gram error
    about 2^-20 of |u_i||u_j|, i.e. ~1e-6 in each exponent at eps = median). Ragged N and d
    cover partial row/column tiles and zero-padded K."""
    X = synth.as_f32(synth.mnist_like(n, seed=4, d=d) if kind == "mnist" else synth.gaussian_mixture(n, d=d, seed=4))
    eps = O.median_sqdist(X)
    h = dm.dm_create(X, eps=eps)
    st = dm.dm_get_stats(h)
    assert st["degree_path"] == (2 if kind == "mnist" else 1)
    q, dg, s = dm.dm_get_degrees(h)
    oq, odg, os_ = O.degrees(X, eps, 1.0)
    np.testing.assert_allclose(q, oq, rtol=5e-6)
    np.testing.assert_allclose(dg, odg, rtol=5e-6)
    np.testing.assert_allclose(s, os_, rtol=5e-6)
    dm.dm_destroy(h)


def test_exact_matvec_before_compress(dm):
    n = 1200
    X = _scurve(n, 2)
    eps = O.median_sqdist(X)
    h = dm.dm_create(X, eps=eps)
    _, _, s = O.degrees(X, eps, 1.0)
    x = synth.random_rhs(n, 2, seed=3).astype(np.float32)
    y = dm.dm_matvec(h, np.asfortranarray(x))
    yr = O.S_matvec(X, eps, s, x.astype(np.float64))
    assert _rel_inf(y, yr, np.abs(x).max()) < 1e-5


# ------------------------------------------------------------------ tree

@pytest.mark.parametrize("n,leaf", [(2048, 128), (1500, 100), (777, 50), (4097, 256), (20000, 512), (17001, 300)])
def test_tree_bit_exact(dm, n, leaf):
    """The permutation equals the oracle's bit for bit; from 8192 points a node is split over
    many CTAs (digit histograms and partition ranks from per-item counts)."""
    X = _scurve(n, 7)
    eps = O.median_sqdist(X)
    h = dm.dm_create(X, eps=eps)
    dm.dm_compress(h, 1e-5, leaf, 32)
    perm, L = dm.dm_get_tree(h)
    operm, oL = O.tree(X, eps, leaf)
    assert L == oL
    assert np.array_equal(perm, operm)


# ------------------------------------------------------------------ H-matvec on a replayed oracle structure

@pytest.mark.parametrize("mode", ["cached", "onthefly"])
@pytest.mark.parametrize("n,leaf,rank,tol", [(2048, 128, 64, 1e-5), (1500, 100, 40, 1e-3), (700, 64, 64, 0.0)])
def test_hmatvec_replay_matches_oracle(dm, mode, n, leaf, rank, tol):
    X = _scurve(n, 11)
    eps = O.median_sqdist(X)
    _, _, s = O.degrees(X, eps, 1.0)
    H = O.compress(X, eps, s, leaf, tol, rank)
    cfg = dm.dm_config_default(near_mode=dm.DM_NEAR_CACHED if mode == "cached" else dm.DM_NEAR_ONTHEFLY)
    h = dm.dm_create(X, eps=eps, cfg=cfg)
    dm.dm_load_hmatrix(h, H.L, H.max_rank, H.perm, H.ranks, H.skel, H.P.astype(np.float32))
    x = synth.random_rhs(n, 3, seed=5).astype(np.float32)
    y = dm.dm_matvec(h, np.asfortranarray(x))
    yr = O.hmatvec(X, eps, s, H, x.astype(np.float64))
    assert _rel_inf(y, yr, np.abs(x).max()) < 1e-5
    # a second call reuses the same buffers: results must not change
    y2 = dm.dm_matvec(h, np.asfortranarray(x))
    assert np.array_equal(y, y2)


def test_hmatvec_paths_match_oracle(dm):
    """The one-cluster tree pass (low ranks) and the chained form (a 64-d cloud at rank 128,
    whose upper tree does not fit the cluster's shared memory) against the oracle."""
    for X, leaf, rank, tol, path in [(_scurve(3000, 12), 128, 64, 1e-5, 0),
                                     (synth.as_f32(synth.gaussian_mixture(4000, d=64, seed=3)), 128, 128, 0.0, 1)]:
        n = X.shape[0]
        eps = O.median_sqdist(X)
        _, _, s = O.degrees(X, eps, 1.0)
        H = O.compress(X, eps, s, leaf, tol, rank)
        h = dm.dm_create(X, eps=eps)
        dm.dm_load_hmatrix(h, H.L, H.max_rank, H.perm, H.ranks, H.skel, H.P.astype(np.float32))
        assert dm.dm_get_stats(h)["hmatvec_path"] == path
        x = synth.random_rhs(n, 2, seed=6).astype(np.float32)
        y = dm.dm_matvec(h, np.asfortranarray(x))
        yr = O.hmatvec(X, eps, s, H, x.astype(np.float64))
        assert _rel_inf(y, yr, np.abs(x).max()) < 1e-5
        dm.dm_destroy(h)


@pytest.mark.parametrize("mode", ["cached", "onthefly"])
@pytest.mark.parametrize("n,leaf,rank,tol,nrhs", [(2048, 128, 64, 1e-5, 16), (1500, 100, 40, 1e-3, 70),
                                                  (3001, 256, 48, 1e-4, 33), (700, 64, 64, 0.0, 5)])
def test_block_hmatvec_replay_matches_oracle(dm, mode, n, leaf, rank, tol, nrhs):
    """The block H-matvec (every operand read once per panel of up to 64 columns; ragged
    panels, leaves and row chunks) against the oracle's evaluation of the same structure,
    and against the single-vector path column by column."""
    X = _scurve(n, 13)
    eps = O.median_sqdist(X)
    _, _, s = O.degrees(X, eps, 1.0)
    H = O.compress(X, eps, s, leaf, tol, rank)
    cfg = dm.dm_config_default(near_mode=dm.DM_NEAR_CACHED if mode == "cached" else dm.DM_NEAR_ONTHEFLY)
    h = dm.dm_create(X, eps=eps, cfg=cfg)
    dm.dm_load_hmatrix(h, H.L, H.max_rank, H.perm, H.ranks, H.skel, H.P.astype(np.float32))
    x = np.asfortranarray(synth.random_rhs(n, nrhs, seed=8).astype(np.float32))
    y = dm.dm_matvec(h, x)
    yr = O.hmatvec(X, eps, s, H, x.astype(np.float64))
    assert _rel_inf(y, yr, np.abs(x).max()) < 1e-5
    for c in (0, nrhs - 1):
        y1 = dm.dm_matvec(h, np.ascontiguousarray(x[:, c]))
        assert _rel_inf(y[:, c], y1, np.abs(x[:, c]).max()) < 1e-5
    dm.dm_destroy(h)


@pytest.mark.parametrize("n,leaf,rank,tol,nrhs", [(2048, 128, 64, 1e-5, 4), (3001, 256, 48, 1e-4, 3),
                                                  (1500, 100, 40, 1e-3, 2), (5000, 128, 64, 1e-5, 4),
                                                  (700, 64, 64, 0.0, 4)])
def test_narrow_block_hmatvec_replay_matches_oracle(dm, n, leaf, rank, tol, nrhs):
    """2..4 right-hand sides through the three chained launches of the single-vector form
    (leaf N2S, the one-cluster tree pass with nrhs-wide skeleton vectors, the near stream with
    the leaf S2N), on the oracle's structure, element-wise against the oracle's Eq. 2.18
    evaluation and column by column against the single-vector path."""
    X = _scurve(n, 19)
    eps = O.median_sqdist(X)
    _, _, s = O.degrees(X, eps, 1.0)
    H = O.compress(X, eps, s, leaf, tol, rank)
    h = dm.dm_create(X, eps=eps, cfg=dm.dm_config_default(near_mode=dm.DM_NEAR_CACHED))
    dm.dm_load_hmatrix(h, H.L, H.max_rank, H.perm, H.ranks, H.skel, H.P.astype(np.float32))
    x = np.asfortranarray(synth.random_rhs(n, nrhs, seed=10).astype(np.float32))
    y = dm.dm_matvec(h, x)
    l0 = dm.dm_kernel_launches()
    y2 = dm.dm_matvec(h, x)
    assert dm.dm_kernel_launches() - l0 == 3, "the narrow-block path (three chained launches) did not run"
    assert np.array_equal(y, y2)
    yr = O.hmatvec(X, eps, s, H, x.astype(np.float64))
    assert _rel_inf(y, yr, np.abs(x).max()) < 1e-5
    for c in range(nrhs):
        y1 = dm.dm_matvec(h, np.ascontiguousarray(x[:, c]))
        assert _rel_inf(y[:, c], y1, np.abs(x[:, c]).max()) < 1e-5
    dm.dm_destroy(h)


@pytest.mark.parametrize("n,leaf,rank,tol,nrhs", [(3001, 256, 48, 1e-4, 16), (2048, 128, 64, 1e-5, 100),
                                                  (700, 64, 64, 0.0, 300), (5000, 512, 64, 1e-5, 33)])
def test_block_hmatvec_tf32_tensor_cores(dm, n, leaf, rank, tol, nrhs):
    """Near field on tcgen05 (TF32 operands, FP32 accumulation): full and tail row tiles,
    one and two column panels. Both TF32 factors are truncated to 10 mantissa bits, so
    each near term carries a relative error below 2 * 2^-10; the bound per row is
    2.5 * 2^-10 (S |x|)_i (all entries of S are positive, so S|x| dominates the near-field
    magnitudes) plus the FP32 tolerance of the rest of the path."""
    X = _scurve(n, 17)
    eps = O.median_sqdist(X)
    _, _, s = O.degrees(X, eps, 1.0)
    H = O.compress(X, eps, s, leaf, tol, rank)
    cfg = dm.dm_config_default(near_mode=dm.DM_NEAR_CACHED, block_precision=dm.DM_PREC_TF32)
    h = dm.dm_create(X, eps=eps, cfg=cfg)
    dm.dm_load_hmatrix(h, H.L, H.max_rank, H.perm, H.ranks, H.skel, H.P.astype(np.float32))
    x = np.asfortranarray(synth.random_rhs(n, nrhs, seed=9).astype(np.float32))
    y = dm.dm_matvec(h, x)
    y2 = dm.dm_matvec(h, x)
    assert np.array_equal(y, y2)
    xd = x.astype(np.float64)
    yr = O.hmatvec(X, eps, s, H, xd)
    for c in range(0, nrhs, max(1, nrhs // 7)):
        bound = 2.5 * 2.0 ** -10 * O.S_matvec(X, eps, s, np.abs(xd[:, c])) + 1e-5 * np.abs(xd[:, c]).max()
        assert np.all(np.abs(y[:, c] - yr[:, c]) <= bound), c
    # and the error is really at TF32 level, not an FP32 path in disguise or garbage
    err = np.abs(y - yr).max() / np.abs(x).max()
    assert 1e-7 < err < 2e-3, err
    dm.dm_destroy(h)


@pytest.mark.parametrize("n,leaf,rank,tol,nrhs", [(3001, 256, 48, 1e-4, 16), (2048, 128, 64, 1e-5, 100),
                                                  (700, 64, 64, 0.0, 300), (5000, 512, 64, 1e-5, 33)])
def test_block_hmatvec_split_tf32_tensor_cores(dm, n, leaf, rank, tol, nrhs):
    """Near field on tcgen05 with three-term split operands (x = hi + lo, hi TF32-exact, lo the
    remainder read as TF32; products hi*hi + hi*lo + lo*hi, FP32 accumulation): each near
    term carries at most 3 * 2^-20 relative error (the dropped lo*lo term and the TF32
    rounding of the remainders), so the per-row bound is 4 * 2^-20 (S|x|)_i plus the FP32
    tolerance of the rest of the path -- a bound the plain TF32 product (2^-9) fails."""
    X = _scurve(n, 17)
    eps = O.median_sqdist(X)
    _, _, s = O.degrees(X, eps, 1.0)
    H = O.compress(X, eps, s, leaf, tol, rank)
    x = np.asfortranarray(synth.random_rhs(n, nrhs, seed=9).astype(np.float32))
    xd = x.astype(np.float64)
    yr = O.hmatvec(X, eps, s, H, xd)
    errs = {}
    for prec in (dm.DM_PREC_TF32, dm.DM_PREC_TF32X3):
        cfg = dm.dm_config_default(near_mode=dm.DM_NEAR_CACHED, block_precision=prec)
        h = dm.dm_create(X, eps=eps, cfg=cfg)
        dm.dm_load_hmatrix(h, H.L, H.max_rank, H.perm, H.ranks, H.skel, H.P.astype(np.float32))
        y = dm.dm_matvec(h, x)
        assert np.array_equal(y, dm.dm_matvec(h, x))
        errs[prec] = np.abs(y - yr).max() / np.abs(x).max()
        if prec == dm.DM_PREC_TF32X3:
            for c in range(0, nrhs, max(1, nrhs // 7)):
                bound = 4.0 * 2.0 ** -20 * O.S_matvec(X, eps, s, np.abs(xd[:, c])) + 1e-5 * np.abs(xd[:, c]).max()
                assert np.all(np.abs(y[:, c] - yr[:, c]) <= bound), c
        dm.dm_destroy(h)
    print(f"near field TF32 {errs[dm.DM_PREC_TF32]:.3e}  split TF32 {errs[dm.DM_PREC_TF32X3]:.3e}")
    assert errs[dm.DM_PREC_TF32X3] < 1e-5
    assert errs[dm.DM_PREC_TF32X3] < 0.05 * errs[dm.DM_PREC_TF32]


# ------------------------------------------------------------------ GPU compression

def test_gpu_compression_exact_at_full_rank(dm):
    n = 256
    X = _scurve(n, 3)
    eps = O.median_sqdist(X)
    _, _, s = O.degrees(X, eps, 1.0)
    h = dm.dm_create(X, eps=eps)
    dm.dm_compress(h, 0.0, 32, 256)
    x = synth.random_rhs(n, 1, seed=8)[:, 0].astype(np.float32)
    y = dm.dm_matvec(h, x)
    yr = O.S_matvec(X, eps, s, x.astype(np.float64))
    assert _rel_inf(y, yr, np.abs(x).max()) < 2e-5


@pytest.mark.parametrize("n,leaf,rank,tol,kind", [(2048, 128, 64, 1e-5, "scurve"), (3001, 200, 48, 1e-4, "scurve"),
                                                  (2500, 160, 64, 1e-4, "mixture64"), (1800, 128, 64, 1e-4, "mnist"),
                                                  (6000, 256, 128, 1e-5, "scurve"), (3000, 256, 128, 1e-4, "mnist")])
def test_gpu_compression_accuracy_and_structure(dm, n, leaf, rank, tol, kind):
    """GPU compression: valid structure and an error against the exact operator next to the
    oracle's own compression; the high-dimensional cases (d = 64, 784) build their sampled
    blocks and near blocks with the coordinate-tiled entry kernel. At rank 128 the sampled
    blocks (266 rows x up to 256 candidates) exceed one CTA's shared memory: those levels run
    the clustered ID (the block split by columns over a cluster of CTAs)."""
    if kind == "scurve":
        X = _scurve(n, 4)
    elif kind == "mixture64":
        X = synth.as_f32(synth.gaussian_mixture(n, d=64, seed=4))
    else:
        X = synth.as_f32(synth.mnist_like(n, seed=4))
    eps = O.median_sqdist(X)
    _, _, s = O.degrees(X, eps, 1.0)
    h = dm.dm_create(X, eps=eps)
    dm.dm_compress(h, tol, leaf, rank)
    perm, L = dm.dm_get_tree(h)
    ranks, skel, P = dm.dm_get_hmatrix(h)
    st = dm.dm_get_stats(h)
    cmax = max(st["leaf_max"], 2 * rank)
    P = P.reshape(-1, rank, cmax)
    # structure: ranks within caps; skeletons are candidates; P(:, J) = I
    assert ranks[0] == 0 and ranks[1:].max() <= rank and ranks[1:].min() >= 1
    for node in range(1, len(ranks)):
        r = ranks[node]
        J = skel[node * rank:node * rank + r]
        st0, sz = O.node_range(n, node)
        lvl = int(math.log2(node + 1))
        if lvl == L:
            C = np.arange(st0, st0 + sz)
        else:
            l, rr = 2 * node + 1, 2 * node + 2
            C = np.concatenate([skel[l * rank:l * rank + ranks[l]], skel[rr * rank:rr * rank + ranks[rr]]])
        assert set(J.tolist()) <= set(C.tolist())
        cols = [int(np.where(C == j)[0][0]) for j in J]
        np.testing.assert_array_equal(P[node][:r, cols], np.eye(r, dtype=np.float32))
    # accuracy against the exact operator, next to the oracle's own compression
    x = synth.random_rhs(n, 1, seed=9)[:, 0]
    yr = O.S_matvec(X, eps, s, x)
    y = dm.dm_matvec(h, x.astype(np.float32))
    err_gpu = np.linalg.norm(y - yr) / np.linalg.norm(yr)
    Ho = O.compress(X, eps, s, leaf, tol, rank)
    err_or = np.linalg.norm(O.hmatvec(X, eps, s, Ho, x) - yr) / np.linalg.norm(yr)
    # The GPU draws the same seeded rows and takes the same candidates; its FP32 pivot and
    # rank decisions can differ from the oracle's FP64 ones only where two residual norms
    # tie within FP32 rounding (~1e-6 relative), which moves the compression error by far
    # less than 2% (measured ratio 1.000-1.001 on all four cases); the FP32 evaluation adds
    # ~1e-7 relative (the additive term).
    print(f"compression error: gpu {err_gpu:.3e} oracle {err_or:.3e} ratio {err_gpu / max(err_or, 1e-300):.3f}")
    assert err_gpu <= 1.02 * err_or + 1e-6, (err_gpu, err_or)


@pytest.mark.parametrize("n,leaf,rank,tol", [(2048, 128, 64, 1e-5), (3000, 128, 128, 1e-5)])
def test_gpu_compression_error_in_the_operator_2norm(dm, n, leaf, rank, tol):
    """||S~_gpu - S||_2 (Eq. 1.1 in the operator 2-norm, relative since ||S||_2 = 1) by power
    iteration on (S~_gpu - S)^2, next to the oracle's own compression's
    oracle.hmatvec_error_2norm. Both products see the same FP32-representable vector each
    iteration, so the GPU side adds only its FP32 arithmetic (~1e-7); pivot choices that
    differ where residual norms tie within FP32 rounding move the error by far less than 5%.
    The rank-128 case runs its internal levels on the clustered ID."""
    X = _scurve(n, 7)
    eps = O.median_sqdist(X)
    _, _, s = O.degrees(X, eps, 1.0)
    h = dm.dm_create(X, eps=eps)
    dm.dm_compress(h, tol, leaf, rank)
    v = O.start_vector(n, 0)
    v /= np.linalg.norm(v)
    est_gpu = 0.0
    for _ in range(60):
        v32 = v.astype(np.float32)
        e = dm.dm_matvec(h, v32).astype(np.float64) - O.S_matvec(X, eps, s, v32.astype(np.float64))
        est_gpu = float(np.linalg.norm(e)) / float(np.linalg.norm(v32.astype(np.float64)))
        e32 = e.astype(np.float32)
        w = dm.dm_matvec(h, e32).astype(np.float64) - O.S_matvec(X, eps, s, e32.astype(np.float64))
        v = w / np.linalg.norm(w)
    dm.dm_destroy(h)
    Ho = O.compress(X, eps, s, leaf, tol, rank)
    est_or = O.hmatvec_error_2norm(X, eps, s, Ho, iters=60)
    print(f"||S~ - S||_2: gpu {est_gpu:.3e} oracle {est_or:.3e} ratio {est_gpu / est_or:.3f}")
    assert est_gpu <= 1.05 * est_or + 2e-6, (est_gpu, est_or)


# ------------------------------------------------------------------ Lanczos

def test_eigs_replayed_structure_match_oracle_lanczos(dm):
    n = 2048
    X = _scurve(n, 0)
    eps = O.median_sqdist(X)
    _, dg, s = O.degrees(X, eps, 1.0)
    H = O.compress(X, eps, s, 128, 1e-5, 64)
    evo, Vo, _, sto = O.lanczos_hmat(X, eps, s, H, 10, conv_tol=1e-10)
    assert sto == 0
    h = dm.dm_create(X, eps=eps)
    dm.dm_load_hmatrix(h, H.L, H.max_rank, H.perm, H.ranks, H.skel, H.P.astype(np.float32))
    ev, V, conv = dm.dm_eigs(h, 10)
    assert conv
    np.testing.assert_allclose(ev, evo, rtol=2e-5, atol=2e-7)
    angles = []
    for i in range(10):
        c = abs(float(np.dot(V[:, i].astype(np.float64), Vo[:, i])))
        angles.append(math.acos(min(1.0, c)))
        assert angles[-1] < 2e-3
    # diffusion coordinates (Algorithm 1: eigenvalues theta^t of P^t, right eigenvectors
    # Dg^-1/2 phi) against the oracle's coordinates of the oracle's own eigenpairs and
    # degrees. Per column: an eigenvector off by angle a moves psi by ~a relative, the
    # eigenvalue's relative error enters t times, and FP32 storage adds ~1e-6; a wrong
    # power of theta (>= 30% off for every non-trivial pair here) or a missing Dg^-1/2
    # fails by orders of magnitude.
    for t in (1, 3):
        psi = dm.dm_coords(h, 10, t).astype(np.float64)
        want = O.diffusion_coords(evo, Vo, dg, t)
        for i in range(10):
            sgn = 1.0 if np.dot(psi[:, i], want[:, i]) >= 0 else -1.0
            err = np.linalg.norm(sgn * psi[:, i] - want[:, i]) / np.linalg.norm(want[:, i])
            bound = 2.0 * angles[i] + t * abs(ev[i] - evo[i]) / evo[i] + 5e-6
            assert err <= bound, (t, i, err, bound)


@pytest.mark.parametrize("b,k,prec", [(8, 10, 0), (16, 10, 0), (4, 6, 0), (16, 10, 1), (16, 10, 2)])
def test_block_lanczos_replayed_structure_match_oracle(dm, b, k, prec):
    """Block Lanczos (b vectors per step, block H-matvec, block CGS2, CholQR2, FP64
    Rayleigh-Ritz through Householder tridiagonalisation) finds the same eigenpairs of the
    same operator as the oracle's single-vector Lanczos. With the TF32 near field the
    operator differs from the oracle's by E with |E|_2 <= 2 * 2^-10 |S_near|_2 <= 2^-9 (each
    near term truncated in both factors; a diagonal block of the PSD S has norm <= |S| = 1):
    eigenvalues are held to Weyl's bound |E|_2 and eigenvectors to Davis-Kahan's
    sin(angle) <= |E|_2 / gap."""
    n = 2048
    X = _scurve(n, 0)
    eps = O.median_sqdist(X)
    _, dg, s = O.degrees(X, eps, 1.0)
    H = O.compress(X, eps, s, 128, 1e-5, 64)
    evo1, Vo1, _, sto = O.lanczos_hmat(X, eps, s, H, k + 1, conv_tol=1e-10)
    assert sto == 0
    evo, Vo = evo1[:k], Vo1[:, :k]
    cfg = dm.dm_config_default(block_size=b, block_precision=prec, near_mode=dm.DM_NEAR_CACHED)
    h = dm.dm_create(X, eps=eps, cfg=cfg)
    dm.dm_load_hmatrix(h, H.L, H.max_rank, H.perm, H.ranks, H.skel, H.P.astype(np.float32))
    ev, V, conv = dm.dm_eigs(h, k)
    assert conv
    weyl = 2.0 ** -9
    if prec != 1:  # FP32, or the split TF32 near field (2^-20 per term: within the FP32 tolerance)
        np.testing.assert_allclose(ev, evo, rtol=2e-5, atol=2e-7)
    else:
        assert np.abs(ev - evo).max() <= weyl
    G = V.astype(np.float64).T @ V.astype(np.float64)
    assert np.abs(G - np.eye(k)).max() < 2e-5
    for i in range(k):
        c = abs(float(np.dot(V[:, i].astype(np.float64), Vo[:, i])))
        if prec != 1:
            assert math.acos(min(1.0, c)) < 2e-3
        else:
            gap = min(abs(evo1[i] - evo1[j]) for j in range(k + 1) if j != i)
            assert math.sqrt(max(0.0, 1.0 - c * c)) <= weyl / gap
    st = dm.dm_get_stats(h)
    assert st["lanczos_iters"] % b == 0
    dm.dm_destroy(h)


@pytest.mark.parametrize("b,k,m_max", [(4, 10, 32), (2, 8, 22), (4, 20, 44), (3, 6, 20)])
def test_thick_restart_matches_unrestarted_oracle(dm, b, k, m_max):
    """Thick restart (the explicit form of Section 2.3's implicit restart with exact shifts):
    with a basis capped below what the unrestarted solve needs, block Lanczos keeps k + p
    Ritz vectors and the newest block at each restart. Its eigenpairs must be those of the
    oracle's unrestarted FP64 Lanczos on the same replayed structure, and the basis must
    really have been restarted (more vectors generated than the cap)."""
    n = 2048
    X = _scurve(n, 0)
    eps = O.median_sqdist(X)
    _, dg, s = O.degrees(X, eps, 1.0)
    H = O.compress(X, eps, s, 128, 1e-5, 64)
    evo1, Vo1, _, sto = O.lanczos_hmat(X, eps, s, H, k + 1, conv_tol=1e-10)
    assert sto == 0
    evo, Vo = evo1[:k], Vo1[:, :k]
    cfg = dm.dm_config_default(block_size=b, m_max=m_max, near_mode=dm.DM_NEAR_CACHED)
    h = dm.dm_create(X, eps=eps, cfg=cfg)
    dm.dm_load_hmatrix(h, H.L, H.max_rank, H.perm, H.ranks, H.skel, H.P.astype(np.float32))
    ev, V, conv = dm.dm_eigs(h, k)
    assert conv
    st = dm.dm_get_stats(h)
    assert st["lanczos_iters"] > m_max, st["lanczos_iters"]
    np.testing.assert_allclose(ev, evo, rtol=2e-5, atol=2e-7)
    G = V.astype(np.float64).T @ V.astype(np.float64)
    assert np.abs(G - np.eye(k)).max() < 2e-5
    for i in range(k):
        c = abs(float(np.dot(V[:, i].astype(np.float64), Vo[:, i])))
        assert math.acos(min(1.0, c)) < 2e-3
    dm.dm_destroy(h)


def test_eigs_c1_workload_against_dense_oracle(dm):
    """2048-point s-curve, leaf 128, rank 64, tol 1e-5, top 10 (the small parity workload)."""
    import json
    import os

    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "scurve_n2048.json")))
    X = _scurve(2048, 0)
    h = dm.dm_create(X, eps=-1.0)
    assert dm.dm_get_eps(h) == g["eps"]
    dm.dm_compress(h, 1e-5, 128, 64)
    ev, V, conv = dm.dm_eigs(h, 10)
    assert conv
    ref = np.array(g["evals_top10"])
    rel = np.abs(ev - ref) / ref
    assert rel.max() < 1e-4, rel
    assert abs(ev[0] - 1.0) < 1e-5
    # orthonormal, signed eigenvectors
    G = V.astype(np.float64).T @ V.astype(np.float64)
    np.testing.assert_allclose(G, np.eye(10), atol=2e-5)
    for i in range(10):
        assert V[np.argmax(np.abs(V[:, i])), i] > 0
    # subspace angle against the exact eigenvectors
    q, dg, s = O.degrees(X, g["eps"], 1.0)
    _, Vo, _, _ = O.lanczos_S(X, g["eps"], s, 10, conv_tol=1e-10)
    sv = np.linalg.svd(Vo.T @ V.astype(np.float64), compute_uv=False)
    assert math.acos(min(1.0, sv.min())) < 1e-3
    # diffusion coordinates psi = theta^t Dg^-1/2 phi against the oracle's coordinates of
    # the exact operator's eigenpairs: the four leading pairs are well separated, so each
    # column agrees to the approximation error of tol 1e-5 (measured ~1e-5 relative)
    evx, Vx, _, _ = O.lanczos_S(X, g["eps"], s, 4, conv_tol=1e-10)
    psi = dm.dm_coords(h, 4, 2).astype(np.float64)
    want = O.diffusion_coords(evx, Vx, dg, 2)
    for i in range(4):
        sgn = 1.0 if np.dot(psi[:, i], want[:, i]) >= 0 else -1.0
        assert np.linalg.norm(sgn * psi[:, i] - want[:, i]) / np.linalg.norm(want[:, i]) < 1e-3


def test_eigs_state_errors(dm):
    X = _scurve(300, 1)
    h = dm.dm_create(X, eps=-1.0)
    with pytest.raises(dm.DmError) as e:
        dm.dm_eigs(h, 3)
    assert e.value.status == dm.DM_ESTATE
    dm.dm_compress(h, 1e-5, 64, 16)
    with pytest.raises(dm.DmError) as e:
        dm.dm_eigs(h, 0)
    assert e.value.status == dm.DM_EINVAL
    with pytest.raises(dm.DmError) as e:
        dm.dm_compress(h, -1.0, 64, 16)
    assert e.value.status == dm.DM_EINVAL
