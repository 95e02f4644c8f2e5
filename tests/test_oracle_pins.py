"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test ties one oracle routine to a closed form, an invariant of the
diffusion-map construction (Algorithm 1, Eq. W, Eq. 2.18, Algorithm 2), brute
force on tiny inputs, or a library special case, so that a dropped term, a
wrong sign or index or a transposed operand in oracle.c fails at least one.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _scurve(n, seed=0):
    return synth.as_f32(synth.s_curve(n, seed))


# ---------------------------------------------------------------- generator

def test_splitmix64_published_outputs():
    want = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l.startswith("0x")]
    assert O.splitmix64_sequence(0, 3) == want


def test_counter_stream_is_the_sequential_generator():
    # or_rng(key, c) must be the (c+1)-th output of the sequential generator started at key
    key = O.stream_key(7, 1, 42)
    assert [O.rng(key, c) for c in range(5)] == O.splitmix64_sequence(key, 5)


# ---------------------------------------------------------------- kernel, bandwidth, degrees

def test_sqdist_bruteforce():
    X = _scurve(20, 3)
    Xd = X.astype(np.float64)
    for i, j in [(0, 1), (5, 19), (7, 7)]:
        assert O.sqdist(X, i, j) == pytest.approx(float(np.sum((Xd[i] - Xd[j]) ** 2)), rel=1e-15, abs=0)


def test_median_all_pairs_matches_numpy():
    X = _scurve(301, 5)  # 45150 pairs (odd count -> the middle value)
    Xd = X.astype(np.float64)
    iu = np.triu_indices(301, 1)
    d2 = np.sum((Xd[iu[0]] - Xd[iu[1]]) ** 2, axis=1)
    assert O.median_sqdist(X) == pytest.approx(float(np.median(d2)), rel=1e-15)
    X2 = _scurve(300, 6)  # even count -> mean of the two middle values
    Xd = X2.astype(np.float64)
    iu = np.triu_indices(300, 1)
    d2 = np.sum((Xd[iu[0]] - Xd[iu[1]]) ** 2, axis=1)
    assert O.median_sqdist(X2) == pytest.approx(float(np.median(d2)), rel=1e-15)


def test_median_sampled_pairs():
    n = 1500  # 1,124,250 pairs > 2^20 -> 2^20 seeded pairs
    X = _scurve(n, 2)
    Xd = X.astype(np.float64)
    key = O.stream_key(11, 3, 0)
    m = 1 << 20
    u = np.array(O.splitmix64_sequence(key, 2 * m), dtype=np.uint64)
    i = ((u[0::2] >> np.uint64(32)) * np.uint64(n)) >> np.uint64(32)
    j = ((u[1::2] >> np.uint64(32)) * np.uint64(n - 1)) >> np.uint64(32)
    j = j + (j >= i)
    i, j = i.astype(np.int64), j.astype(np.int64)
    assert np.all(i != j)
    d2 = np.sum((Xd[i] - Xd[j]) ** 2, axis=1)
    assert O.median_sqdist(X, seed=11) == pytest.approx(float(np.median(d2)), rel=1e-15)


def test_degrees_bruteforce_tiny():
    X = _scurve(9, 4)
    eps, alpha = 0.7, 1.0
    pts = [[float(v) for v in row] for row in X]
    n = len(pts)

    def w(i, j):
        return math.exp(-sum((a - b) ** 2 for a, b in zip(pts[i], pts[j])) / eps)

    q = [sum(w(i, j) for j in range(n)) for i in range(n)]
    walpha = [[w(i, j) / (q[i] ** alpha * q[j] ** alpha) for j in range(n)] for i in range(n)]
    dg = [sum(r) for r in walpha]
    s = [q[i] ** -alpha / math.sqrt(dg[i]) for i in range(n)]
    oq, odg, os_ = O.degrees(X, eps, alpha)
    np.testing.assert_allclose(oq, q, rtol=1e-14)
    np.testing.assert_allclose(odg, dg, rtol=1e-14)
    np.testing.assert_allclose(os_, s, rtol=1e-14)


@pytest.mark.parametrize("alpha", [1.0, 0.5, 0.0])
def test_markov_rows_sum_to_one(alpha):
    X = _scurve(200, 1)
    eps = O.median_sqdist(X)
    W = O.kernel_W(X, eps)
    q, dg, s = O.degrees(X, eps, alpha)
    Wa = W / np.outer(q ** alpha, q ** alpha)
    P = Wa / dg[:, None]  # Algorithm 1's Markov normalisation with the row-sum denominator
    np.testing.assert_allclose(P.sum(axis=1), 1.0, rtol=0, atol=1e-13)
    # S = diag(s) W diag(s) is the symmetric conjugate Dg^1/2 P Dg^-1/2
    S = s[:, None] * W * s[None, :]
    np.testing.assert_allclose(S, np.sqrt(dg)[:, None] * P / np.sqrt(dg)[None, :], rtol=1e-12, atol=0)


def test_alpha_zero_special_case():
    X = _scurve(150, 2)
    eps = O.median_sqdist(X)
    q, dg, s = O.degrees(X, eps, 0.0)
    np.testing.assert_allclose(dg, q, rtol=1e-14)  # W^0 = W
    np.testing.assert_allclose(s, q ** -0.5, rtol=1e-14)


def test_top_eigenpair_is_one_and_sqrt_degree():
    X = _scurve(300, 8)
    eps = O.median_sqdist(X)
    q, dg, s = O.degrees(X, eps, 1.0)
    phi = np.sqrt(dg)
    y = O.S_matvec(X, eps, s, phi)
    np.testing.assert_allclose(y, phi, rtol=1e-13)
    W = O.kernel_W(X, eps)
    ev, V = O.jacobi(s[:, None] * W * s[None, :])
    assert ev[0] == pytest.approx(1.0, abs=1e-13)
    v = V[:, 0] * np.sign(V[0, 0])
    np.testing.assert_allclose(v, phi / np.linalg.norm(phi) * np.sign(phi[0]), atol=1e-12)
    assert ev[1] < 1.0 - 1e-6


@pytest.mark.parametrize("n,eps", [(64, 0.5), (101, 2.0), (48, 0.05)])
def test_circle_closed_form_spectrum(n, eps):
    """Equally spaced points on a circle: W is circulant (w_k = exp(-(2R sin(pi k/n))^2/eps)),
    q is constant, S = W / sum_k w_k and its eigenvalues are the DFT of w over sum w.
    Float32 storage of the coordinates perturbs distances by ~1e-7, hence the tolerance."""
    X = synth.as_f32(synth.circle(n, 1.0))
    wk = np.array([math.exp(-(2.0 * math.sin(math.pi * k / n)) ** 2 / eps) for k in range(n)])
    lam = np.array([sum(wk[k] * math.cos(2 * math.pi * k * m / n) for k in range(n)) for m in range(n)]) / wk.sum()
    q, dg, s = O.degrees(X, eps, 1.0)
    np.testing.assert_allclose(q, wk.sum(), rtol=1e-6)
    W = O.kernel_W(X, eps)
    ev, _ = O.jacobi(s[:, None] * W * s[None, :])
    np.testing.assert_allclose(ev, np.sort(lam)[::-1], rtol=0, atol=2e-6)


# ---------------------------------------------------------------- dense eigensolvers

def test_jacobi_matches_library_eigh():
    g = np.random.default_rng(3)
    B = g.normal(size=(40, 40))
    A = B + B.T
    ev, V = O.jacobi(A)
    ref = np.linalg.eigh(A)[0][::-1]
    np.testing.assert_allclose(ev, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    np.testing.assert_allclose(V.T @ V, np.eye(40), atol=1e-12)
    np.testing.assert_allclose(A @ V, V * ev[None, :], atol=1e-11)


def test_jacobi_tridiagonal_closed_form():
    n = 37
    A = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    ev, _ = O.jacobi(A)
    want = np.sort(2 - 2 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1)))[::-1]
    np.testing.assert_allclose(ev, want, atol=1e-13)


def test_lanczos_on_diagonal_matrix():
    n = 200
    d = np.linspace(0.0, 1.0, n) ** 3
    ev, V, it, st = O.lanczos_dense(np.diag(d), k=6, conv_tol=1e-12)
    assert st == 0
    np.testing.assert_allclose(ev, np.sort(d)[::-1][:6], atol=1e-13)
    for i in range(6):
        j = n - 1 - i
        assert abs(abs(V[j, i]) - 1.0) < 1e-9


def test_lanczos_matches_jacobi_on_S():
    X = _scurve(400, 9)
    eps = O.median_sqdist(X)
    q, dg, s = O.degrees(X, eps, 1.0)
    W = O.kernel_W(X, eps)
    S = s[:, None] * W * s[None, :]
    evj, Vj = O.jacobi(S)
    k = 10
    ev, V, it, st = O.lanczos_S(X, eps, s, k, conv_tol=1e-12)
    assert st == 0 and it < 200
    np.testing.assert_allclose(ev, evj[:k], rtol=1e-11)
    for i in range(k):
        c = abs(float(V[:, i] @ Vj[:, i]))
        assert math.acos(min(1.0, c)) < 1e-6
    # sign convention: largest-magnitude entry positive
    for i in range(k):
        assert V[np.argmax(np.abs(V[:, i])), i] > 0


# ---------------------------------------------------------------- tree

def test_tree_depth_and_ranges():
    assert O.tree_depth(100_000, 512) == 8
    assert O.tree_depth(2048, 128) == 4
    assert O.tree_depth(60_000, 256) == 8
    assert O.tree_depth(512, 512) == 0
    assert O.tree_depth(513, 512) == 1
    n, L = 100_000, 8
    sizes = [O.node_range(n, (1 << L) - 1 + k)[1] for k in range(1 << L)]
    assert sum(sizes) == n and set(sizes) == {390, 391}
    st = 0
    for k in range(1 << L):
        s0, sz = O.node_range(n, (1 << L) - 1 + k)
        assert s0 == st
        st += sz


def test_tree_split_rule_bruteforce():
    n, leaf = 700, 60
    X = _scurve(n, 12)
    Xd = X.astype(np.float64)
    eps = O.median_sqdist(X)
    perm, L = O.tree(X, eps, leaf)
    assert sorted(perm.tolist()) == list(range(n))
    assert L == O.tree_depth(n, leaf)

    def W(i, idx):
        return np.exp(-np.sum((Xd[idx] - Xd[i]) ** 2, axis=1) / eps)

    for node in range((1 << L) - 1):
        st, sz = O.node_range(n, node)
        idx = np.sort(perm[st:st + sz])
        lst, lsz = O.node_range(n, 2 * node + 1)
        left = perm[lst:lst + lsz]
        right = perm[lst + lsz:st + sz]
        assert lsz == (sz + 1) // 2
        i0 = idx[0]
        # farthest in the Gram distance 2 - 2 W: largest squared distance, lowest index on ties
        r0 = np.sum((Xd[idx] - Xd[i0]) ** 2, axis=1)
        p = idx[np.lexsort((idx, -r0))[0]]
        assert W(i0, idx)[np.searchsorted(idx, p)] == W(i0, idx).min()
        rp = np.sum((Xd[idx] - Xd[p]) ** 2, axis=1)
        q = idx[np.lexsort((idx, -rp))[0]]
        wp = W(p, idx)
        key = {int(i): float(v) for i, v in zip(idx, W(q, idx) - wp)}
        kl = max((key[int(i)], int(i)) for i in left)
        kr = min((key[int(i)], int(i)) for i in right)
        assert kl < kr
    # leaves keep their points in increasing original index
    for k in range(1 << L):
        st, sz = O.node_range(n, (1 << L) - 1 + k)
        assert np.all(np.diff(perm[st:st + sz]) > 0)


# ---------------------------------------------------------------- skeletonization and HSS matvec

def _setup(n, seed, leaf):
    X = _scurve(n, seed)
    eps = O.median_sqdist(X)
    q, dg, s = O.degrees(X, eps, 1.0)
    return X, eps, s


def test_hmatvec_exact_at_zero_tolerance_full_rank():
    X, eps, s = _setup(256, 3, 32)
    H = O.compress(X, eps, s, 32, 0.0, 256)
    x = synth.random_rhs(256, 3, 5)
    y = O.S_matvec(X, eps, s, x)
    yh = O.hmatvec(X, eps, s, H, x)
    np.testing.assert_allclose(yh, y, rtol=0, atol=1e-13 * np.abs(y).max())


def test_interpolative_decomposition_exact_low_rank_block():
    """With every off-node row sampled and tol 0, each node's ID reproduces its sampled
    block exactly: K(R, C) = K(R, J) P with P(:, J) = I."""
    n = 256
    X, eps, s = _setup(n, 4, 32)
    perm, L = O.tree(X, eps, 32)
    H = O.skeletonize(X, eps, s, perm, L, 0.0, 40, seed=0)  # rank cap 40 < leaf: P nontrivial
    W = O.kernel_W(X, eps)
    K = s[:, None] * W * s[None, :]
    Kp = K[np.ix_(perm, perm)]
    for node in [(1 << L) - 1, (1 << L), 3, 1]:
        st, sz = O.node_range(n, node)
        r = H.ranks[node]
        lvl = int(math.log2(node + 1))
        if lvl == L:
            C = np.arange(st, st + sz)
        else:
            l, rr = 2 * node + 1, 2 * node + 2
            C = np.concatenate([H.skel[l * H.max_rank:l * H.max_rank + H.ranks[l]],
                                H.skel[rr * H.max_rank:rr * H.max_rank + H.ranks[rr]]])
        Pn = H.P[node * H.max_rank * H.cmax:(node + 1) * H.max_rank * H.cmax].reshape(H.max_rank, H.cmax)[:r, :len(C)]
        J = H.skel[node * H.max_rank:node * H.max_rank + r]
        off = np.concatenate([np.arange(0, st), np.arange(st + sz, n)])
        A = Kp[np.ix_(off, C)]
        # skeleton columns are identity columns of P
        cols = [int(np.where(C == j)[0][0]) for j in J]
        np.testing.assert_allclose(Pn[:, cols], np.eye(r), atol=0)
        err = np.linalg.norm(A - Kp[np.ix_(off, J)] @ Pn) / np.linalg.norm(A)
        # rank-capped ID: error at most the discarded singular part, and exact when rank == |C|
        if r == len(C):
            assert err < 1e-13
        else:
            sv = np.linalg.svd(A, compute_uv=False)
            assert err <= 50 * sv[r] / sv[0] + 1e-14


def test_hmatvec_error_decreases_with_tolerance():
    n = 1024
    X, eps, s = _setup(n, 6, 64)
    x = synth.random_rhs(n, 1, 2)[:, 0]
    y = O.S_matvec(X, eps, s, x)
    errs = []
    for tol in [1e-2, 1e-4, 1e-6, 1e-8]:
        H = O.compress(X, eps, s, 64, tol, 64)
        errs.append(np.linalg.norm(O.hmatvec(X, eps, s, H, x) - y) / np.linalg.norm(y))
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[1] < 1e-2 and errs[3] < 1e-5


def test_hmatvec_is_symmetric():
    """Far field is P_l^T K(S_l,S_r) P_r + its transpose: x^T K~ y = y^T K~ x."""
    n = 900
    X, eps, s = _setup(n, 7, 50)
    H = O.compress(X, eps, s, 50, 1e-3, 20)
    xy = synth.random_rhs(n, 2, 9)
    a = float(xy[:, 0] @ O.hmatvec(X, eps, s, H, xy[:, 1]))
    b = float(xy[:, 1] @ O.hmatvec(X, eps, s, H, xy[:, 0]))
    assert abs(a - b) <= 1e-13 * abs(a)


def test_rank_caps():
    n = 1000
    X, eps, s = _setup(n, 2, 100)
    H = O.compress(X, eps, s, 100, 1e-12, 17)
    assert H.ranks[0] == 0
    assert H.ranks[1:].max() <= 17
    assert np.all(H.ranks[1:] >= 1)


def test_lanczos_on_hmatrix_approaches_exact():
    n = 1024
    X, eps, s = _setup(n, 1, 64)
    ev, _, _, st = O.lanczos_S(X, eps, s, 8, conv_tol=1e-11)
    assert st == 0
    errs = []
    for tol in [1e-3, 1e-6]:
        H = O.compress(X, eps, s, 64, tol, 64)
        evh, _, _, sth = O.lanczos_hmat(X, eps, s, H, 8, conv_tol=1e-11)
        assert sth == 0
        errs.append(np.max(np.abs(evh - ev) / ev))
    assert errs[1] < errs[0] and errs[1] < 1e-5


def test_golden_scurve_2048_regression():
    """Oracle output at the 2048-point s-curve workload, stored by tests/golden/make_golden.py."""
    import json
    g = json.load(open(os.path.join(GOLDEN, "scurve_n2048.json")))
    X = _scurve(2048, 0)
    eps = O.median_sqdist(X)
    assert eps == pytest.approx(g["eps"], rel=1e-15)
    q, dg, s = O.degrees(X, eps, 1.0)
    ev, _, _, st = O.lanczos_S(X, eps, s, 10, conv_tol=1e-10)
    assert st == 0
    np.testing.assert_allclose(ev, g["evals_top10"], rtol=1e-10)


# ------------------------------------------------------------------ intrinsic dimension d(t) (Algorithm 1)

def test_intrinsic_dim_worked_example():
    """lambda = 1, 0.8, 0.6, 0.3, 0.1 and delta = 0.2, powers worked out by hand:
    t = 1: threshold 0.16 passes 0.8, 0.6, 0.3 -> 3; t = 2: 0.128 passes 0.64, 0.36 -> 2;
    t = 5: 0.065536 passes 0.32768, 0.07776 -> 2; t = 6: 0.0524288 passes 0.262144 only -> 1."""
    lam = [1.0, 0.8, 0.6, 0.3, 0.1]
    assert O.intrinsic_dim(lam, 1, 0.2) == (3, False)
    assert O.intrinsic_dim(lam, 2, 0.2) == (2, False)
    assert O.intrinsic_dim(lam, 5, 0.2) == (2, False)
    assert O.intrinsic_dim(lam, 6, 0.2) == (1, False)
    assert O.intrinsic_dim(lam, 1, 0.01) == (4, True)  # all pass: more pairs needed
    assert O.intrinsic_dim([1.0, 0.0, 0.0], 1, 0.5) == (0, False)


def test_intrinsic_dim_bruteforce_exact_powers():
    """Against the definition evaluated in exact rational arithmetic (|lambda_l|^t vs
    delta |lambda_1|^t), on random spectra away from exact ties."""
    from fractions import Fraction

    rng = np.random.default_rng(7)
    checked = 0
    for _ in range(400):
        k = int(rng.integers(2, 12))
        lam = [Fraction(1)] + sorted((Fraction(int(v), 1000) for v in rng.integers(-999, 1000, k - 1)),
                                     reverse=True)
        t = int(rng.integers(1, 9))
        delta = Fraction(int(rng.integers(1, 100)), 100)
        thr = delta * abs(lam[1]) ** t
        if any(abs(abs(x) ** t - thr) <= Fraction(1, 10**9) * max(thr, Fraction(1, 10**30)) for x in lam[1:]):
            continue
        want = max([l for l in range(1, k) if abs(lam[l]) ** t > thr], default=0)
        got, at_k = O.intrinsic_dim([float(x) for x in lam], t, float(delta))
        assert got == want, (lam, t, delta)
        assert at_k == (want == k - 1)
        checked += 1
    assert checked > 300


def test_intrinsic_dim_non_increasing_in_t():
    rng = np.random.default_rng(8)
    for _ in range(50):
        lam = np.concatenate([[1.0], np.sort(rng.random(15))[::-1]])
        ds = [O.intrinsic_dim(lam, t, 0.1)[0] for t in range(1, 40)]
        assert all(a >= b for a, b in zip(ds, ds[1:]))


def test_residual_bound_identity_of_the_ritz_check():
    """The convergence check's residual bound uses |y_m|^2 = |p_{m-1}(theta) / p_m'(theta)|
    (y the unit eigenvector of T_m for theta, p_i the characteristic polynomials of the
    leading i x i submatrices): checked against numpy's eigh on random tridiagonals."""
    rng = np.random.default_rng(21)
    for _ in range(20):
        m = int(rng.integers(5, 40))
        a, b = rng.uniform(-1, 1, m), rng.uniform(0.05, 1, m - 1)
        T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
        w, Y = np.linalg.eigh(T)
        for i in range(m):
            th = w[i]
            pm, p, dpm, dp = 1.0, a[0] - th, 0.0, -1.0
            for r in range(1, m):
                t = a[r] - th
                pm, p, dpm, dp = p, t * p - b[r - 1] ** 2 * pm, dp, t * dp - p - b[r - 1] ** 2 * dpm
            # p_{m-1} = pm, p_m' = dp
            assert abs(abs(pm / dp) - Y[m - 1, i] ** 2) < 1e-8 * max(1.0, Y[m - 1, i] ** 2)


@pytest.mark.parametrize("alpha", [1.0, 0.5])
def test_diffusion_coords_are_right_eigenvectors_of_P(alpha):
    """psi_i(t) = theta_i^t Dg^-1/2 phi_i: P psi_i(0) = theta_i psi_i(0) for the dense
    Markov matrix P = Dg^-1 W^alpha built from the kernel, and P^t psi_i(0) = psi_i(t)."""
    X = synth.as_f32(synth.s_curve(300, seed=5))
    eps = O.median_sqdist(X)
    q, dg, s = O.degrees(X, eps, alpha)
    W = O.kernel_W(X, eps)
    Wa = W / np.outer(q ** alpha, q ** alpha)
    P = Wa / dg[:, None]
    S = s[:, None] * W * s[None, :]
    ev, V = O.jacobi(S)
    k = 6
    psi0 = O.diffusion_coords(ev[:k], V[:, :k], dg, 0)
    np.testing.assert_allclose(P @ psi0, psi0 * ev[:k][None, :], rtol=0, atol=1e-10)
    psi3 = O.diffusion_coords(ev[:k], V[:, :k], dg, 3)
    np.testing.assert_allclose(np.linalg.matrix_power(P, 3) @ psi0, psi3, rtol=0, atol=1e-10)


@pytest.mark.parametrize("tol", [1e-2, 1e-4, 1e-6])
def test_id_pivots_and_rank_match_lapack_pivoted_qr(tol):
    """The ID's pivot order and its stopping rule (stop at the first pivot whose residual
    column norm is <= tol x the first pivot's) against LAPACK's column-pivoted QR
    (scipy.linalg.qr, pivoting=True) of the same sampled block, where every off-node
    row is sampled (n = 128, leaf 32, max rank 48: at most 106 rows per node)."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    n, leaf, max_rank = 128, 32, 48
    X, eps, s = _setup(n, 9, leaf)
    perm, L = O.tree(X, eps, leaf)
    H = O.skeletonize(X, eps, s, perm, L, tol, max_rank, seed=0)
    W = O.kernel_W(X, eps)
    Kp = (s[:, None] * W * s[None, :])[np.ix_(perm, perm)]
    compared = 0
    for node in range(1, (1 << (L + 1)) - 1):
        st, sz = O.node_range(n, node)
        if int(math.log2(node + 1)) == L:
            C = np.arange(st, st + sz)
        else:
            l, rr = 2 * node + 1, 2 * node + 2
            C = np.concatenate([H.skel[l * max_rank:l * max_rank + H.ranks[l]],
                                H.skel[rr * max_rank:rr * max_rank + H.ranks[rr]]])
        off = np.concatenate([np.arange(0, st), np.arange(st + sz, n)])
        A = Kp[np.ix_(off, C)]
        _, R, piv = scipy_linalg.qr(A, pivoting=True, mode="economic")
        d = np.abs(np.diag(R))
        kmax = min(max_rank, len(C), len(off))
        thr = tol * d[0]
        r_lapack = next((j for j in range(kmax) if d[j] <= thr), kmax)
        if np.any(np.abs(d[:kmax + 1] - thr) <= 1e-9 * thr):
            continue  # a residual norm at the threshold within rounding: no sharp answer
        r = H.ranks[node]
        assert r == r_lapack, (node, r, r_lapack)
        J = H.skel[node * max_rank:node * max_rank + r]
        # pivots agree until two residual norms tie within rounding
        sharp = r
        for j in range(r - 1):
            if abs(d[j] - d[j + 1]) <= 1e-12 * d[0]:
                sharp = j
                break
        np.testing.assert_array_equal(J[:sharp], C[piv[:sharp]])
        compared += 1
    assert compared >= 4


def test_hmatvec_equals_dense_assembly_of_eq_2_18():
    """At a tolerance where the bases are truncated, the H-matvec equals K~ x for K~
    assembled densely from Eq. 2.18's parts: D = the leaf diagonal blocks, and for every
    sibling pair (l, r) the block V_l^T K(J_l, J_r) V_r (and its transpose), where the
    nested basis is V_leaf = P_leaf and V_node = P_node blockdiag(V_left, V_right)."""
    n, leaf, max_rank = 600, 40, 24
    X, eps, s = _setup(n, 13, leaf)
    H = O.compress(X, eps, s, leaf, 1e-3, max_rank)
    L, perm = H.L, H.perm
    W = O.kernel_W(X, eps)
    Kp = (s[:, None] * W * s[None, :])[np.ix_(perm, perm)]
    Pn = H.P.reshape(-1, H.max_rank, H.cmax)
    V = {}
    for node in range((1 << (L + 1)) - 2, 0, -1):  # children before parents
        r = H.ranks[node]
        st, sz = O.node_range(n, node)
        if int(math.log2(node + 1)) == L:
            V[node] = Pn[node, :r, :sz]
        else:
            l, rr = 2 * node + 1, 2 * node + 2
            Vl, Vr = V[l], V[rr]
            blk = np.zeros((Vl.shape[0] + Vr.shape[0], Vl.shape[1] + Vr.shape[1]))
            blk[:Vl.shape[0], :Vl.shape[1]] = Vl
            blk[Vl.shape[0]:, Vl.shape[1]:] = Vr
            V[node] = Pn[node, :r, :Vl.shape[0] + Vr.shape[0]] @ blk
    Kt = np.zeros((n, n))
    for leaf_node in range((1 << L) - 1, (1 << (L + 1)) - 1):
        st, sz = O.node_range(n, leaf_node)
        Kt[st:st + sz, st:st + sz] = Kp[st:st + sz, st:st + sz]
    for p in range(0, (1 << L) - 1):
        l, rr = 2 * p + 1, 2 * p + 2
        sl, sr = O.node_range(n, l), O.node_range(n, rr)
        Jl = H.skel[l * H.max_rank:l * H.max_rank + H.ranks[l]]
        Jr = H.skel[rr * H.max_rank:rr * H.max_rank + H.ranks[rr]]
        F = V[l].T @ Kp[np.ix_(Jl, Jr)] @ V[rr]
        Kt[sl[0]:sl[0] + sl[1], sr[0]:sr[0] + sr[1]] = F
        Kt[sr[0]:sr[0] + sr[1], sl[0]:sl[0] + sl[1]] = F.T
    Korig = np.empty_like(Kt)
    Korig[np.ix_(perm, perm)] = Kt
    x = synth.random_rhs(n, 2, 17)
    yh = O.hmatvec(X, eps, s, H, x)
    y = Korig @ x
    np.testing.assert_allclose(yh, y, rtol=0, atol=1e-12 * np.abs(y).max())
    # and the truncation really happened: K~ differs from K
    assert np.abs(Korig - (s[:, None] * W * s[None, :])).max() > 1e-8


@pytest.mark.parametrize("conv_tol", [1e-4, 1e-7])
def test_lanczos_stop_rule_bounds_the_true_residuals(conv_tol):
    """With full reorthogonalisation the stop rule's bound beta_m |y_m| is the residual
    |S phi - theta phi| of each Ritz pair, so at the stop every wanted pair's true
    residual is within conv_tol theta_1 (up to rounding); a looser tolerance stops no later."""
    X = _scurve(600, 14)
    eps = O.median_sqdist(X)
    q, dg, s = O.degrees(X, eps, 1.0)
    W = O.kernel_W(X, eps)
    S = s[:, None] * W * s[None, :]
    k = 8
    ev, V, it, st = O.lanczos_S(X, eps, s, k, conv_tol=conv_tol)
    assert st == 0
    res = np.linalg.norm(S @ V - V * ev[None, :], axis=0)
    assert np.all(res <= conv_tol * ev[0] * (1 + 1e-6) + 1e-13), res
    _, _, it_tight, _ = O.lanczos_S(X, eps, s, k, conv_tol=conv_tol * 1e-3)
    assert it <= it_tight


def test_S_matvec_rows_matches_full_product_and_top_eigenpair():
    """or_S_matvec_rows (the row-sampled checker of the full-size tests) against the full
    product on chosen rows, and against S dg^1/2 = dg^1/2 (Algorithm 1: the Markov matrix
    P = Dg^-1 W^a has P 1 = 1, so its conjugate S fixes dg^1/2). Dropping s_i, s_j or the
    kernel's exponent scale breaks the invariant even where both routines would agree."""
    n = 700
    X = _scurve(n, 15)
    eps = O.median_sqdist(X)
    q, dg, s = O.degrees(X, eps, 1.0)
    rows = np.array([0, 1, 77, 350, 351, 698, 699, 77])
    x = synth.random_rhs(n, 1, 21)[:, 0]
    full = O.S_matvec(X, eps, s, x)
    np.testing.assert_allclose(O.S_matvec_rows(X, eps, s, x, rows), full[rows], rtol=1e-13, atol=0)
    r = np.sqrt(dg)
    np.testing.assert_allclose(O.S_matvec_rows(X, eps, s, r, rows), r[rows], rtol=1e-12, atol=0)
    # alpha = 0.5 gives another s; the invariant holds for every alpha
    _, dg5, s5 = O.degrees(X, eps, 0.5)
    r5 = np.sqrt(dg5)
    np.testing.assert_allclose(O.S_matvec_rows(X, eps, s5, r5, rows), r5[rows], rtol=1e-12, atol=0)


def _id_rows_recomputed(n, st, sz, rtarget, seed, node):
    """The ID's sampled rows, recomputed from the published SplitMix64 stream: draw t is
    u = floor(hi32(rng(key, t)) * off / 2^32) over the off = n - sz off-node positions,
    mapped past the node's own range [st, st + sz)."""
    off = n - sz
    key = O.stream_key(seed, 1, node)
    u = np.array(O.splitmix64_sequence(key, rtarget), dtype=np.uint64)
    u = ((u >> np.uint64(32)) * np.uint64(off)) >> np.uint64(32)
    u = u.astype(np.int64)
    return np.where(u < st, u, u + sz)


@pytest.mark.parametrize("seed", [0, 5])
def test_id_sampled_rows_branch_matches_recomputed_draws(seed):
    """The sampled-row branch of the ID (more off-node points than 2 max_rank + 10): the
    oracle's ranks, skeletons and interpolation matrices equal LAPACK's column-pivoted QR
    (scipy.linalg.qr, pivoting=True) of K(R, C) with R recomputed here from the seeded
    stream, so a wrong draw, a row inside the node or a wrong offset changes the result."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    n, leaf, max_rank, tol = 600, 40, 24, 1e-5
    X, eps, s = _setup(n, 16, leaf)
    perm, L = O.tree(X, eps, leaf)
    H = O.skeletonize(X, eps, s, perm, L, tol, max_rank, seed=seed)
    W = O.kernel_W(X, eps)
    Kp = (s[:, None] * W * s[None, :])[np.ix_(perm, perm)]
    Pn = H.P.reshape(-1, H.max_rank, H.cmax)
    rtarget = 2 * max_rank + 10
    compared = 0
    for node in range(1, (1 << (L + 1)) - 1):
        st, sz = O.node_range(n, node)
        assert n - sz > rtarget  # every node takes the sampled branch here
        R = _id_rows_recomputed(n, st, sz, rtarget, seed, node)
        assert R.min() >= 0 and R.max() < n and not np.any((R >= st) & (R < st + sz))
        if int(math.log2(node + 1)) == L:
            C = np.arange(st, st + sz)
        else:
            l, rr = 2 * node + 1, 2 * node + 2
            C = np.concatenate([H.skel[l * max_rank:l * max_rank + H.ranks[l]],
                                H.skel[rr * max_rank:rr * max_rank + H.ranks[rr]]])
        A = Kp[np.ix_(R, C)]
        _, Rq, piv = scipy_linalg.qr(A, pivoting=True, mode="economic")
        d = np.abs(np.diag(Rq))
        kmax = min(max_rank, len(C), rtarget)
        thr = tol * d[0]
        r_lapack = next((j for j in range(kmax) if d[j] <= thr), kmax)
        if np.any(np.abs(d[:kmax + 1] - thr) <= 1e-9 * thr):
            continue
        if any(abs(d[j] - d[j + 1]) <= 1e-12 * d[0] for j in range(r_lapack)):
            continue  # pivot ties within rounding: the order is not sharp
        r = H.ranks[node]
        assert r == r_lapack, (node, r, r_lapack)
        J = H.skel[node * max_rank:node * max_rank + r]
        np.testing.assert_array_equal(J, C[piv[:r]])
        # P(:, J) = I and P(:, rest) = R11^-1 R12 (invariant to the sign convention of the QR)
        want = np.zeros((r, len(C)))
        want[:, piv[:r]] = np.eye(r)
        want[:, piv[r:]] = scipy_linalg.solve_triangular(Rq[:r, :r], Rq[:r, r:len(C)])
        np.testing.assert_allclose(Pn[node, :r, :len(C)], want, rtol=0, atol=1e-7 * max(1.0, np.abs(want).max()))
        compared += 1
    assert compared >= 10


@pytest.mark.parametrize("n,leaf,rank,tol", [(400, 32, 16, 1e-3), (512, 64, 32, 1e-5)])
def test_hmatvec_error_2norm_matches_svd_of_the_dense_difference(n, leaf, rank, tol):
    """The power-iteration estimate of ||S~ - S||_2 (Eq. 1.1 in the operator 2-norm)
    against the largest singular value of the assembled difference: S~ column by column from
    the H-matvec of the identity, S from the dense kernel (Eq. W) and the scaling s; the
    estimate is a lower bound that reaches it within 1e-3."""
    X = _scurve(n, 3)
    eps = O.median_sqdist(X)
    _, _, s = O.degrees(X, eps, 1.0)
    H = O.compress(X, eps, s, leaf, tol, rank)
    St = O.hmatvec(X, eps, s, H, np.eye(n))
    S = s[:, None] * O.kernel_W(X, eps) * s[None, :]
    exact = np.linalg.norm(St - S, 2)
    est = O.hmatvec_error_2norm(X, eps, s, H, iters=60)
    assert est <= exact * (1 + 1e-12) + 1e-15
    assert est >= exact * (1 - 1e-3)


def test_hmatvec_error_2norm_vanishes_at_zero_tolerance_full_rank():
    X = _scurve(256, 3)
    eps = O.median_sqdist(X)
    _, _, s = O.degrees(X, eps, 1.0)
    H = O.compress(X, eps, s, 32, 0.0, 256)
    assert O.hmatvec_error_2norm(X, eps, s, H, iters=10) < 1e-12
