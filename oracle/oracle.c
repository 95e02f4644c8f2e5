/*
 * oracle.c -- plain, slow, FP64 CPU reference ("oracle") for the diffusion-map
 * hierarchical matvec and Lanczos eigensolver of Gaddameedi, Reiz, Neckel and
 * Bungartz, "Efficient and Scalable Kernel Matrix Approximations using
 * Hierarchical Decomposition" (arXiv 2311.06115).
 *
 * TEST INFRASTRUCTURE ONLY: it is called by the tests, by the smoke check and
 * by the CPU-baseline leg of the benchmark, never by the product path, and it
 * shares no code with the CUDA library.
 *
 * What each part follows:
 *   - Gaussian kernel W_ij = exp(-|x_i - x_j|^2 / eps), eps = sigma^2   (Eq. W, Section 2.1)
 *   - q = W 1, W^a_ij = W_ij / (q_i^a q_j^a), dg = W^a 1, P = Dg^-1 W^a  (Algorithm 1: similarity
 *     matrix and normalisations; the Markov denominator is read as the Coifman-Lafon row
 *     sum of W^a, which makes P row-stochastic)
 *   - S = Dg^-1/2 W^a Dg^-1/2 = diag(s) W diag(s), s = q^-a dg^-1/2: the symmetric
 *     conjugate of P with the same eigenvalues (Section 2.1, SPD requirement of Section 1.2)
 *   - H-matrix form K~ = D + UV (Eq. 2.18) with a balanced binary partition tree and
 *     nested interpolative-decomposition bases (the GOFMM form the paper uses; the paper
 *     gives only its parameters, Section 4.2 footnote) -- the tree rule and the ID stopping
 *     rule are readings of this implementation (the paper does not describe them)
 *   - relative-error target ||K~ - K|| / ||K|| <= eps_tol                 (Eq. 1.1)
 *   - Krylov basis and projection by Gram-Schmidt                        (Algorithm 2,
 *     Eq. arnoldi; symmetric case: Lanczos, Section 2.3.1), done twice per step
 *   - eigenpairs of the projected tridiagonal by cyclic Jacobi rotations (dense, FP64)
 *
 * Build with -ffp-contract=off so no fused multiply-add changes rounding between
 * machines: the tree and the bandwidth median are integer decisions that the
 * CUDA path reproduces in the same FP64 arithmetic.
 *
 * Parity pins live in tests/test_oracle_pins.py (closed forms, invariants, brute force).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_GOLDEN 0x9E3779B97F4A7C15ULL
#define OR_TAG_ROWS 1u
#define OR_TAG_V0 2u
#define OR_TAG_PAIRS 3u

/* ------------------------------------------------------------------------- */
/* SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number      */
/* generators", OOPSLA 2014): state += golden gamma, then a 64-bit finaliser. */
/* ------------------------------------------------------------------------- */
static uint64_t or_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t or_splitmix64_next(uint64_t *state) {
    *state += OR_GOLDEN;
    return or_mix64(*state);
}

/* Independent stream per (seed, purpose tag, id); counter ctr gives the
 * (ctr+1)-th SplitMix64 output of a generator whose state starts at key. */
uint64_t or_stream_key(uint64_t seed, uint32_t tag, uint64_t id) {
    return or_mix64(seed * OR_GOLDEN + ((uint64_t)tag << 48) + id);
}

uint64_t or_rng(uint64_t key, uint64_t ctr) { return or_mix64(key + (ctr + 1) * OR_GOLDEN); }

static uint64_t or_below(uint64_t u, uint64_t n) { return ((u >> 32) * n) >> 32; }
static double or_unit(uint64_t u) { return (double)(u >> 11) * (1.0 / 9007199254740992.0); }

/* ------------------------------------------------------------------------- */
/* Kernel entries                                                            */
/* ------------------------------------------------------------------------- */
double or_sqdist(const float *X, int32_t d, int64_t i, int64_t j) {
    const float *a = X + i * d, *b = X + j * d;
    double r2 = 0.0;
    for (int32_t k = 0; k < d; ++k) {
        double t = (double)a[k] - (double)b[k];
        r2 = r2 + t * t;
    }
    return r2;
}

/* Eq. W: W_ij = exp(-||x_i - x_j||^2 / sigma^2), with eps = sigma^2. */
static double or_w(const float *X, int32_t d, double eps, int64_t i, int64_t j) {
    return exp(-or_sqdist(X, d, i, j) / eps);
}

static int or_cmp_double(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Bandwidth eps = median squared pairwise distance (the workload's kernel scale;
 * the paper leaves sigma free). All i<j pairs when there are at most 2^20 of them,
 * else 2^20 seeded pairs i != j; an even count averages the two middle values. */
double or_median_sqdist(const float *X, int64_t N, int32_t d, uint64_t seed) {
    const int64_t cap = (int64_t)1 << 20;
    int64_t npairs = N * (N - 1) / 2;
    int64_t m = npairs <= cap ? npairs : cap;
    double *v = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    if (npairs <= cap) {
        int64_t c = 0;
        for (int64_t i = 0; i < N; ++i)
            for (int64_t j = i + 1; j < N; ++j) v[c++] = or_sqdist(X, d, i, j);
    } else {
        uint64_t key = or_stream_key(seed, OR_TAG_PAIRS, 0);
        for (int64_t c = 0; c < m; ++c) {
            int64_t i = (int64_t)or_below(or_rng(key, 2 * (uint64_t)c), (uint64_t)N);
            int64_t j = (int64_t)or_below(or_rng(key, 2 * (uint64_t)c + 1), (uint64_t)(N - 1));
            if (j >= i) j += 1;
            v[c] = or_sqdist(X, d, i, j);
        }
    }
    qsort(v, (size_t)m, sizeof(double), or_cmp_double);
    double med = (m % 2 == 0) ? 0.5 * (v[m / 2 - 1] + v[m / 2]) : v[m / 2];
    free(v);
    return med;
}

void or_kernel_W(const float *X, int64_t N, int32_t d, double eps, double *W) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < N; ++j) W[i * N + j] = or_w(X, d, eps, i, j);
}

/* Algorithm 1, similarity matrix and normalisations: q_i = sum_j W_ij; dg_i = q_i^-a sum_j W_ij q_j^-a
 * (the row sum of W^a); s_i = q_i^-a dg_i^-1/2 so that S = diag(s) W diag(s). */
void or_degrees(const float *X, int64_t N, int32_t d, double eps, double alpha,
                double *q, double *dg, double *s) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double acc = 0.0;
        for (int64_t j = 0; j < N; ++j) acc += or_w(X, d, eps, i, j);
        q[i] = acc;
    }
    double *qa = (double *)malloc(sizeof(double) * (size_t)N);
    for (int64_t i = 0; i < N; ++i) qa[i] = pow(q[i], -alpha);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double acc = 0.0;
        for (int64_t j = 0; j < N; ++j) acc += or_w(X, d, eps, i, j) * qa[j];
        dg[i] = qa[i] * acc;
    }
    for (int64_t i = 0; i < N; ++i) s[i] = qa[i] / sqrt(dg[i]);
    free(qa);
}

void or_q_rows(const float *X, int64_t N, int32_t d, double eps,
               const int64_t *rows, int64_t nrows, double *q_rows) {
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < nrows; ++r) {
        double acc = 0.0;
        for (int64_t j = 0; j < N; ++j) acc += or_w(X, d, eps, rows[r], j);
        q_rows[r] = acc;
    }
}

/* Exact y = S x, entries generated on the fly; x, y are N x nrhs column-major. */
void or_S_matvec(const float *X, int64_t N, int32_t d, double eps, const double *s,
                 const double *x, int32_t nrhs, double *y) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        for (int32_t c = 0; c < nrhs; ++c) y[(int64_t)c * N + i] = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            double kij = s[i] * or_w(X, d, eps, i, j) * s[j];
            for (int32_t c = 0; c < nrhs; ++c) y[(int64_t)c * N + i] += kij * x[(int64_t)c * N + j];
        }
    }
}

void or_S_matvec_rows(const float *X, int64_t N, int32_t d, double eps, const double *s,
                      const double *x, const int64_t *rows, int64_t nrows, double *y_rows) {
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows[r];
        double acc = 0.0;
        for (int64_t j = 0; j < N; ++j) acc += s[i] * or_w(X, d, eps, i, j) * s[j] * x[j];
        y_rows[r] = acc;
    }
}

/* ------------------------------------------------------------------------- */
/* Partition tree. Perfect binary tree of depth L, L the least depth with    */
/* ceil(N / 2^L) <= leaf_size; node (level l, k) has heap index 2^l - 1 + k; */
/* a node of n points splits into ceil(n/2) (left) and floor(n/2) (right).   */
/* ------------------------------------------------------------------------- */
int32_t or_tree_depth(int64_t N, int64_t leaf_size) {
    int32_t L = 0;
    while (((N + ((int64_t)1 << L) - 1) >> L) > leaf_size) ++L;
    return L;
}

void or_node_range(int64_t N, int32_t node, int64_t *start, int64_t *size) {
    /* walk from the root following the bits of node+1 below its leading one */
    int64_t st = 0, sz = N;
    uint32_t h = (uint32_t)node + 1u;
    int lvl = 0;
    while ((h >> (lvl + 1)) != 0) ++lvl;
    for (int b = lvl - 1; b >= 0; --b) {
        int64_t left = (sz + 1) / 2;
        if ((h >> b) & 1u) { st += left; sz = sz - left; }
        else { sz = left; }
    }
    *start = st;
    *size = sz;
}

typedef struct { double key; int32_t idx; } or_keyed;

static int or_cmp_keyed(const void *a, const void *b) {
    const or_keyed *x = (const or_keyed *)a, *y = (const or_keyed *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* Farthest point from `from` in the Gram distance of W, d^2(i,j) = W_ii + W_jj - 2 W_ij
 * = 2 - 2 exp(-r_ij^2 / eps). That distance is strictly increasing in r_ij^2 (Eq. W),
 * so the farthest point is the one with the largest squared distance; comparing r^2
 * keeps the integer decision free of exp rounding. Ties go to the lowest original index. */
static int32_t or_farthest(const float *X, int32_t d, const int32_t *idx, int64_t n, int32_t from) {
    int32_t best = idx[0];
    double br = or_sqdist(X, d, from, idx[0]);
    for (int64_t t = 1; t < n; ++t) {
        double r = or_sqdist(X, d, from, idx[t]);
        if (r > br || (r == br && idx[t] < best)) { br = r; best = idx[t]; }
    }
    return best;
}

/* Split one node whose points idx[0..n) are in increasing original index:
 * anchor i0 = idx[0]; p = farthest from i0; q = farthest from p; key_i = W_iq - W_ip
 * (= half the projection d^2(i,p) - d^2(i,q)); the ceil(n/2) smallest (key, index)
 * go left; each child keeps increasing original-index order. */
static void or_split(const float *X, int32_t d, double eps, int32_t *idx, int64_t n) {
    int32_t i0 = idx[0];
    int32_t p = or_farthest(X, d, idx, n, i0);
    int32_t q = or_farthest(X, d, idx, n, p);
    or_keyed *kv = (or_keyed *)malloc(sizeof(or_keyed) * (size_t)n);
    for (int64_t t = 0; t < n; ++t) {
        kv[t].key = or_w(X, d, eps, idx[t], q) - or_w(X, d, eps, idx[t], p);
        kv[t].idx = idx[t];
    }
    qsort(kv, (size_t)n, sizeof(or_keyed), or_cmp_keyed);
    int64_t nl = (n + 1) / 2;
    /* mark the left set, then rewrite idx as left-then-right, each in index order */
    char *isleft = (char *)calloc((size_t)n, 1);
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    or_keyed *lsorted = (or_keyed *)malloc(sizeof(or_keyed) * (size_t)nl);
    for (int64_t t = 0; t < nl; ++t) { lsorted[t].key = 0.0; lsorted[t].idx = kv[t].idx; }
    qsort(lsorted, (size_t)nl, sizeof(or_keyed), or_cmp_keyed); /* by index */
    /* idx is sorted by index: two-pointer walk marks the left members */
    int64_t a = 0;
    for (int64_t t = 0; t < n && a < nl; ++t)
        if (idx[t] == lsorted[a].idx) { isleft[t] = 1; ++a; }
    int64_t wl = 0, wr = nl;
    for (int64_t t = 0; t < n; ++t) {
        if (isleft[t]) tmp[wl++] = idx[t];
        else tmp[wr++] = idx[t];
    }
    memcpy(idx, tmp, sizeof(int32_t) * (size_t)n);
    free(kv); free(isleft); free(tmp); free(lsorted);
}

int32_t or_tree(const float *X, int64_t N, int32_t d, double eps, int64_t leaf_size, int32_t *perm) {
    int32_t L = or_tree_depth(N, leaf_size);
    for (int64_t i = 0; i < N; ++i) perm[i] = (int32_t)i;
    for (int32_t lvl = 0; lvl < L; ++lvl) {
        int32_t first = (1 << lvl) - 1, count = 1 << lvl;
#pragma omp parallel for schedule(dynamic)
        for (int32_t k = 0; k < count; ++k) {
            int64_t st, sz;
            or_node_range(N, first + k, &st, &sz);
            if (sz >= 2) or_split(X, d, eps, perm + st, sz);
        }
    }
    return L;
}

/* ------------------------------------------------------------------------- */
/* Skeletonization: per non-root node, bottom-up, an interpolative           */
/* decomposition of the sampled off-node block A = K(R, C) by column-pivoted */
/* Householder QR (Businger-Golub): A(:,J) P ~= A with P(:,J) = I and         */
/* P(:,rest) = R11^-1 R12; rank = number of pivots whose residual column norm */
/* exceeds tol * (first pivot norm), capped by max_rank and min(r, c).        */
/* Candidates C: a leaf's own points; an internal node's children skeletons. */
/* Rows R: every off-node point if there are at most 2 max_rank + 10 of      */
/* them, else that many seeded uniform draws (with replacement).             */
/* ------------------------------------------------------------------------- */
static double or_kentry(const float *X, int32_t d, double eps, const double *s, const int32_t *perm,
                        int64_t pi, int64_t pj) {
    int64_t i = perm[pi], j = perm[pj];
    return s[i] * or_w(X, d, eps, i, j) * s[j];
}

int32_t or_skeletonize(const float *X, int64_t N, int32_t d, double eps, const double *s,
                       const int32_t *perm, int32_t L, double tol, int32_t max_rank,
                       int32_t cmax, uint64_t seed, int32_t *ranks, int32_t *skel, double *P) {
    int32_t nnodes = (1 << (L + 1)) - 1;
    int32_t rtarget = 2 * max_rank + 10;
    ranks[0] = 0;
    for (int32_t lvl = L; lvl >= 1; --lvl) {
        int32_t first = (1 << lvl) - 1, count = 1 << lvl;
#pragma omp parallel for schedule(dynamic)
        for (int32_t k = 0; k < count; ++k) {
            int32_t node = first + k;
            int64_t st, sz;
            or_node_range(N, node, &st, &sz);
            /* candidate positions */
            int32_t c;
            int64_t *C;
            if (lvl == L) {
                c = (int32_t)sz;
                C = (int64_t *)malloc(sizeof(int64_t) * (size_t)c);
                for (int32_t j = 0; j < c; ++j) C[j] = st + j;
            } else {
                int32_t l = 2 * node + 1, r = 2 * node + 2;
                c = ranks[l] + ranks[r];
                C = (int64_t *)malloc(sizeof(int64_t) * (size_t)(c > 0 ? c : 1));
                for (int32_t j = 0; j < ranks[l]; ++j) C[j] = skel[(int64_t)l * max_rank + j];
                for (int32_t j = 0; j < ranks[r]; ++j) C[ranks[l] + j] = skel[(int64_t)r * max_rank + j];
            }
            /* sample rows */
            int64_t off = N - sz;
            int64_t rr = off <= rtarget ? off : rtarget;
            int64_t *R = (int64_t *)malloc(sizeof(int64_t) * (size_t)(rr > 0 ? rr : 1));
            if (off <= rtarget) {
                int64_t t = 0;
                for (int64_t p = 0; p < N; ++p)
                    if (p < st || p >= st + sz) R[t++] = p;
            } else {
                uint64_t key = or_stream_key(seed, OR_TAG_ROWS, (uint64_t)node);
                for (int64_t t = 0; t < rr; ++t) {
                    int64_t u = (int64_t)or_below(or_rng(key, (uint64_t)t), (uint64_t)off);
                    R[t] = u < st ? u : u + sz;
                }
            }
            /* A (rr x c), column-major */
            double *A = (double *)malloc(sizeof(double) * (size_t)(rr * (c > 0 ? c : 1)));
            for (int32_t j = 0; j < c; ++j)
                for (int64_t i = 0; i < rr; ++i) A[(int64_t)j * rr + i] = or_kentry(X, d, eps, s, perm, R[i], C[j]);
            int32_t *colid = (int32_t *)malloc(sizeof(int32_t) * (size_t)(c > 0 ? c : 1));
            for (int32_t j = 0; j < c; ++j) colid[j] = j;
            int32_t kmax = max_rank;
            if (kmax > c) kmax = c;
            if (kmax > rr) kmax = (int32_t)rr;
            double first_norm = 0.0;
            int32_t rank = 0;
            double *vh = (double *)malloc(sizeof(double) * (size_t)(rr > 0 ? rr : 1));
            for (int32_t kk = 0; kk < kmax; ++kk) {
                /* residual norms of the trailing columns, recomputed from rows kk.. */
                int32_t piv = -1;
                double pn = -1.0;
                for (int32_t j = kk; j < c; ++j) {
                    double acc = 0.0;
                    for (int64_t i = kk; i < rr; ++i) acc += A[(int64_t)j * rr + i] * A[(int64_t)j * rr + i];
                    double nrm = sqrt(acc);
                    if (nrm > pn || (nrm == pn && colid[j] < colid[piv])) { pn = nrm; piv = j; }
                }
                if (kk == 0) first_norm = pn;
                if (pn <= tol * first_norm || pn == 0.0) break;
                /* swap column piv into position kk */
                if (piv != kk) {
                    for (int64_t i = 0; i < rr; ++i) {
                        double t = A[(int64_t)kk * rr + i];
                        A[(int64_t)kk * rr + i] = A[(int64_t)piv * rr + i];
                        A[(int64_t)piv * rr + i] = t;
                    }
                    int32_t t = colid[kk]; colid[kk] = colid[piv]; colid[piv] = t;
                }
                /* Householder reflector for A(kk:, kk) */
                double *a = A + (int64_t)kk * rr;
                double alpha = (a[kk] >= 0.0 ? -pn : pn);
                for (int64_t i = kk; i < rr; ++i) vh[i] = a[i];
                vh[kk] -= alpha;
                double vnorm2 = 0.0;
                for (int64_t i = kk; i < rr; ++i) vnorm2 += vh[i] * vh[i];
                if (vnorm2 > 0.0) {
                    for (int32_t j = kk; j < c; ++j) {
                        double *aj = A + (int64_t)j * rr;
                        double dot = 0.0;
                        for (int64_t i = kk; i < rr; ++i) dot += vh[i] * aj[i];
                        double f = 2.0 * dot / vnorm2;
                        for (int64_t i = kk; i < rr; ++i) aj[i] -= f * vh[i];
                    }
                }
                rank = kk + 1;
            }
            /* P (rank x c) stored row-major with leading dimension cmax */
            double *Pn = P + (int64_t)node * max_rank * cmax;
            for (int64_t t = 0; t < (int64_t)max_rank * cmax; ++t) Pn[t] = 0.0;
            for (int32_t t = 0; t < rank; ++t) Pn[(int64_t)t * cmax + colid[t]] = 1.0;
            for (int32_t j = rank; j < c; ++j) {
                /* solve R11 z = R12(:, j) by back substitution; R is in A's upper triangle */
                double *z = vh;
                for (int32_t t = rank - 1; t >= 0; --t) {
                    double acc = A[(int64_t)j * rr + t];
                    for (int32_t u = t + 1; u < rank; ++u) acc -= A[(int64_t)u * rr + t] * z[u];
                    z[t] = acc / A[(int64_t)t * rr + t];
                }
                for (int32_t t = 0; t < rank; ++t) Pn[(int64_t)t * cmax + colid[j]] = z[t];
            }
            ranks[node] = rank;
            for (int32_t t = 0; t < max_rank; ++t)
                skel[(int64_t)node * max_rank + t] = t < rank ? (int32_t)C[colid[t]] : -1;
            free(C); free(R); free(A); free(colid); free(vh);
        }
    }
    (void)nnodes;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* HSS matvec y = K~ x (Eq. 2.18 with D = diagonal leaf blocks and UV the    */
/* nested skeleton products of sibling pairs), on the fly, original order.   */
/*   near:  y~(I_a) = K(I_a, I_a) x~(I_a)                         (leaves)    */
/*   N2S:   w_a = P_a x~(I_a) (leaf), w_a = P_a [w_l; w_r] (internal)         */
/*   S2S:   u_l += K(S_l, S_r) w_r,  u_r += K(S_r, S_l) w_l   (sibling pairs) */
/*   S2N:   [u_l; u_r] += P_a^T u_a (internal), y~(I_a) += P_a^T u_a (leaf)   */
/* ------------------------------------------------------------------------- */
void or_hmatvec(const float *X, int64_t N, int32_t d, double eps, const double *s,
                const int32_t *perm, int32_t L, int32_t max_rank, int32_t cmax,
                const int32_t *ranks, const int32_t *skel, const double *P,
                const double *x, int32_t nrhs, double *y) {
    int32_t nnodes = (1 << (L + 1)) - 1;
    double *xt = (double *)malloc(sizeof(double) * (size_t)N);
    double *yt = (double *)malloc(sizeof(double) * (size_t)N);
    double *w = (double *)malloc(sizeof(double) * (size_t)nnodes * max_rank);
    double *u = (double *)malloc(sizeof(double) * (size_t)nnodes * max_rank);
    for (int32_t c = 0; c < nrhs; ++c) {
        for (int64_t p = 0; p < N; ++p) xt[p] = x[(int64_t)c * N + perm[p]];
        for (int64_t t = 0; t < (int64_t)nnodes * max_rank; ++t) { w[t] = 0.0; u[t] = 0.0; }
        int32_t firstleaf = (1 << L) - 1, nleaves = 1 << L;
        /* near field */
#pragma omp parallel for schedule(dynamic)
        for (int32_t k = 0; k < nleaves; ++k) {
            int64_t st, sz;
            or_node_range(N, firstleaf + k, &st, &sz);
            for (int64_t i = st; i < st + sz; ++i) {
                double acc = 0.0;
                for (int64_t j = st; j < st + sz; ++j) acc += or_kentry(X, d, eps, s, perm, i, j) * xt[j];
                yt[i] = acc;
            }
        }
        /* N2S, bottom-up */
        for (int32_t lvl = L; lvl >= 1; --lvl) {
            int32_t first = (1 << lvl) - 1, count = 1 << lvl;
            for (int32_t k = 0; k < count; ++k) {
                int32_t node = first + k;
                const double *Pn = P + (int64_t)node * max_rank * cmax;
                double *wn = w + (int64_t)node * max_rank;
                if (lvl == L) {
                    int64_t st, sz;
                    or_node_range(N, node, &st, &sz);
                    for (int32_t t = 0; t < ranks[node]; ++t) {
                        double acc = 0.0;
                        for (int64_t j = 0; j < sz; ++j) acc += Pn[(int64_t)t * cmax + j] * xt[st + j];
                        wn[t] = acc;
                    }
                } else {
                    int32_t l = 2 * node + 1, r = 2 * node + 2;
                    for (int32_t t = 0; t < ranks[node]; ++t) {
                        double acc = 0.0;
                        for (int32_t j = 0; j < ranks[l]; ++j) acc += Pn[(int64_t)t * cmax + j] * w[(int64_t)l * max_rank + j];
                        for (int32_t j = 0; j < ranks[r]; ++j)
                            acc += Pn[(int64_t)t * cmax + ranks[l] + j] * w[(int64_t)r * max_rank + j];
                        wn[t] = acc;
                    }
                }
            }
        }
        /* S2S across every sibling pair (children of each internal node, root included) */
        for (int32_t node = 0; node < (1 << L) - 1; ++node) {
            int32_t l = 2 * node + 1, r = 2 * node + 2;
            for (int32_t a = 0; a < ranks[l]; ++a) {
                double acc = 0.0;
                for (int32_t b = 0; b < ranks[r]; ++b)
                    acc += or_kentry(X, d, eps, s, perm, skel[(int64_t)l * max_rank + a], skel[(int64_t)r * max_rank + b]) *
                           w[(int64_t)r * max_rank + b];
                u[(int64_t)l * max_rank + a] += acc;
            }
            for (int32_t b = 0; b < ranks[r]; ++b) {
                double acc = 0.0;
                for (int32_t a = 0; a < ranks[l]; ++a)
                    acc += or_kentry(X, d, eps, s, perm, skel[(int64_t)r * max_rank + b], skel[(int64_t)l * max_rank + a]) *
                           w[(int64_t)l * max_rank + a];
                u[(int64_t)r * max_rank + b] += acc;
            }
        }
        /* S2N, top-down */
        for (int32_t lvl = 1; lvl <= L; ++lvl) {
            int32_t first = (1 << lvl) - 1, count = 1 << lvl;
            for (int32_t k = 0; k < count; ++k) {
                int32_t node = first + k;
                const double *Pn = P + (int64_t)node * max_rank * cmax;
                const double *un = u + (int64_t)node * max_rank;
                if (lvl == L) {
                    int64_t st, sz;
                    or_node_range(N, node, &st, &sz);
                    for (int64_t j = 0; j < sz; ++j) {
                        double acc = 0.0;
                        for (int32_t t = 0; t < ranks[node]; ++t) acc += Pn[(int64_t)t * cmax + j] * un[t];
                        yt[st + j] += acc;
                    }
                } else {
                    int32_t l = 2 * node + 1, r = 2 * node + 2;
                    for (int32_t j = 0; j < ranks[l]; ++j) {
                        double acc = 0.0;
                        for (int32_t t = 0; t < ranks[node]; ++t) acc += Pn[(int64_t)t * cmax + j] * un[t];
                        u[(int64_t)l * max_rank + j] += acc;
                    }
                    for (int32_t j = 0; j < ranks[r]; ++j) {
                        double acc = 0.0;
                        for (int32_t t = 0; t < ranks[node]; ++t) acc += Pn[(int64_t)t * cmax + ranks[l] + j] * un[t];
                        u[(int64_t)r * max_rank + j] += acc;
                    }
                }
            }
        }
        for (int64_t p = 0; p < N; ++p) y[(int64_t)c * N + perm[p]] = yt[p];
    }
    free(xt); free(yt); free(w); free(u);
}

/* ------------------------------------------------------------------------- */
/* Cyclic Jacobi eigensolver for a dense symmetric matrix (row-major n x n). */
/* Returns eigenvalues in descending order; eigenvectors as columns of the   */
/* row-major n x n matrix evecs. Returns the number of sweeps used.          */
/* ------------------------------------------------------------------------- */
int32_t or_jacobi(const double *A0, int32_t n, double *evals, double *evecs) {
    double *A = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *V = (double *)malloc(sizeof(double) * (size_t)n * n);
    memcpy(A, A0, sizeof(double) * (size_t)n * n);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < n; ++j) V[(int64_t)i * n + j] = (i == j) ? 1.0 : 0.0;
    double fro = 0.0;
    for (int64_t t = 0; t < (int64_t)n * n; ++t) fro += A[t] * A[t];
    fro = sqrt(fro);
    int32_t sweep = 0;
    for (sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int32_t i = 0; i < n; ++i)
            for (int32_t j = i + 1; j < n; ++j) off += A[(int64_t)i * n + j] * A[(int64_t)i * n + j];
        if (sqrt(off) <= 1e-17 * fro || off == 0.0) break;
        for (int32_t p = 0; p < n; ++p) {
            for (int32_t q = p + 1; q < n; ++q) {
                double apq = A[(int64_t)p * n + q];
                if (apq == 0.0) continue;
                double app = A[(int64_t)p * n + p], aqq = A[(int64_t)q * n + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
                /* A <- J^T A J with J the rotation in the (p, q) plane */
                for (int32_t k = 0; k < n; ++k) {
                    double akp = A[(int64_t)k * n + p], akq = A[(int64_t)k * n + q];
                    A[(int64_t)k * n + p] = cs * akp - sn * akq;
                    A[(int64_t)k * n + q] = sn * akp + cs * akq;
                }
                for (int32_t k = 0; k < n; ++k) {
                    double apk = A[(int64_t)p * n + k], aqk = A[(int64_t)q * n + k];
                    A[(int64_t)p * n + k] = cs * apk - sn * aqk;
                    A[(int64_t)q * n + k] = sn * apk + cs * aqk;
                }
                A[(int64_t)p * n + q] = 0.0;
                A[(int64_t)q * n + p] = 0.0;
                for (int32_t k = 0; k < n; ++k) {
                    double vkp = V[(int64_t)k * n + p], vkq = V[(int64_t)k * n + q];
                    V[(int64_t)k * n + p] = cs * vkp - sn * vkq;
                    V[(int64_t)k * n + q] = sn * vkp + cs * vkq;
                }
            }
        }
    }
    /* sort descending (selection sort keeps it obvious) */
    int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int32_t i = 0; i < n; ++i) ord[i] = i;
    for (int32_t i = 0; i < n; ++i) {
        int32_t b = i;
        for (int32_t j = i + 1; j < n; ++j)
            if (A[(int64_t)ord[j] * n + ord[j]] > A[(int64_t)ord[b] * n + ord[b]]) b = j;
        int32_t t = ord[i]; ord[i] = ord[b]; ord[b] = t;
    }
    for (int32_t i = 0; i < n; ++i) {
        evals[i] = A[(int64_t)ord[i] * n + ord[i]];
        for (int32_t k = 0; k < n; ++k) evecs[(int64_t)k * n + i] = V[(int64_t)k * n + ord[i]];
    }
    free(A); free(V); free(ord);
    return sweep;
}

/* ------------------------------------------------------------------------- */
/* Lanczos with full reorthogonalization (Algorithm 2 in its symmetric form):  */
/*   x_1 = v0/|v0|; each step z = A x_j, h = X^T z, r = z - X h done twice      */
/*   (Gram-Schmidt "twice is enough"), alpha_j = accumulated h_j,             */
/*   beta_j = |r|, x_{j+1} = r / beta_j. Every few steps the tridiagonal T_j  */
/*   is diagonalised; Ritz pair i is converged when beta_j |y_{j,i}| <=       */
/*   conv_tol * theta_1. Returns 0 if the top k converged, 1 otherwise.       */
/* ------------------------------------------------------------------------- */
typedef void (*or_op_fn)(void *ctx, const double *x, double *y);

static void or_sign_normalise(double *v, int64_t n) {
    int64_t b = 0;
    for (int64_t i = 1; i < n; ++i)
        if (fabs(v[i]) > fabs(v[b])) b = i;
    if (v[b] < 0.0)
        for (int64_t i = 0; i < n; ++i) v[i] = -v[i];
}

static int32_t or_lanczos(or_op_fn op, void *ctx, int64_t n, int32_t k, int32_t m_max, double conv_tol,
                          const double *v0, double *evals, double *evecs, int32_t *iters) {
    if (m_max > n) m_max = (int32_t)n;
    double *V = (double *)malloc(sizeof(double) * (size_t)n * (m_max + 1));
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *h = (double *)malloc(sizeof(double) * (size_t)(m_max + 1));
    double *al = (double *)calloc((size_t)m_max + 1, sizeof(double));
    double *be = (double *)calloc((size_t)m_max + 1, sizeof(double));
    double *T = (double *)malloc(sizeof(double) * (size_t)m_max * m_max);
    double *th = (double *)malloc(sizeof(double) * (size_t)m_max);
    double *Y = (double *)malloc(sizeof(double) * (size_t)m_max * m_max);
    double nrm = 0.0;
    for (int64_t i = 0; i < n; ++i) nrm += v0[i] * v0[i];
    nrm = sqrt(nrm);
    for (int64_t i = 0; i < n; ++i) V[i] = v0[i] / nrm;
    int32_t status = 1, m = 0;
    for (int32_t j = 0; j < m_max; ++j) {
        op(ctx, V + (int64_t)j * n, z);
        al[j] = 0.0;
        for (int pass = 0; pass < 2; ++pass) {
            for (int32_t c = 0; c <= j; ++c) {
                double acc = 0.0;
                for (int64_t i = 0; i < n; ++i) acc += V[(int64_t)c * n + i] * z[i];
                h[c] = acc;
            }
            for (int32_t c = 0; c <= j; ++c)
                for (int64_t i = 0; i < n; ++i) z[i] -= V[(int64_t)c * n + i] * h[c];
            al[j] += h[j];
        }
        double b = 0.0;
        for (int64_t i = 0; i < n; ++i) b += z[i] * z[i];
        be[j] = sqrt(b);
        m = j + 1;
        int last = (m == m_max) || (be[j] <= 1e-14 * fabs(al[0]));
        if (m >= k && (last || m % 5 == 0)) {
            for (int32_t a = 0; a < m; ++a)
                for (int32_t c = 0; c < m; ++c)
                    T[(int64_t)a * m + c] = (a == c) ? al[a] : (abs(a - c) == 1 ? be[a < c ? a : c] : 0.0);
            or_jacobi(T, m, th, Y);
            int conv = 1;
            for (int32_t i = 0; i < k; ++i)
                if (be[j] * fabs(Y[(int64_t)(m - 1) * m + i]) > conv_tol * fabs(th[0])) conv = 0;
            if (conv || last) {
                status = conv ? 0 : 1;
                for (int32_t i = 0; i < k; ++i) {
                    evals[i] = th[i];
                    double *e = evecs + (int64_t)i * n;
                    for (int64_t r = 0; r < n; ++r) e[r] = 0.0;
                    for (int32_t c = 0; c < m; ++c) {
                        double yc = Y[(int64_t)c * m + i];
                        for (int64_t r = 0; r < n; ++r) e[r] += V[(int64_t)c * n + r] * yc;
                    }
                    double en = 0.0;
                    for (int64_t r = 0; r < n; ++r) en += e[r] * e[r];
                    en = sqrt(en);
                    for (int64_t r = 0; r < n; ++r) e[r] /= en;
                    or_sign_normalise(e, n);
                }
                break;
            }
        }
        for (int64_t i = 0; i < n; ++i) V[(int64_t)(j + 1) * n + i] = z[i] / be[j];
    }
    *iters = m;
    free(V); free(z); free(h); free(al); free(be); free(T); free(th); free(Y);
    return status;
}

typedef struct { const double *A; int64_t n; } or_dense_ctx;
static void or_dense_op(void *vctx, const double *x, double *y) {
    or_dense_ctx *c = (or_dense_ctx *)vctx;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < c->n; ++i) {
        double acc = 0.0;
        for (int64_t j = 0; j < c->n; ++j) acc += c->A[i * c->n + j] * x[j];
        y[i] = acc;
    }
}

int32_t or_lanczos_dense(const double *A, int64_t n, int32_t k, int32_t m_max, double conv_tol,
                         const double *v0, double *evals, double *evecs, int32_t *iters) {
    or_dense_ctx c = {A, n};
    return or_lanczos(or_dense_op, &c, n, k, m_max, conv_tol, v0, evals, evecs, iters);
}

typedef struct { const float *X; int64_t N; int32_t d; double eps; const double *s; } or_S_ctx;
static void or_S_op(void *vctx, const double *x, double *y) {
    or_S_ctx *c = (or_S_ctx *)vctx;
    or_S_matvec(c->X, c->N, c->d, c->eps, c->s, x, 1, y);
}

int32_t or_lanczos_S(const float *X, int64_t N, int32_t d, double eps, const double *s,
                     int32_t k, int32_t m_max, double conv_tol, const double *v0,
                     double *evals, double *evecs, int32_t *iters) {
    or_S_ctx c = {X, N, d, eps, s};
    return or_lanczos(or_S_op, &c, N, k, m_max, conv_tol, v0, evals, evecs, iters);
}

typedef struct {
    const float *X; int64_t N; int32_t d; double eps; const double *s; const int32_t *perm;
    int32_t L, max_rank, cmax; const int32_t *ranks, *skel; const double *P;
} or_H_ctx;
static void or_H_op(void *vctx, const double *x, double *y) {
    or_H_ctx *c = (or_H_ctx *)vctx;
    or_hmatvec(c->X, c->N, c->d, c->eps, c->s, c->perm, c->L, c->max_rank, c->cmax, c->ranks, c->skel, c->P, x, 1, y);
}

int32_t or_lanczos_hmat(const float *X, int64_t N, int32_t d, double eps, const double *s,
                        const int32_t *perm, int32_t L, int32_t max_rank, int32_t cmax,
                        const int32_t *ranks, const int32_t *skel, const double *P,
                        int32_t k, int32_t m_max, double conv_tol, const double *v0,
                        double *evals, double *evecs, int32_t *iters) {
    or_H_ctx c = {X, N, d, eps, s, perm, L, max_rank, cmax, ranks, skel, P};
    return or_lanczos(or_H_op, &c, N, k, m_max, conv_tol, v0, evals, evecs, iters);
}

/* Lanczos start vector: v0_i = 2u - 1, u the SplitMix64 draw for original index i. */
void or_start_vector(int64_t N, uint64_t seed, double *v0) {
    uint64_t key = or_stream_key(seed, OR_TAG_V0, 0);
    for (int64_t i = 0; i < N; ++i) v0[i] = 2.0 * or_unit(or_rng(key, (uint64_t)i)) - 1.0;
}
