/*
 * oracle.h -- plain FP64 CPU reference for the diffusion-map H-matvec Lanczos path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product (the CUDA library, its
 * Python binding) may include, link or call this code; only tests/, the
 * smoke check and the CPU-baseline leg of the benchmark do.
 *
 * Conventions: points X are N x d row-major float32 (the storage type of the
 * product's input), promoted to double on load; every computed quantity is
 * double. Indices of points are "original" (row of X) unless called
 * "positions", which index the tree permutation perm[pos] = original index.
 */
#ifndef DM_ORACLE_H
#define DM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- counter-based random numbers (SplitMix64, Steele/Lea/Flood 2014) ---- */
uint64_t or_splitmix64_next(uint64_t *state);
uint64_t or_stream_key(uint64_t seed, uint32_t tag, uint64_t id);
uint64_t or_rng(uint64_t key, uint64_t ctr);

/* ---- kernel, bandwidth, degrees (Eq. W and Algorithm 1: similarity matrix and normalisations) ---- */
double or_sqdist(const float *X, int32_t d, int64_t i, int64_t j);
double or_median_sqdist(const float *X, int64_t N, int32_t d, uint64_t seed);
void or_kernel_W(const float *X, int64_t N, int32_t d, double eps, double *W);
void or_degrees(const float *X, int64_t N, int32_t d, double eps, double alpha,
                double *q, double *dg, double *s);
void or_q_rows(const float *X, int64_t N, int32_t d, double eps,
               const int64_t *rows, int64_t nrows, double *q_rows);
void or_S_matvec(const float *X, int64_t N, int32_t d, double eps, const double *s,
                 const double *x, int32_t nrhs, double *y);
void or_S_matvec_rows(const float *X, int64_t N, int32_t d, double eps, const double *s,
                      const double *x, const int64_t *rows, int64_t nrows, double *y_rows);

/* ---- partition tree (geometry-oblivious ball tree) ---- */
int32_t or_tree_depth(int64_t N, int64_t leaf_size);
void or_node_range(int64_t N, int32_t node, int64_t *start, int64_t *size);
int32_t or_tree(const float *X, int64_t N, int32_t d, double eps, int64_t leaf_size, int32_t *perm);

/* ---- skeletonization (interpolative decomposition) and HSS matvec (Eq. 2.18) ---- */
int32_t or_skeletonize(const float *X, int64_t N, int32_t d, double eps, const double *s,
                       const int32_t *perm, int32_t L, double tol, int32_t max_rank,
                       int32_t cmax, uint64_t seed, int32_t *ranks, int32_t *skel, double *P);
void or_hmatvec(const float *X, int64_t N, int32_t d, double eps, const double *s,
                const int32_t *perm, int32_t L, int32_t max_rank, int32_t cmax,
                const int32_t *ranks, const int32_t *skel, const double *P,
                const double *x, int32_t nrhs, double *y);

/* ---- dense symmetric eigensolver and Lanczos (Algorithm 2, Section 2.3) ---- */
int32_t or_jacobi(const double *A, int32_t n, double *evals, double *evecs);
int32_t or_lanczos_dense(const double *A, int64_t n, int32_t k, int32_t m_max, double conv_tol,
                         const double *v0, double *evals, double *evecs, int32_t *iters);
int32_t or_lanczos_S(const float *X, int64_t N, int32_t d, double eps, const double *s,
                     int32_t k, int32_t m_max, double conv_tol, const double *v0,
                     double *evals, double *evecs, int32_t *iters);
int32_t or_lanczos_hmat(const float *X, int64_t N, int32_t d, double eps, const double *s,
                        const int32_t *perm, int32_t L, int32_t max_rank, int32_t cmax,
                        const int32_t *ranks, const int32_t *skel, const double *P,
                        int32_t k, int32_t m_max, double conv_tol, const double *v0,
                        double *evals, double *evecs, int32_t *iters);
void or_start_vector(int64_t N, uint64_t seed, double *v0);

#ifdef __cplusplus
}
#endif
#endif
