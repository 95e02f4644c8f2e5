/*
 * dmaps.h -- C ABI of the GB300 (sm_103a) diffusion-map eigensolver.
 *
 * The library computes the top-k eigenpairs of the diffusion-map matrix of
 * Gaddameedi, Reiz, Neckel, Bungartz, "Efficient and Scalable Kernel Matrix
 * Approximations using Hierarchical Decomposition" (arXiv 2311.06115):
 *
 *   W_ij  = exp(-||x_i - x_j||^2 / eps)                 (Eq. W, eps = sigma^2)
 *   q     = W 1,  W^a_ij = W_ij / (q_i^a q_j^a)          (Algorithm 1: similarity, density normalisation)
 *   P     = Dg^-1 W^a,  dg = W^a 1                       (Algorithm 1: Markov normalisation)
 *   S     = Dg^-1/2 W^a Dg^-1/2 = diag(s) W diag(s),  s = q^-a dg^-1/2
 *
 * S is the symmetric conjugate of P (same eigenvalues; right eigenvectors of P
 * are psi = Dg^-1/2 phi for eigenvectors phi of S). S is approximated by an
 * H-matrix K~ = D + UV (Eq. 2.18) built once (dm_compress) and applied in every
 * iteration of a Lanczos eigensolver (Algorithm 2 in its symmetric form,
 * Section 2.3.1), which is what scipy's eigsh does with the paper's
 * LinearOperator (Section 3.3).
 *
 * Conventions for every call:
 *   - Return value: DM_OK (0) or a negative DM_E* status; dm_status_str() names it
 *     and dm_last_error() gives the message of the calling thread's last failure.
 *   - Buffers may be host or device memory; the library detects which with
 *     cudaPointerGetAttributes and copies host buffers through the handle's
 *     stream. The caller owns every buffer it passes; the library keeps no
 *     pointer to it after the call returns.
 *   - Vectors are float32 in the ORIGINAL point order; blocks of vectors are
 *     N x nrhs column-major (column c starts at element c*N).
 *   - Calls on one handle are not thread-safe; distinct handles are independent.
 *     All device work of a handle runs on its stream; every call that returns
 *     results to the caller synchronises that stream before returning.
 */
#ifndef DMAPS_H
#define DMAPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define DM_OK 0
#define DM_EINVAL (-1)   /* bad argument (sizes, eps, k, tolerances, NULL pointers) */
#define DM_ENOMEM (-2)   /* device allocation failed */
#define DM_ESTATE (-3)   /* call out of order (e.g. dm_eigs before dm_compress) */
#define DM_ENOCONV (-4)  /* Lanczos reached m_max before the top k converged; results still written */
#define DM_ETIMEOUT (-5) /* a bounded device-side wait gave up */
#define DM_ECUDA (-6)    /* a CUDA runtime call failed */
#define DM_EBUSY (-7)    /* serving queue full or ticket still running */

typedef struct dm_ctx *dm_handle;
typedef uint64_t dm_ticket;

/* Device allocator hooks (e.g. a framework's caching allocator). alloc returns a
 * device pointer aligned to at least 256 bytes, or NULL on failure. */
typedef void *(*dm_alloc_fn)(size_t bytes, void *user);
typedef void (*dm_free_fn)(void *ptr, size_t bytes, void *user);

#define DM_NEAR_AUTO 0   /* pick the faster near-field variant */
#define DM_NEAR_CACHED 1 /* store the leaf blocks K(I_a, I_a) in HBM and stream them */
#define DM_NEAR_ONTHEFLY 2 /* recompute leaf-block entries from the points in every matvec */

typedef struct dm_config {
    uint64_t seed;        /* random choices: ID row samples, Lanczos start vector, bandwidth pairs */
    int32_t near_mode;    /* DM_NEAR_* */
    int32_t m_max;        /* Lanczos basis cap (default 300) */
    double conv_tol;      /* Ritz residual bound beta_j |y_j| <= conv_tol * theta_1 (default 1e-7) */
    int32_t check_every;  /* Lanczos steps between convergence checks, from step ceil(5k/4)+5 on (default 1) */
    int32_t device;       /* CUDA device ordinal (default: the current device) */
    void *stream;         /* cudaStream_t to run on; NULL = a stream the handle creates */
    dm_alloc_fn alloc;    /* NULL = cudaMalloc */
    dm_free_fn free;      /* NULL = cudaFree */
    void *alloc_user;
    int32_t profile;      /* 1 = time every H-matvec of dm_eigs with CUDA events on the handle's stream */
    int32_t shared_device; /* 1 = the device runs other work concurrently (other solves, other
                              processes): each Lanczos step then runs as five ordinary launches
                              instead of one cooperative launch whose blocks wait on one another,
                              so it never depends on SMs that other kernels hold. 0 (default) =
                              one cooperative launch per step. */
    int32_t block_precision; /* near field of the block H-matvec (dm_matvec with nrhs >= 5, or 2..4
                                when the narrow-block form does not apply; cached mode):
                                DM_PREC_FP32 (default, FP32 FMA on the CUDA cores), DM_PREC_TF32
                                (tcgen05 tensor cores, TF32 inputs, FP32 accumulation: about 2^-10
                                relative per term) or DM_PREC_TF32X3 (tcgen05 with each operand
                                split into a TF32 high part and a TF32 remainder, three products
                                hi*hi + hi*lo + lo*hi: about 2^-20 relative per term) */
    int32_t block_size;   /* dm_eigs: 0 or 1 = single-vector Lanczos (default); 2..16 = block Lanczos
                             with this many vectors per step (one block H-matvec per step) */
} dm_config;

#define DM_PREC_FP32 0
#define DM_PREC_TF32 1
#define DM_PREC_TF32X3 2

/* Fill *cfg with the defaults listed above. */
void dm_config_default(dm_config *cfg);

/* Create a handle for N points in R^d (points: N x d row-major float32, host or
 * device). eps > 0 is the kernel scale sigma^2 of Eq. W; eps <= 0 selects the
 * median squared pairwise distance (all pairs when N(N-1)/2 <= 2^20, else 2^20
 * pairs drawn with cfg->seed). alpha is the density exponent of Algorithm 1,
 * step 2 (the paper uses alpha = 1). Computes the degree vectors q, dg and the
 * scaling s exactly (O(N^2) kernel evaluations, FP32 exp, FP64 sums).
 * cfg may be NULL (defaults). points is copied before the call returns; the degree
 * passes may still be running on the handle's stream then (every later call on the
 * handle is ordered after them). Errors: DM_EINVAL if N < 2, d < 1, alpha < 0 or
 * a pointer is NULL; DM_ENOMEM; DM_ECUDA. */
int dm_create(const float *points, int64_t N, int32_t d, double eps, double alpha,
              const dm_config *cfg, dm_handle *out);

/* Build the H-matrix approximation of S (Eq. 2.18, accuracy target Eq. 1.1):
 * a balanced binary partition tree of depth L = min{L : ceil(N/2^L) <= leaf_size}
 * in the Gram distance of W, then per node (bottom-up) an interpolative
 * decomposition of a sampled off-node block whose rank stops at the first
 * pivot with residual norm <= tol * (first pivot norm), capped at max_rank;
 * finally the near (leaf) and far (sibling skeleton) blocks are packed.
 * Errors: DM_EINVAL if tol < 0, leaf_size < 1, max_rank < 1 or the tree would
 * exceed 2^20 leaves; DM_ENOMEM; DM_ECUDA. Replaces any earlier structure. */
int dm_compress(dm_handle h, double tol, int32_t leaf_size, int32_t max_rank);

/* y = K~ x for nrhs right-hand sides (N x nrhs column-major, original order),
 * the LinearOperator matvec/matmat of Section 3.3. Before dm_compress it
 * applies the exact S with entries generated on the fly (O(N^2) per column).
 * x and y must not overlap. Errors: DM_EINVAL (nrhs < 1, NULL); DM_ECUDA. */
int dm_matvec(dm_handle h, const float *x, float *y, int32_t nrhs);

/* Top-k eigenpairs of K~ by Lanczos with full reorthogonalisation (eigsh's
 * role in Section 3.3; Algorithm 2 in symmetric form). evals: k doubles,
 * descending (the first is 1 up to the approximation error). evecs: N x k
 * column-major float32 (may be NULL), orthonormal, in original point order,
 * each column signed so its largest-magnitude entry is positive.
 * Errors: DM_ESTATE before dm_compress; DM_EINVAL if k < 1 or k >= N or
 * k > m_max; DM_ENOCONV if m_max steps did not converge (best Ritz pairs are
 * still written); DM_ECUDA. */
int dm_eigs(dm_handle h, int32_t k, double *evals, float *evecs);

/* Top-k eigenpairs of `count` compressed handles at once: the batching of many uneven point
 * clouds (no paper counterpart; each handle's solve is dm_eigs' single-vector Lanczos of
 * Algorithm 2 in its symmetric form, Section 2.3.1). Every Lanczos step of every handle not
 * yet converged runs in the same launches, each handle at its own step: the H-matvec of
 * Eq. 2.18 in three launches for all handles (leaf N2S and the climb up each tree; the
 * top-down sweep of the trees' internal levels, split over subtrees; the near field fused
 * with the leaf S2N), and the three Gram-Schmidt passes. The start vectors of the handles, and the
 * Ritz vectors of the handles finishing at the same step, are formed in shared launches too.
 * Each handle is checked on its own schedule (from step ceil(5k/4)+5, every check_every
 * steps); the checks due after a step share one launch of Ritz values, read by the host one
 * step later while the next step runs, so a converged handle takes one step more than its
 * solo solve before it leaves (its Ritz pairs are those of the checked step). The launch
 * count per step does not grow with the number of handles. Each handle keeps its own seed,
 * m_max, check_every and conv_tol; cfg.block_size and block_precision are ignored.
 * hs: `count` distinct compressed handles on one device; the work runs on hs[0]'s stream
 * after the queued work of every handle. evals: count x k doubles, handle i at i k,
 * descending (host or device). evecs: NULL, or `count` pointers, each NULL or N_i x k floats
 * (host or device, as dm_eigs). status: NULL or `count` ints, DM_OK or DM_ENOCONV per handle.
 * Returns DM_OK when every handle converged, DM_ENOCONV when some reached m_max (all results
 * still written). Errors: DM_EINVAL (NULL arguments, count < 1, k outside [1, 32] or >= some
 * N, handles repeated or on different devices); DM_ESTATE (a handle not compressed);
 * DM_ENOMEM; DM_ECUDA. */
int dm_eigs_batch(dm_handle *hs, int32_t count, int32_t k, double *evals, float **evecs, int32_t *status);

/* Diffusion coordinates of the last dm_eigs: psi_i = theta_i^t Dg^-1/2 phi_i
 * (Algorithm 1: t-step random walk and eigendecomposition; the eigenvalues of
 * P^t are theta^t and its right eigenvectors Dg^-1/2 phi). psi: N x k
 * column-major float32 (k <= the k of the last dm_eigs). Errors: DM_ESTATE if
 * dm_eigs has not run; DM_EINVAL. */
int dm_coords(dm_handle h, int32_t k, int32_t t, float *psi);

/* Intrinsic dimension d(t) (Algorithm 1, its lower dimension) from the eigenvalues of a
 * dm_eigs call. The paper's inequality is garbled and its delta unspecified; the
 * reading is Coifman and Lafon's definition, which the paper's Algorithm 1 restates:
 * with the eigenvalues indexed from the trivial one, lambda_0 = evals[0] (= 1), d(t) is the largest
 * l >= 1 with |lambda_l|^t > delta |lambda_1|^t, i.e. the number of non-trivial
 * diffusion coordinates still above the precision factor delta after t steps.
 * evals: k host doubles, descending as dm_eigs returns them. t >= 1; 0 < delta < 1.
 * *d receives d(t) (0 when lambda_1 = 0); *at_k (may be NULL) receives 1 when
 * d(t) = k - 1, i.e. every eigenvalue given passed and the true d(t) may be larger.
 * Errors: DM_EINVAL for NULL evals or d, k < 2, t < 1, delta outside (0, 1) or a
 * NaN eigenvalue. Host computation only; no device work. */
int dm_intrinsic_dim(const double *evals, int32_t k, int32_t t, double delta, int32_t *d, int32_t *at_k);

/* Leaf-size autotuner (no counterpart in the paper: GOFMM takes max_leaf_node_size from the
 * user). For each of the ncand candidate leaf sizes, compresses the handle's operator with
 * (tol, leaf, max_rank), times the compression and one nrhs = 1 H-matvec (median of 5, CUDA
 * events on the handle's stream) and scores cost = compression + (2k + 20) H-matvecs, the
 * usual Lanczos step count for k pairs. *best_leaf gets the cheapest candidate and the
 * handle is left compressed with it; cost_ms (may be NULL) gets every candidate's score.
 * Errors: DM_EINVAL (no candidates, k < 1, a candidate dm_compress rejects); DM_ECUDA. */
int dm_tune_leaf(dm_handle h, double tol, int32_t max_rank, int32_t k, const int32_t *candidates, int32_t ncand,
                 int32_t *best_leaf, float *cost_ms);

/* Release every device buffer, stream and event of the handle, ordered after the work
 * it has queued (no paper counterpart). The handle must not be used afterwards.
 * Errors: DM_EINVAL for a NULL handle. */
int dm_destroy(dm_handle h);

/* Name of a status code ("DM_OK", "DM_EINVAL", ...; "DM_UNKNOWN" otherwise), and the
 * message of the calling thread's last failure (empty if none). Both strings are
 * library-owned; the message stays valid until this thread's next failing call. */
const char *dm_status_str(int status);
const char *dm_last_error(void);

/* ---- introspection (tests, checkpointing) ---- */
typedef struct dm_stats {
    int64_t N;
    int32_t d, L;
    double eps, alpha, tol;
    int32_t leaf_max, max_rank, rank_min, rank_max;
    double rank_mean;
    int64_t near_bytes;      /* stored leaf blocks (cached mode) */
    int64_t basis_bytes;     /* P matrices actually used (sum of s_a * |C_a| * 4) */
    int64_t far_bytes;       /* sibling skeleton blocks (sum of s_l * s_r * 4) */
    int64_t matvec_bytes;    /* algorithmic bytes of one nrhs=1 H-matvec in the active near mode */
    int32_t near_mode;       /* mode in use after AUTO resolution */
    int32_t lanczos_iters;   /* steps of the last dm_eigs */
    int32_t converged;       /* 1 if the last dm_eigs converged */
    float ms_create, ms_tree, ms_skeleton, ms_pack, ms_eigs; /* device time of each phase */
    int32_t matvec_calls;    /* H-matvecs timed in the last dm_eigs (profile = 1) */
    float ms_matvec;         /* their summed device time */
    int32_t hmatvec_path;    /* 0 = leaf N2S + one-cluster tree pass + near stream (the upper
                                tree fits the shared memory of a cluster of 8 CTAs), 2 = the same
                                with a cluster of 16 CTAs (higher ranks), 1 = chained two-launch
                                form (deep trees at ranks too high for either cluster) */
    int32_t degree_path;     /* degree passes of dm_create: 0 = CUDA cores (FP32 entries),
                                1 = tensor cores, TF32 three-term split Gram matrix (d >= 16),
                                2 = tensor cores, exact BF16 Gram matrix (8-bit quantised data) */
    float ms_degrees;        /* device time of the two degree passes of dm_create, including the
                                q^-a step between them (tensor-core path: and the operand packing) */
} dm_stats;

/* Phase times and structure statistics of the handle's last calls (introspection; no
 * paper counterpart), copied into the caller's struct. Errors: DM_EINVAL for NULL. */
int dm_get_stats(dm_handle h, dm_stats *st);

/* Number of CUDA kernels this library has launched in this process (all handles). */
int64_t dm_kernel_launches(void);

/* Throughput of the GPU's MUFU ex2 instruction, the exponential of every kernel entry in
 * the degree passes and the on-the-fly near field (no paper counterpart; the denominator
 * of those kernels' roofline). Runs 8 x SMs blocks of 256 threads, each thread 8 independent
 * chains of 4096 exponentials, once to warm up and once timed with CUDA events on the legacy
 * default stream of the current device. *ex2_count: exponentials of the timed launch;
 * *ms: its duration. Allocates and frees a small device buffer; synchronous.
 * Errors: DM_EINVAL for NULL outputs; DM_ENOMEM; DM_ECUDA. */
int dm_sfu_peak(int64_t *ex2_count, float *ms);

/* Failure-detection self-test of the bounded grid barrier that separates the passes of
 * the cooperative Lanczos step (no paper counterpart). `blocks` (1..8, always resident at
 * once) blocks meet at that barrier, whose target counts `missing` more arrivals than
 * there are blocks. Each block polls at most `spin_limit` (1..2^24) times, about 0.1-1 us
 * per poll, then raises the device error flag and returns, exactly as the Lanczos step
 * does. *passed (may be NULL) receives the number of blocks that got through.
 * Returns DM_OK when every block passed (missing = 0), DM_ETIMEOUT when the wait gave up
 * (missing > 0: nothing can complete the count), so the timeout path is exercised
 * without faulting or hanging the device; the device stays usable either way.
 * Allocates and frees 16 bytes of device memory on the current device; synchronous.
 * Errors: DM_EINVAL for arguments out of range; DM_ENOMEM; DM_ECUDA. */
int dm_selftest_wait_timeout(int32_t blocks, int32_t missing, int64_t spin_limit, int32_t *passed);

/* ---- serving: continuous admission of independent solves ----
 * A process-wide server builds `slots` requests at once (dm_create + dm_compress), each slot
 * on its own CUDA stream, so their kernels overlap on the device. Requests wait in a queue
 * and are admitted first-fit, in arrival order, whenever a slot is free and the request's
 * device footprint (dm_request_bytes) fits in what is left of the HBM budget (a request
 * larger than the whole budget runs alone). A built single-vector request (block_size 0 or
 * 1) then joins a batched eigensolver of dm_eigs_batch, run by a thread of the server (four,
 * by request size: up to 5,000, 15,000, 40,000 points and beyond, the smaller on
 * higher-priority streams, so that small requests are not held to large ones' step time):
 * every resident request's Lanczos step runs in the same launches, each at its own step, and
 * a request leaves (its results copied out, its memory released) when its own check says it
 * converged; requests join between steps (continuous batching at the step level). Block
 * requests run their eigensolve on their slot. Each result is that of dm_create +
 * dm_compress + dm_eigs on a fresh handle with check_every = 2: the same Lanczos steps and
 * checks, equal up to the FP32 summation order of the batched H-matvec.
 * Submit and poll are thread-safe. No counterpart in the paper. */
typedef struct dm_request {
    const float *points;   /* N x d row-major float32, host memory; copied by dm_submit */
    int64_t N;
    int32_t d;
    double eps, alpha;     /* as dm_create (eps <= 0: median squared distance) */
    double tol;            /* as dm_compress */
    int32_t leaf_size, max_rank;
    int32_t k;             /* eigenpairs wanted (as dm_eigs) */
    int32_t want_vectors;  /* 1: return the N x k eigenvectors too */
    uint64_t seed;
    int32_t block_size;    /* as dm_config.block_size: 0/1 single-vector, 2..16 block Lanczos */
} dm_request;

typedef struct dm_result {
    int32_t status;        /* DM_OK, DM_ENOCONV or the failing call's status */
    int32_t k;
    int64_t N;
    const double *evals;   /* k values, descending; library-owned until dm_release */
    const float *evecs;    /* N x k column-major, or NULL; library-owned until dm_release */
    double submit_ms, start_ms, done_ms;  /* wall-clock times since dm_serve_start */
    int32_t lanczos_iters;
    const char *error;     /* message of the failing call ("" on success); library-owned */
    double built_ms;       /* wall-clock time since dm_serve_start when the request's build
                              (dm_create + dm_compress) ended and its eigensolve began */
} dm_result;

typedef struct dm_serve_config {
    int32_t device;             /* CUDA device ordinal (-1: current) */
    int32_t slots;              /* concurrent builds (and block solves) (default 4) */
    uint64_t hbm_budget_bytes;  /* admission budget (0: 150 GB) */
    int32_t queue_capacity;     /* waiting requests before DM_EBUSY (0: 65536) */
} dm_serve_config;

/* Device bytes one solve of `r` allocates at its peak (the admission estimate). */
uint64_t dm_request_bytes(const dm_request *r);
/* Start the server (DM_ESTATE if running; DM_ECUDA without a device). */
int dm_serve_start(const dm_serve_config *cfg);
/* Stop accepting work, finish the running builds and every resident solve, drop queued
 * requests (their status becomes DM_ESTATE), join the threads and free every result. */
int dm_serve_stop(void);
/* Queue a request; *t identifies it. DM_EINVAL for an invalid request, DM_ESTATE
 * if the server is not running, DM_EBUSY if the queue is full. */
int dm_submit(const dm_request *r, dm_ticket *t);
/* Non-blocking: *done = 1 once the solve finished (r, if not NULL, then holds the
 * result); 0 while queued or running. DM_EINVAL for an unknown ticket. */
int dm_poll(dm_ticket t, dm_result *r, int32_t *done);
/* Free a finished request's result buffers (DM_EBUSY while it is still running). */
int dm_release(dm_ticket t);

/* ---- allocation-free entry point (no counterpart in the paper) ----
 * For callers that cannot let a library allocate device memory: code running
 * inside a framework that owns all device memory and forbids side allocations,
 * services with a memory budget fixed up front, and hot paths that must not take
 * cudaMalloc's implicit device-wide synchronisation.
 *
 * Computes the degree vectors of dm_create (q = W 1, dg = W^a 1,
 * s = q^-a dg^-1/2, each N doubles in the original point order) for N points
 * (N x d row-major float32) with an explicit eps > 0, enqueued on `stream`
 * (a cudaStream_t; NULL = the legacy default stream) and not synchronised: the
 * outputs are ready when the stream reaches this work. Its kernel entries are
 * always the FP32 difference form |x_i - x_j|^2, where dm_create takes a centred
 * dot-product form at d = 3 and a tensor-core Gram matrix at d >= 16, so the two
 * agree to rounding, not bit for bit: within 2e-6 relative at d <= 15 and 5e-6
 * relative at d >= 16 (FP32 entries, FP64 sums). All four pointers must be
 * device memory the caller owns, on the current device. It calls no cudaMalloc, cudaFree or other
 * allocating routine: its intermediate arrays live in one fixed 16 MiB
 * module-scope device array that every GPU loading this library holds until
 * the process exits, which limits N * (4 d + 16) bytes (rounded up to 256-byte
 * pieces) to 16 MiB — about 670,000 points at d = 3.
 * The first call on a device looks up that array's device address with that
 * device current; make this first call before any stream capture. The address
 * is kept for the life of the process: after cudaDeviceReset on a device, do not
 * call this function on that device again.
 * Every call shares the one array, so calls whose work overlaps on the GPU
 * (different streams, threads or devices' streams racing on one device) race;
 * serialise them. Errors: DM_EINVAL on a NULL or host pointer, a pointer to
 * another device's memory, N < 2, d < 1, eps <= 0, alpha < 0, or a size above
 * the limit; DM_ECUDA if a launch fails. The output pointers must each hold N
 * doubles: the library cannot check the size of a raw device buffer. */
int dm_degrees_noalloc(const float *points, int64_t N, int32_t d, double eps, double alpha,
                       double *q, double *dg, double *s, void *stream);

/* eps in use, and the degree vectors of Algorithm 1 (N doubles each, original
 * order, host or device buffers; for dm_get_degrees any of q, dg, s may be NULL).
 * Errors: DM_EINVAL for a NULL handle (or a NULL eps); DM_ECUDA. */
int dm_get_eps(dm_handle h, double *eps);
int dm_get_degrees(dm_handle h, double *q, double *dg, double *s);

/* The compressed structure, in the layout dm_load_hmatrix accepts:
 * perm[N] (perm[pos] = original index); ranks[2^(L+1)-1] (root 0);
 * skel[node*max_rank + t] = position of skeleton t of node (-1 past the rank);
 * P[(node*max_rank + t)*cmax + j] = interpolation matrix entry (row t, candidate
 * j; candidates of a leaf are its positions in order, of an internal node the
 * left then right child skeletons), cmax = max(ceil(N/2^L), 2*max_rank).
 * Query sizes first with dm_get_tree(h, &L, NULL) and dm_get_stats. Buffers are
 * caller-owned (host or device); a NULL output is skipped. Errors: DM_EINVAL for a NULL
 * handle; DM_ESTATE before dm_compress or dm_load_hmatrix; DM_ECUDA. */
int dm_get_tree(dm_handle h, int32_t *L, int32_t *perm);
int dm_get_hmatrix(dm_handle h, int32_t *ranks, int32_t *skel, float *P);

/* Adopt an externally built structure (same layout as dm_get_hmatrix; host
 * buffers) instead of running dm_compress: checkpoint/resume of a compressed
 * operator, and replay of a reference structure. The near and far blocks are
 * packed from the handle's own points and scaling. Errors: DM_EINVAL on an
 * inconsistent structure (bad permutation, ranks above max_rank, skeleton
 * positions outside their node); DM_ENOMEM; DM_ECUDA. */
int dm_load_hmatrix(dm_handle h, int32_t L, int32_t max_rank, const int32_t *perm,
                    const int32_t *ranks, const int32_t *skel, const float *P);

#ifdef __cplusplus
}
#endif
#endif /* DMAPS_H */
