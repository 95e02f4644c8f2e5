// dm_internal.cuh -- shared definitions of the CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <vector>
#include <stdint.h>

#include "dmaps.h"

#define DM_WARP 32

// process-wide count of kernel launches (dm_kernel_launches)
void dm_count_launches(long long n);
// record `msg` as the calling thread's last error (dm_last_error) and return `code`
int dm_fail_msg(int code, const char *msg);
#define DM_FULL 0xffffffffu

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) used as a counter-based
// generator: output (key, ctr) is the (ctr+1)-th draw of a generator whose
// state starts at key; streams are keyed by (seed, purpose tag, id).
// ---------------------------------------------------------------------------
#define DM_GAMMA 0x9E3779B97F4A7C15ULL
#define DM_TAG_ROWS 1u
#define DM_TAG_V0 2u
#define DM_TAG_PAIRS 3u

__host__ __device__ __forceinline__ uint64_t dm_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t dm_stream_key(uint64_t seed, uint32_t tag, uint64_t id) {
    return dm_mix64(seed * DM_GAMMA + ((uint64_t)tag << 48) + id);
}
__host__ __device__ __forceinline__ uint64_t dm_rng(uint64_t key, uint64_t ctr) {
    return dm_mix64(key + (ctr + 1) * DM_GAMMA);
}
// integer in [0, n) from the top 32 bits (n < 2^32)
__host__ __device__ __forceinline__ uint64_t dm_below(uint64_t u, uint64_t n) { return ((u >> 32) * n) >> 32; }
// double in [0, 1) from the top 53 bits
__host__ __device__ __forceinline__ double dm_unit(uint64_t u) {
    return (double)(u >> 11) * (1.0 / 9007199254740992.0);
}

// ---------------------------------------------------------------------------
// Perfect binary partition tree: node (level l, k) has heap id 2^l - 1 + k; a
// node of n points splits into ceil(n/2) (left) and floor(n/2) (right).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int dm_level_of(int node) {
    int l = 0;
    unsigned h = (unsigned)node + 1u;
    while (h >> (l + 1)) ++l;
    return l;
}
__host__ __device__ __forceinline__ void dm_node_range(int64_t N, int node, int64_t *start, int64_t *size) {
    int64_t st = 0, sz = N;
    unsigned h = (unsigned)node + 1u;
    int lvl = dm_level_of(node);
    for (int b = lvl - 1; b >= 0; --b) {
        int64_t left = (sz + 1) / 2;
        if ((h >> b) & 1u) {
            st += left;
            sz -= left;
        } else {
            sz = left;
        }
    }
    *start = st;
    *size = sz;
}
static inline int dm_depth_for(int64_t N, int64_t leaf) {
    int L = 0;
    while (((N + ((int64_t)1 << L) - 1) >> L) > leaf) ++L;
    return L;
}

// FP64 -> uint64 whose unsigned order is the numeric order (no NaNs here).
__device__ __forceinline__ uint64_t dm_order_key(double v) {
    uint64_t u = (uint64_t)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ULL);
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ float dm_warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(DM_FULL, v, o);
    return v;
}
__device__ __forceinline__ double dm_warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(DM_FULL, v, o);
    return v;
}

// Asynchronous global->shared copies (cp.async): issued back to back with no register
// round trip, completed by dm_cp_async_wait_all(). A block must wait for its own copies
// before it exits or reuses the destination.
__device__ __forceinline__ void dm_cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void dm_cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void dm_cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Grid-wide barrier of a cooperative launch (every block resident) with a bounded wait:
// block threads 0 arrive on *ctr and poll it (acquire) until it reaches `target`; a block
// that polls more than spin_limit times, or sees *err raised, raises *err and reports
// false, and the kernel returns. Counters grow monotonically within a launch sequence.
constexpr long long kBarrierSpinLimit = 1ll << 22;

__device__ __forceinline__ unsigned dm_ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// returns false when the barrier timed out (in this or another block)
__device__ __forceinline__ bool grid_barrier(unsigned *ctr, unsigned target, int *err,
                                             long long spin_limit = kBarrierSpinLimit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
        int ok = 1;
        long long spins = 0;
        while (dm_ld_acquire_gpu(ctr) < target) {
            if (++spins > spin_limit || *((volatile int *)err) != 0) {
                ok = 0;
                atomicExch(err, 1);
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// 1/sqrt(d) for d > 0 without the FP64 divide and square-root sequences (slow on this part's
// narrow FP64 pipe): d is scaled by an even power of two into [1, 4), an FP32 estimate is
// refined by two Newton steps y <- y (3 - d y^2) / 2 in FP64 (relative error 2^-23, then
// ~2^-45, then below FP64 rounding), and the power of two is restored.
__device__ __forceinline__ double dm_rsqrt_fp64(double d) {
    const long long bits = __double_as_longlong(d);
    const int ex = (int)((bits >> 52) & 0x7ff) - 1023;
    const int half = ex >= 0 ? ex / 2 : -((1 - ex) / 2);
    const double down = __longlong_as_double((long long)(1023 - 2 * half) << 52);  // 2^-2half
    const double ds = d * down;
    double y = (double)rsqrtf((float)ds);
    y = y * (1.5 - 0.5 * ds * y * y);
    y = y * (1.5 - 0.5 * ds * y * y);
    return y * __longlong_as_double((long long)(1023 - half) << 52);  // 2^-half
}

// exp2 on the MUFU unit (PTX ex2.approx.ftz.f32: documented max error ~2 ulp over its range)
__device__ __forceinline__ float dm_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// binary32 -> binary64 on the integer pipes (IEEE 754 formats: the exponent is rebiased by
// 1023 - 127 = 896 and the 23 fraction bits move to the top of the 52): exact, so identical to
// the conversion instruction, which runs on the FP64 pipe that bounds the distance sums below.
// Zeros keep their sign; subnormals, infinities and NaNs take the conversion instruction.
__device__ __forceinline__ double dm_widen(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0xffu || (e == 0u && (u & 0x7fffffu) != 0u)) return (double)f;
    const unsigned mag = e == 0u ? 0u : ((e + 896u) << 20) | ((u >> 3) & 0xfffffu);
    return __hiloint2double((int)((u & 0x80000000u) | mag), (int)(u << 29));
}
__device__ __forceinline__ double dm_widen(double f) { return f; }

// Squared distance of two FP32 points in FP64 without contraction, in the order
// k = 0..d-1 (reproducible bit for bit on any IEEE machine).
// T = float, or double for points widened once beforehand (the same operations in the same
// order either way)
template <class T>
__device__ __forceinline__ double dm_sqdist64(const T *a, const T *b, int d) {
    double r2 = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = __dsub_rn(dm_widen(a[k]), dm_widen(b[k]));
        r2 = __dadd_rn(r2, __dmul_rn(t, t));
    }
    return r2;
}
// dimension from which the tree build reads an FP64 copy of the points (its distance sums
// stream each node's rows: at high dimension the FP64 copy's reads cost less than widening
// every coordinate per pass; the sampled median pairs, which read rows at random, widen)
constexpr int kWideMinD = 16;

// ---------------------------------------------------------------------------
// Device-side structure of a compressed operator (all pointers device memory).
// ---------------------------------------------------------------------------
// dynamic shared memory per CTA that the cluster pass over the upper tree may use
constexpr int kTreeSmemBudget = 226 * 1024;  // under the 227 KB opt-in limit of one CTA
constexpr int kTreeMaxCtas = 16;  // largest cluster of the one-cluster tree pass

struct DmHmat {
    int64_t N;
    int d;
    int L;              // tree depth; leaves are level L
    int leaf_max;       // ceil(N / 2^L)
    int ldk;            // leading dimension of a stored leaf block (leaf_max rounded up to 4)
    int max_rank;
    int rank_hi;        // largest rank actually present (<= max_rank)
    int cmax;           // max candidates of a node = max(leaf_max, 2 max_rank)
    int ldp;            // row stride of a P slot (cmax rounded up to 4)
    const int32_t *perm;   // perm[pos] = original index
    const int32_t *ranks;  // per node
    const int32_t *skel;   // per node, max_rank positions
    const float *P;        // per node slot max_rank x ldp, row-major
    const float *PT;       // per leaf: P_leaf transposed (point-major), leaf_max rows of pt_ld[leaf] floats
                           // from PT + pt_off[leaf], zero past the leaf's rank
    int ldt;               // rank_hi rounded up to 4 (the largest pt_ld)
    const int64_t *pt_off; // per leaf: offset of its PT rows (floats)
    const int *pt_ld;      // per leaf: row stride of its PT rows, its rank rounded up to 4 (>= 4)
    const float *B;        // per internal node slot max_rank x max_rank: K(S_l, S_r), row-major s_l x s_r
    const float *Knear;    // per leaf slot leaf_max x ldk (cached mode)
    const float *Xs;       // points in position order, scaled by sqrt(log2(e)/eps), N x d (on-the-fly mode)
    const float *sp;       // s in position order (FP32)
    float *what;           // per node max_rank: skeleton weights (N2S)
    float *uhat;           // per node max_rank: S2S parts
    float *ynear;          // N, near-field result in position order
    unsigned *cnt;         // per node arrival counters of the upward pass (zero between calls)
    // Upper-tree layout for the cluster pass (tree_ok = 1): the tree is cut at level tree_ls
    // into 2^tree_ls subtrees, one CTA of a cluster each; CTA 0 also owns the levels above.
    // tlay[node] = {P offset, B offset, vector offset, mirror offset} in floats within the
    // owning CTA's shared memory; -1 = not resident (P, B read from global memory) or none.
    const int4 *tlay;
    const int2 *town;      // per node: offsets of its own w and u in its owner's shared memory
    int tree_ok;
    int tree_ls;
    int tree_smem;         // bytes of dynamic shared memory per CTA of the cluster pass
    float *timg;           // per CTA: its shared-memory image (metadata, B and P operands)
    const int *timg_off;   // 2^tree_ls + 1 offsets (floats, multiples of 4) of the images in timg
    int *err;              // set when a bounded wait of the H-matvec gives up
};

// row i of leaf `leaf`'s point-major basis (pt_ld[leaf] floats, 16-byte aligned)
__device__ __forceinline__ const float *dm_pt_row(const DmHmat &H, int leaf, int i) {
    return H.PT + H.pt_off[leaf] + (size_t)i * H.pt_ld[leaf];
}

// ---------------------------------------------------------------------------
// Launchers (host functions in each .cu; all enqueue on `st` and return the
// launch status).
// ---------------------------------------------------------------------------
// k_degrees.cu
cudaError_t dm_launch_pair_sqdist(const float *X, int64_t N, int d, uint64_t seed, double *out, int64_t m,
                                  cudaStream_t st);
// out[0..n) = X[0..n) in FP64
cudaError_t dm_launch_widen(const float *X, int64_t n, double *out, cudaStream_t st);
size_t dm_select_state_bytes();
// st2, fork, join (optional, all three or none): a second stream for the second order statistic
cudaError_t dm_launch_select_median(double *vals, int64_t m, void *state, double *result, cudaStream_t st,
                                    cudaStream_t st2 = nullptr, cudaEvent_t fork = nullptr, cudaEvent_t join = nullptr);
cudaError_t dm_launch_scale_points(const float *X, int64_t N, int d, double eps, float *Xs, cudaStream_t st);
cudaError_t dm_launch_degree_pass(const float *Xs, int64_t N, int d, const float *wcol, double *out,
                                  cudaStream_t st);
cudaError_t dm_launch_center_scale(const float *X, int64_t N, int d, double eps, float *Xs, float *nrm, float *nmax,
                                   double *work, cudaStream_t st);
cudaError_t dm_launch_degree_pass_centered(const float *Xs, const float *nrm, const float *nmax, int64_t N, int d,
                                           const float *wcol, double *out, cudaStream_t st);
cudaError_t dm_launch_finish_degrees(int64_t N, double alpha, const double *q, double *qa, float *qaf,
                                     cudaStream_t st);
cudaError_t dm_launch_finish_scaling(int64_t N, const double *qa, double *dgsum, double *s, float *sf,
                                     cudaStream_t st);
cudaError_t dm_launch_dense_matvec_ws(const float *Xs, const float *sf, int64_t N, int d, const float *x, float *y,
                                      float *tmpw, double *acc, cudaStream_t st);

// k_degtc.cu -- degree passes of high-dimensional points on the tensor cores
struct DmDegTc {
    int64_t N;
    int d, dpad, kpad;  // kpad: K of the GEMM (dpad for quantised data, 3 dpad otherwise)
    bool quant;         // BF16-exact quantised operands (else the TF32 three-term split)
    float kappa;        // log2(e) sigma^2 / eps
    void *A, *B;        // N x kpad operands (BF16 or FP32)
    float *an;          // kappa n_i
    double *sums;       // column sums
    unsigned *q_bad;
};
constexpr int kDegTcMinD = 16;  // dimensions from which the degree passes use the tensor cores
size_t dm_degtc_work_bytes(int64_t N, int d);
bool dm_degtc_available();
cudaError_t dm_degtc_prepare(const float *X, int64_t N, int d, double eps, void *work, DmDegTc *S,
                             cudaStream_t st);
cudaError_t dm_degtc_pass(const DmDegTc &S, const float *w, double *out, int *err, cudaStream_t st);

// k_tree.cu
struct DmTreeWork {
    double *wbuf;     // N doubles
    uint64_t *keys;   // N keys
    void *items;      // dm_tree_items_bound(N, L) items of dm_tree_item_bytes() each
    void *cand1;      // as many candidates of dm_tree_cand_bytes() each
    void *cand2;
    int max_items;
    // multi-CTA split of large nodes (sel == nullptr: one CTA per node at every level)
    void *sel;        // max_big per-node select states of dm_tree_sel_bytes()
    unsigned *hist;   // max_big x 256 digit histograms
    void *icnt;       // max_items int2 per-item counts
    int max_big;
};
size_t dm_tree_items_bound(int64_t N, int L);
size_t dm_tree_item_bytes();
size_t dm_tree_sel_bytes();
int64_t dm_tree_big_node();  // nodes above this many points split over many CTAs
size_t dm_tree_cand_bytes();
// X64: NULL, or the FP64 copy of X, read instead of X
cudaError_t dm_tree_build(const float *X, const double *X64, int64_t N, int d, double eps, int L, int32_t *perm_a,
                          int32_t *perm_b, int32_t **perm_out, DmTreeWork *w, cudaStream_t st);

// k_skel.cu
struct DmSkelWork {
    float *A;      // per node slot cmax x ldr (column-major sampled block)
    float *R;      // per node slot max_rank x cmax
    float *Q;      // per node slot max_rank x ldr
    int rmax;
    int ldr;       // rmax rounded up to 4
};
int dm_skel_max_candidates();
size_t dm_skel_smem_bytes(int cmax, int rmax, int max_rank);
cudaError_t dm_skeletonize(const float *Xs, const float *sf, int64_t N, int d, int L, const int32_t *perm,
                           double tol, int max_rank, int cmax, int ldp, uint64_t seed, int32_t *ranks,
                           int32_t *skel, float *P, DmSkelWork *w, cudaStream_t st);
cudaError_t dm_pack(const DmHmat &H, float *Knear, float *B, bool pack_near, cudaStream_t st);
cudaError_t dm_transpose_leaf_bases(const DmHmat &H, float *PT, cudaStream_t st);
cudaError_t dm_permute_points(const float *Xs, const float *sf, const int32_t *perm, int64_t N, int d,
                              float *Xp, float *sp, cudaStream_t st);

// k_hmatvec.cu
// x, y: FP32 vectors; `permuted` = vectors are in position order (Lanczos) instead of original order.
cudaError_t dm_hmatvec(const DmHmat &H, int near_mode, const float *x, float *y, bool permuted, cudaStream_t st);
int dm_near_rows(int near_mode, int leaf_max);
// Raise a kernel's dynamic shared memory cap to at least `bytes` on the current device.
// Process-wide and monotone (never lowers the cap), so concurrent solves on other host
// threads cannot shrink it between another thread's check and its launch.
cudaError_t dm_allow_smem(const void *kern, size_t bytes);
// the chained two-launch form (k_hmatvec.cu), used when the cluster pass does not fit
// launch shape of the chained form for one problem (blocks of its two launches, shared memory)
struct DmChainShape {
    int near_rows, up_blocks, near_blocks, down_blocks, climb_smem, chain_smem;
    size_t smem1, smem2;
};
DmChainShape dm_chain_shape(const DmHmat &H, int near_mode);
// one problem of a batched chained H-matvec (device array entry)
struct DmChainProblem {
    DmHmat H;
    const float *x;  // input at step j: x + j xstep (position order when permuted = 1)
    int64_t xstep;
    float *y;        // output
    int permuted, near_mode, near_rows, climb_smem, chain_smem;
};
// y = K~ x for many problems in three launches: map_up[block] = {problem, leaf} (leaf N2S and
// the climb), map_sweep[block] = {problem, subtree} (the top-down sweep of each tree's
// internal levels), then map_near[block] = {problem, near item} (near rows and the leaf S2N).
// Per problem: dm_batch_shape's climbs, sweeps and items; shared memory the largest of the
// problems'. jv[p] selects problem p's input x + jv[p] xstep. In DmChainProblem, near_rows =
// item_rows.
struct DmBatchShape {
    int climbs, sweeps, items, item_rows, climb_smem;
    size_t smem_up, smem_sweep, smem_near;
};
DmBatchShape dm_batch_shape(const DmHmat &H, int near_mode);
cudaError_t dm_hmatvec_batch(const DmChainProblem *P, const int2 *map_up, int n_up, size_t smem_up,
                             const int2 *map_sweep, int n_sweep, size_t smem_sweep, const int2 *map_near, int n_near,
                             size_t smem_near, const int *jv, cudaStream_t st);
cudaError_t dm_hmatvec_chain(const DmHmat &H, int near_mode, const float *x, float *y, bool permuted,
                             cudaStream_t st);
int dm_near_item_rows(int near_mode, int leaf_max);
// write each cluster CTA's shared-memory image of the upper tree (after packing)
cudaError_t dm_tree_image(const DmHmat &H, cudaStream_t st);
// MUFU ex2 throughput kernel: blocks x 256 threads x 8 chains x iters exponentials into out
// (blocks x 256 floats)
cudaError_t dm_launch_ex2_peak(float *out, int blocks, int iters, cudaStream_t st);
// whether the device can run the one-cluster tree pass as a cluster of `ctas` CTAs with the
// largest shared-memory budget (16 needs the non-portable cluster size)
bool dm_tree_cluster_supported(int ctas);

// k_hnb.cu -- H-matvec of a narrow block (2 <= nb <= 4 columns) through the three chained
// launches of the single-vector form, the cluster pass holding nb-wide skeleton vectors
struct DmNbTree {
    int nb;                 // columns (0: not built)
    int ls;                 // cut level of the cluster (2^ls CTAs)
    int smem;               // dynamic shared memory per CTA of the cluster pass (bytes)
    const int4 *lay;        // per node {P, B, pair slot, scratch} offsets (floats) in its owner's image
    const int2 *own;        // per node: offsets of its own w and u (nb-wide rows) in its owner's image
    const int *owner;       // per node: CTA of the cluster that holds it
    float *img;             // per CTA: metadata, operands, vector slots
    const int *img_off;     // 2^ls + 1 image offsets (floats, multiples of 4)
    float *what, *uhat;     // per node max_rank x nb (row t, column c at t nb + c): leaf w in, leaf u out
};
struct DmNbLayout {
    std::vector<int4> lay;
    std::vector<int2> own;
    std::vector<int> owner;
    std::vector<int> img_off;
    int ls = 0, smem = 0;
};
bool dm_nb_tree_layout(const std::vector<int32_t> &rk, int L, int nb, int budget_floats, DmNbLayout &out);
cudaError_t dm_nb_tree_image(const DmHmat &H, const DmNbTree &T, cudaStream_t st);
// Y = K~ X for nb columns (column strides ldx, ldy; original point order unless permuted)
cudaError_t dm_hmatvec_nb(const DmHmat &H, const DmNbTree &T, int nb, const float *x, int64_t ldx, float *y,
                          int64_t ldy, bool permuted, cudaStream_t st);

// k_hblock.cu -- H-matvec of a block of right-hand sides
struct DmBlockWork {
    int nb_max;           // columns per call
    int64_t ldx;          // column stride of the padded leaf layout (nleaves * ldk)
    float *Xb, *Yb;       // nb_max columns of ldx floats each
    float *Wb, *Ub;       // per node max_rank x nb_max (row-major, row stride = the call's nb)
    cudaStream_t side;    // stream of the near-field GEMM (nullptr: the caller's stream)
    cudaEvent_t fork, join;
};
int64_t dm_block_ldx(const DmHmat &H);
// Y = K~ X for nb columns. X: original order with column stride ldin when perm_in = H.perm,
// position order when perm_in = nullptr, or already in the padded leaf layout (x_padded,
// column stride W.ldx). Y (column stride ldo): DM_BLK_ORIGINAL, DM_BLK_POSITION or
// DM_BLK_PADDED (the padded leaf layout).
// near_prec (cached near field): DM_PREC_FP32 on the CUDA cores, DM_PREC_TF32 on the tensor
// cores, DM_PREC_TF32X3 on the tensor cores with three-term split operands.
enum { DM_BLK_PADDED = 0, DM_BLK_ORIGINAL = 1, DM_BLK_POSITION = 2 };
cudaError_t dm_hmatvec_block(const DmHmat &H, int near_mode, int near_prec, const DmBlockWork &W, int nb,
                             const float *x, int64_t ldin, const int32_t *perm_in, bool x_padded, float *y,
                             int64_t ldo, int y_layout, cudaStream_t st);
// k_tc.cu: Yb = K_a Xb per leaf on tcgen05 (TF32 in, FP32 accumulate); *err set when a
// bounded wait gave up. dm_tc_available: the driver provides cuTensorMapEncodeTiled.
bool dm_tc_available();
cudaError_t dm_launch_near_tc(const DmHmat &H, const float *Xb, int64_t ldx, int nb, float *Yb, int *err,
                              bool split, cudaStream_t st);

// k_lanczos.cu
struct DmLanczos {
    int64_t N;
    int64_t ldv;      // column stride of V (N rounded up to 64)
    int m_max;
    float *V;         // (m_max+1) columns
    float *z;         // work vector (ldv, zero padded)
    double *alpha;    // m_max
    double *beta;     // m_max (beta[j] = |r_j|)
    double *h;        // 2 parities x (h0, h1: m_max+1 each; |z'|^2; pad) projection accumulators
    double *nrm2;     // scalar accumulator
    double *theta;    // kmax Ritz values (descending)
    double *resid;    // kmax residual bounds
    double *Y;        // kmax columns of length m_max: eigenvectors of T
    float *Yf;        // m_max x kmax FP32 copy
    double *twork;    // kmax x (6 m_max) doubles for inverse iteration
    double *colsum;   // kmax
    float *phi;       // N x kmax Ritz vectors in position order
    unsigned long long *best;  // kmax
    int *neg;         // kmax
    unsigned *bar;    // grid-barrier counter of the fused step
    int *err;         // set when a bounded device wait gave up
};
int dm_lanczos_kmax();
// one problem of a batched single-vector Lanczos (device array entry): its basis, work vector,
// accumulators (hstride = dm_lanczos_hstride(m_max) per parity), coefficients and Ritz buffers
struct DmLanczosProblem {
    float *V;
    int64_t ldv;
    float *z;
    double *h;
    int hstride;
    double *alpha, *beta;
    int m_max, qt;
    double *theta, *resid;
    int k;  // eigenpairs wanted (Ritz checks)
};
int dm_lanczos_hstride(int m_max);
int dm_step_phased_threads();
int dm_step_tile_quads(int m_max);
// shared memory of one problem's blocks in the batched step (tile of dm_step_tile_quads(m_max))
size_t dm_step_batch_smem(int m_max);
// the three Gram-Schmidt passes of the current step of many problems (three launches), each
// problem at its own step jv[p], which the last pass moves to jv[p] + 1 (arrive[p]: a zeroed
// counter per problem). map[block] = {problem, its block index, its block count, 0}; shm: the
// largest dm_step_batch_smem of the problems
cudaError_t dm_lanczos_step_batch(const DmLanczosProblem *P, const int4 *map, int nblocks, int *jv,
                                  unsigned *arrive, size_t shm, cudaStream_t st);
// Ritz values / residual bounds of the problems act[0..nact) after their jv[p] completed steps
// (k = P[p].k pairs each), one launch; the values also land in theta_out / resid_out
// (kstride = k_hi per slot, slot order) and beta_{m-1} in beta_out; m_hi >= every jv[p]
cudaError_t dm_lanczos_ritz_batch(const DmLanczosProblem *P, const int *act, int nact, const int *jv, int m_hi,
                                  int k_hi, double *theta_out, double *resid_out, double *beta_out, cudaStream_t st);

// Ritz vectors of many finished single-vector problems in six launches (tridiagonal
// eigenvectors, their orthogonalisation, V Y, column maxima, signs, normalised scatter to the
// original point order). map[block] = {problem, its block of 256 positions}: dm_finish_blocks(N)
// blocks per problem; m_hi / k_hi bound the problems' m and k.
struct DmFinish {
    const double *alpha, *beta, *theta;
    double *Y, *twork, *colsum;
    float *Yf, *phi, *evecs;
    const float *V;
    int64_t ldv, N;
    const int32_t *perm;
    unsigned long long *best;
    int *neg;
    int ldy, m, k, pad;
};
int dm_finish_blocks(int64_t N);
// start vectors of many problems (the draws of dm_lanczos_start): h[0..hlen), *nrm2 and *jv zeroed,
// z = uniform(-1, 1) per original index, V[:, 0] = z / |z|; map as for dm_lanczos_finish_batch
struct DmStart {
    const int32_t *perm;
    int64_t N;
    uint64_t key;  // dm_start_key(seed)
    float *z, *V;
    double *nrm2, *h;
    int *jv;  // the problem's step counter, set to 0
    int hlen, pad;
};
uint64_t dm_start_key(uint64_t seed);
cudaError_t dm_lanczos_start_batch(const DmStart *S, int ns, const int2 *map, int nmap, cudaStream_t st);
cudaError_t dm_lanczos_finish_batch(const DmFinish *F, int nf, const int2 *map, int nmap, int m_hi, int k_hi,
                                    cudaStream_t st);

// Single-vector Lanczos of many compressed handles advanced together (dm_eigs_batch and the
// request server). Problems join (dm_batch_add) and leave (on convergence, breakdown or m_max)
// between steps; every step of every active problem runs in the same launches, each problem at
// its own step, and the convergence checks due at a step share one launch and one host read.
struct DmBatchSolver;
struct DmBatchDone {
    dm_handle h = nullptr;
    void *tag = nullptr;
    int status = 0;  // DM_OK (converged or invariant subspace) or DM_ENOCONV (m_max reached)
    int iters = 0, k = 0;
    std::vector<double> theta;    // the k largest Ritz values, descending
    const float *evecs = nullptr;  // device, N x k column-major in original point order
    // the vectors are complete, and the solver done with the handle, when this event has
    // completed (valid until the next dm_batch_step call)
    cudaEvent_t ready = nullptr;
};
DmBatchSolver *dm_batch_create(int device, cudaStream_t st);
void dm_batch_destroy(DmBatchSolver *B);
// room for n problems at once (grows the solver's arrays now rather than while joining)
int dm_batch_reserve(DmBatchSolver *B, int n);
int dm_batch_active(const DmBatchSolver *B);
// on the handle's own stream (call from the thread that runs it): allocate the eigensolver's
// buffers and record *ready (created here; the caller destroys it after dm_batch_add)
int dm_batch_prepare(dm_handle h, cudaEvent_t *ready);
// join: the solver's stream waits for `ready`. The solver works on its own stream only; with
// a non-null `adopt` the handle's own stream becomes `adopt` (a stream of the caller's that
// the handle's later work and dm_destroy's wait use: the caller destroys the handle after
// the DmBatchDone's `ready` event has completed)
int dm_batch_add(DmBatchSolver *B, dm_handle h, int k, void *tag, cudaEvent_t ready, cudaStream_t adopt);
// one step of every stepping problem and the checks due after it. Problems finished are
// appended to `done` one call after their check decided (see DmBatchDone.ready); the solver
// is empty once dm_batch_active returns 0
int dm_batch_step(DmBatchSolver *B, std::vector<DmBatchDone> &done);
cudaError_t dm_launch_barrier_selftest(unsigned *ctr, int *err, int blocks, int missing, long long spin_limit,
                                       cudaStream_t st);
cudaError_t dm_lanczos_start(DmLanczos &Lz, const int32_t *perm, uint64_t seed, cudaStream_t st);
cudaError_t dm_lanczos_orth(DmLanczos &Lz, int j, bool phased, cudaStream_t st);
cudaError_t dm_lanczos_ritz(DmLanczos &Lz, int m, int k, double conv_tol, cudaStream_t st);
cudaError_t dm_lanczos_vectors(DmLanczos &Lz, int m, int k, const int32_t *perm, float *evecs_orig,
                               cudaStream_t st);
// the two halves of dm_lanczos_vectors: eigenvectors of the tridiagonal (Y, FP32 copy Yf),
// then the Ritz vectors V Yf, normalised, signed and scattered to the original order
cudaError_t dm_lanczos_tvecs(DmLanczos &Lz, int m, int k, cudaStream_t st);
cudaError_t dm_lanczos_phi(DmLanczos &Lz, int m, int k, const int32_t *perm, float *evecs_orig, cudaStream_t st);
// thick restart of a dense-T (block) Lanczos: V[:, 0:kr] = normalised V[:, 0:m] Y[:, 0:kr] (Yf of a
// Rayleigh-Ritz step with kr pairs), V[:, kr:kr+b] = V[:, src:src+b], T = diag(theta[0:kr])
cudaError_t dm_lanczos_restart(DmLanczos &Lz, int m, int kr, int src, int b, double *T, int ldT, cudaStream_t st);

// k_blanczos.cu -- block Lanczos (block size b <= dm_block_lanczos_max_b()); the basis lives
// in Lz.V (position order), the Ritz data in Lz.alpha/beta/theta/resid/Y/Yf.
struct DmBlockLanczos {
    int b;
    int nparts, ldpart;   // partial-sum blocks of the projections; ldpart >= m_max + 1
    float *Z;             // b columns of Lz.ldv
    float *part;          // nparts x ldpart x b
    double *H;            // ldpart x b projection coefficients (row-major)
    double *Rinv, *Bacc;  // b x b
    double *T, *W;        // m_max x m_max (column-major): projected matrix, tridiagonalisation work
    double *hb;           // m_max Householder coefficients
    int *flag;            // set when a block lost rank (breakdown)
    double *H1;           // ldpart x b second-pass coefficients of the one-launch step (b <= 4)
    double *Gacc;         // 3 x b x b Gram accumulators of the one-launch step (G1, G2 by parity)
};
int dm_block_lanczos_max_b();
cudaError_t dm_bl_start(DmLanczos &Lz, DmBlockLanczos &B, const int32_t *perm, uint64_t seed, cudaStream_t st);
// the random start block in B.Z (seeded, one key per column), T and the breakdown flag cleared
cudaError_t dm_bl_random_block(DmLanczos &Lz, DmBlockLanczos &B, const int32_t *perm, uint64_t seed,
                               cudaStream_t st);
cudaError_t dm_bl_cholqr(DmLanczos &Lz, DmBlockLanczos &B, int j, bool next_block, cudaStream_t st);
cudaError_t dm_bl_orth(DmLanczos &Lz, DmBlockLanczos &B, int j, cudaStream_t st);
cudaError_t dm_bl_ritz(DmLanczos &Lz, DmBlockLanczos &B, int m, int k, cudaStream_t st);
// k_bstep.cu -- one block-Lanczos step for b <= dm_bstep_max_b() in one cooperative launch of
// `blocks` 512-thread blocks (one per SM): CGS2 of Z against V[:, 0:ncols), CholQR2, the new
// block written to V[:, out:out+b), T(0:ncols, out-b:out) = the projection coefficients,
// Bj = the block's R factor. H0, H1 (ncols x b), G1 (b x b) zero on entry and on return;
// G2 two b x b buffers (the one of parity `par` used, the other cleared); `bar` counts
// arrivals monotonically from bar_base (three barriers of `blocks` arrivals each).
// H0, H1: dm_bstep_hcopies() copies of ncols x b each, `hstride` doubles apart.
int dm_bstep_max_b();
int dm_bstep_hcopies();
cudaError_t dm_bstep(int b, float *V, int64_t ldv, int ncols, int out, const float *Z, double *H0, double *H1,
                     int64_t hstride, double *G1, double *G2, int par, double *T, int ldT, double *Bj, int *flag,
                     unsigned *bar, unsigned bar_base, int *err, int blocks, cudaStream_t st);
cudaError_t dm_launch_coords(const float *evecs, const double *theta, const double *dg, int64_t N, int k, int t,
                             float *psi, cudaStream_t st);

// ---------------------------------------------------------------------------
// CTA-wide exact selection: the k-th smallest (0-based) of n uint64 keys given
// by key(i), by most-significant-digit radix passes (8 bits per pass) with
// warp-aggregated shared-memory histograms. Every thread of the CTA must call
// it; all threads receive the key. `hist` is 256 unsigned of shared memory.
// On return *below holds the number of keys strictly smaller than the result.
// ---------------------------------------------------------------------------
template <class KeyFn>
__device__ uint64_t dm_cta_select(KeyFn key, int64_t n, int64_t k, unsigned *hist, int64_t *below) {
    __shared__ uint64_t s_prefix;
    __shared__ int64_t s_k, s_below;
    __shared__ int64_t s_wsum[8];
    __shared__ int s_bin;
    uint64_t prefix = 0, mask = 0;
    if (threadIdx.x == 0) { s_below = 0; }
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        const int lane = threadIdx.x & 31;
        for (int64_t base = 0; base < n; base += blockDim.x) {
            int64_t i = base + threadIdx.x;
            bool act = false;
            unsigned bin = 0;
            if (i < n) {
                uint64_t u = key(i);
                if ((u & mask) == prefix) { act = true; bin = (unsigned)((u >> shift) & 255u); }
            }
            unsigned am = __ballot_sync(DM_FULL, act);
            if (act) {
                unsigned peers = __match_any_sync(am, bin);
                int leader = __ffs(peers) - 1;
                if (lane == leader) atomicAdd(&hist[bin], (unsigned)__popc(peers));
            }
        }
        __syncthreads();
        // the digit: first bin whose inclusive count exceeds the rank still sought, by a scan
        // of the 256 counts over the first eight warps (blockDim.x >= 256)
        const int64_t kk = (shift == 56) ? k : s_k;
        int64_t h = 0, x = 0;
        if (threadIdx.x < 256) {
            h = (int64_t)hist[threadIdx.x];
            x = h;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(DM_FULL, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) s_wsum[threadIdx.x >> 5] = x;
        }
        if (threadIdx.x == 0) s_bin = 256;
        __syncthreads();
        int64_t excl = 0;
        if (threadIdx.x < 256) {
            int64_t off = 0;
            for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) off += s_wsum[w];
            excl = off + x - h;
            if (off + x > kk) atomicMin(&s_bin, (int)threadIdx.x);
        }
        __syncthreads();
        if ((int)threadIdx.x == s_bin) {
            s_k = kk - excl;
            s_below += excl;
            s_prefix = prefix | ((uint64_t)threadIdx.x << shift);
        }
        __syncthreads();
        prefix = s_prefix;
        mask |= (uint64_t)255 << shift;
        __syncthreads();
    }
    *below = s_below;
    return prefix;
}
