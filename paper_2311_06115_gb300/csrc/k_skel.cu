// k_skel.cu -- skeletonization (sampled interpolative decomposition) and block packing.
//
// The far field of the H-matrix K~ = D + UV (Eq. 2.18) is built from nested
// skeleton bases: for every non-root node a (bottom-up), with candidate columns
// C_a (a leaf's own points, an internal node's children skeletons) and sampled
// off-node rows R_a, an interpolative decomposition K(R_a, C_a) ~= K(R_a, J_a) P_a
// picks the skeleton J_a subset of C_a with P_a(:, J_a) = I. The rank stops at the first
// pivot whose residual column norm is <= tol * (first pivot norm) -- the block-relative
// reading of the tolerance of Eq. 1.1 -- or at max_rank.
//
// GPU design: one CTA per node of a level. The sampled block A = K(R_a, C_a) is stored
// column-major (a candidate column is one contiguous vector of ldr >= r floats) in shared
// memory when it fits (internal levels: at most two children's skeletons), else its leading
// columns there and the rest in a per-CTA slot of global memory; an internal level whose
// blocks do not fit one CTA runs as a cluster of CTAs per node when the clusters fit one
// wave (skel_cluster_kernel: the columns spread over the CTAs' shared memories, the same
// operations in the same order per column). Column-pivoted modified Gram-Schmidt with explicit
// residual updates (each step recomputes every remaining column norm from its updated
// residual, so no norm downdating loses the small residuals that decide the rank) and one
// re-orthogonalisation of the pivot column. A warp owns whole columns: one read-modify-
// write pass per step gives q_k^T a_j (warp reduction), the update a_j -= (q_k^T a_j) q_k
// and the new norm |a_j|, for a few columns at a time so that every lane keeps several
// 16-byte loads in flight; each warp keeps its best remaining column, and every warp finds
// the next pivot itself from those per-warp candidates,
// so a step needs three block barriers. P_a = [I, R11^-1 R12] by back substitution.
#include <cooperative_groups.h>

#include <mutex>

#include "dm_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kSkelThreads = 512;
constexpr int kSkelWarps = kSkelThreads / 32;

__device__ __forceinline__ float kentry(const float *__restrict__ Xp, const float *__restrict__ sp, int d,
                                        int64_t a, int64_t b) {
    const float *xa = Xp + a * d, *xb = Xp + b * d;
    float r2 = 0.f;
    for (int k = 0; k < d; ++k) {
        float t = xa[k] - xb[k];
        r2 = fmaf(t, t, r2);
    }
    return sp[a] * sp[b] * dm_ex2(-r2);
}

struct SkelArgs {
    const float *Xp;  // points in position order, pre-scaled
    const float *sp;  // s in position order
    int64_t N;
    int d, L, level;
    float tol;
    int max_rank, cmax, ldp, rmax, ldr;
    uint64_t seed;
    int32_t *ranks;
    int32_t *skel;
    float *P;
    float *A;   // per-CTA slot cmax x ldr, column-major: A[j][i], j a candidate, i a sampled row
    float *R;   // per-CTA slot max_rank x cmax, row-major
    float *Q;   // per-CTA slot max_rank x ldr: orthonormal pivot columns, one contiguous vector each
    int prefilled;  // 1: A already holds K(R, C) (written by fill_entries_kernel for d > 3)
    int smem_base;  // bytes of the fixed shared-memory layout (16-byte multiple)
    int smem_extra; // dynamic shared memory beyond it: the sampled block when it fits, then rows of Q,
                    // then (after the pivot steps) the triangular solve for P
};

constexpr int kSkelMaxCand = 512;  // candidates per node (leaf points or two children's skeletons)
constexpr int kSkelMaxF4 = 5;      // float4 rows per lane in the column passes: r <= 640

// ---- kernel entries of a block for d > 3, tiled over the coordinates ------------------
// E[r][c] = s_row s_col 2^-|xs_row - xs_col|^2 for up to 32 rows and 32 QN columns per CTA
// (columns z 32 QN + [0, 32 QN) of the block for blockIdx.z = z, so that a level with few
// nodes still fills the GPU). Both point sets are staged through shared memory 32
// coordinates at a time; each thread owns 4 rows x QN columns (columns g + 32 q) of squared
// distances in registers, summed over the coordinates in order exactly as kentry does.
// Work item `mode`: 0 = the sampled block K(R, C) of node (2^level - 1 + blockIdx.x), rows
// drawn exactly as in skel_level_kernel, into its A slot; 1 = the leaf block K(I_a, I_a) of
// leaf blockIdx.x into its Knear slot (zero padded); 2 = the sibling block
// B_p = K(S_l, S_r) of internal node p = blockIdx.x (rows the left child's skeleton, columns
// the right child's), row-major s_l x s_r at B + p max_rank^2.
constexpr int kFillRows = 32;
constexpr int kFillK = 32;

template <int QN>
__global__ void __launch_bounds__(256, QN <= 8 ? 4 : 1) fill_entries_kernel(SkelArgs a, int mode, float *__restrict__ Knear,
                                                           int leaf_max, int ldk) {
    constexpr int kCols = 32 * QN;
    extern __shared__ float fsm[];
    float *xr = fsm;                                  // kFillRows x (kFillK + 1)
    float *xc = xr + kFillRows * (kFillK + 1);         // kCols x (kFillK + 1)
    int *rowpos = reinterpret_cast<int *>(xc + kCols * (kFillK + 1));  // kFillRows
    int *colpos = rowpos + kFillRows;                 // kCols
    __shared__ int s_c, s_r;
    const int tid = threadIdx.x;
    const int node = mode == 0 ? (1 << a.level) - 1 + (int)blockIdx.x
                     : mode == 1 ? (1 << a.L) - 1 + (int)blockIdx.x : (int)blockIdx.x;
    int64_t st, sz;
    dm_node_range(a.N, node, &st, &sz);
    const int t0 = blockIdx.y * kFillRows;
    const int j0 = (int)blockIdx.z * kCols;  // first column of this CTA's tile
    if (tid == 0) {
        if (mode == 2) {
            s_r = a.ranks[2 * node + 1];
            s_c = a.ranks[2 * node + 2];
        } else if (mode == 0) {
            const int64_t off = a.N - sz;
            const int rtarget = 2 * a.max_rank + 10;
            s_r = (int)(off <= rtarget ? off : rtarget);
            s_c = a.level == a.L ? (int)sz : a.ranks[2 * node + 1] + a.ranks[2 * node + 2];
        } else {
            s_r = (int)sz;
            s_c = (int)sz;
        }
    }
    __syncthreads();
    const int r = s_r, c_all = s_c;
    // the host sizes QN and the column tiles to the columns; the near blocks (mode 1) also
    // write the zero padding of rows up to leaf_max and columns up to ldk
    if (c_all > (int)gridDim.z * kCols || (t0 >= r && !(mode == 1 && t0 < leaf_max))) return;
    if (mode != 1 && j0 >= c_all) return;
    const int c = c_all - j0 < kCols ? (c_all - j0 > 0 ? c_all - j0 : 0) : kCols;  // this tile's columns
    // row and column positions
    if (tid < kFillRows) {
        const int t = t0 + tid;
        int pos = -1;
        if (t < r) {
            if (mode == 2) {
                pos = a.skel[(int64_t)(2 * node + 1) * a.max_rank + t];
            } else if (mode == 0) {
                const int64_t off = a.N - sz;
                const int rtarget = 2 * a.max_rank + 10;
                const uint64_t key = dm_stream_key(a.seed, DM_TAG_ROWS, (uint64_t)node);
                const int64_t u = (off <= rtarget) ? (int64_t)t : (int64_t)dm_below(dm_rng(key, (uint64_t)t), (uint64_t)off);
                pos = (int)(u < st ? u : u + sz);
            } else {
                pos = (int)(st + t);
            }
        }
        rowpos[tid] = pos;
    }
    for (int jt = tid; jt < c; jt += blockDim.x) {
        const int j = j0 + jt;
        int pos;
        if (mode == 2) pos = a.skel[(int64_t)(2 * node + 2) * a.max_rank + j];
        else if (mode == 1 || a.level == a.L) pos = (int)(st + j);
        else {
            const int l = 2 * node + 1, rr = 2 * node + 2, sl = a.ranks[l];
            pos = j < sl ? a.skel[(int64_t)l * a.max_rank + j] : a.skel[(int64_t)rr * a.max_rank + (j - sl)];
        }
        colpos[jt] = pos;
    }
    __syncthreads();
    const int rg = tid & 7, cg = tid >> 3;  // rows 4 rg .. 4 rg + 3; tile columns cg + 32 q
    float acc[4][QN];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < QN; ++q) acc[i][q] = 0.f;
    const int d = a.d;
    for (int k0 = 0; k0 < d; k0 += kFillK) {
        __syncthreads();
        for (int e = tid; e < kFillRows * kFillK; e += blockDim.x) {
            const int i = e / kFillK, k = e - i * kFillK;
            const int pos = rowpos[i];
            xr[i * (kFillK + 1) + k] = (pos >= 0 && k0 + k < d) ? a.Xp[(int64_t)pos * d + k0 + k] : 0.f;
        }
        for (int e = tid; e < c * kFillK; e += blockDim.x) {
            const int j = e / kFillK, k = e - j * kFillK;
            xc[j * (kFillK + 1) + k] = (k0 + k < d) ? a.Xp[(int64_t)colpos[j] * d + k0 + k] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < kFillK; ++k) {
            float xv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) xv[i] = xr[(4 * rg + i) * (kFillK + 1) + k];
#pragma unroll
            for (int q = 0; q < QN; ++q) {
                const float cv = xc[(cg + 32 * q) * (kFillK + 1) + k];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float t = xv[i] - cv;
                    acc[i][q] = fmaf(t, t, acc[i][q]);
                }
            }
        }
    }
    // entries, written with zero padding
    if (mode == 2) {
        float *Bn = Knear + (size_t)blockIdx.x * a.max_rank * a.max_rank;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int t = t0 + 4 * rg + i;
            if (t >= r) continue;
            const float si = a.sp[rowpos[4 * rg + i]];
#pragma unroll
            for (int q = 0; q < QN; ++q) {
                const int jt = cg + 32 * q;
                if (jt < c) Bn[(size_t)t * c_all + j0 + jt] = si * a.sp[colpos[jt]] * dm_ex2(-acc[i][q]);
            }
        }
        return;
    }
    if (mode == 0) {
        // column-major: the thread's four consecutive rows of column j are one 16-byte store;
        // rows from r up to the next multiple of four are written as zeros
        const int tq = t0 + 4 * rg;
        if (tq < r) {
            float si[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) si[i] = rowpos[4 * rg + i] >= 0 ? a.sp[rowpos[4 * rg + i]] : 0.f;
            float *slot = a.A + (size_t)blockIdx.x * a.cmax * a.ldr;
#pragma unroll
            for (int q = 0; q < QN; ++q) {
                const int jt = cg + 32 * q;
                if (jt >= c) continue;
                const float sj = a.sp[colpos[jt]];
                float v[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) v[i] = rowpos[4 * rg + i] >= 0 ? si[i] * sj * dm_ex2(-acc[i][q]) : 0.f;
                *reinterpret_cast<float4 *>(slot + (size_t)(j0 + jt) * a.ldr + tq) = make_float4(v[0], v[1], v[2], v[3]);
            }
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int t = t0 + 4 * rg + i;
        const int pos = rowpos[4 * rg + i];
        if (t >= leaf_max) continue;
        float *out = Knear + ((size_t)blockIdx.x * leaf_max + t) * ldk;
        const float si = pos >= 0 ? a.sp[pos] : 0.f;
#pragma unroll
        for (int q = 0; q < QN; ++q) {
            const int jt = cg + 32 * q, j = j0 + jt;
            if (j < ldk) out[j] = (pos >= 0 && jt < c) ? si * a.sp[colpos[jt]] * dm_ex2(-acc[i][q]) : 0.f;
        }
    }
}

__device__ __forceinline__ float dot4(float4 a, float4 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w))); }
__device__ __forceinline__ float4 scale4(float4 a, float s) { return make_float4(a.x * s, a.y * s, a.z * s, a.w * s); }
__device__ __forceinline__ float warp_allsum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(DM_FULL, v, o);
    return v;
}

// One pass over a batch of CB of the warp's columns: stored column l = warp + kSkelWarps (b CB + u)
// (l < cn) is candidate j = g0 + gs l (all candidates: g0 = 0, gs = 1; one CTA of a cluster:
// its share g0 + gs l). d_j = q^T a_j, a_j -= d_j q, R(k, j) = d_j, and the lane's running best
// (|a_j|, j) for the next pivot (lowest index on ties). Lane holds float4 rows
// f = lane + 32 m, m < M, of each column (f < nf), as two packed FP32x2 halves. q = qv * inv,
// recomputed from shared memory at each use (the same product every time).
template <int M, int CB>
__device__ __forceinline__ void column_batch(float *At, int ncs, float *Ag, int ldr, int nf, int cn, int g0, int gs,
                                             int b, const float4 *qv, float inv, const int *selpos, float &best_v,
                                             int &best_j, float *Rk) {
    // stored column l lives at At + l ldr for l < ncs (shared memory), else at Ag + l ldr
    auto colp = [&](int l) { return (l < ncs ? At : Ag) + (size_t)l * ldr; };
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int jl[CB], jb[CB];
    bool ok[CB];
#pragma unroll
    for (int u = 0; u < CB; ++u) {
        jl[u] = warp + kSkelWarps * (b * CB + u);
        jb[u] = g0 + gs * jl[u];
        ok[u] = jl[u] < cn && selpos[jb[u]] < 0;
    }
    float4 v[CB][M];
#pragma unroll
    for (int u = 0; u < CB; ++u) {
        const float4 *col = reinterpret_cast<const float4 *>(colp(jl[u]));
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int f = lane + 32 * m;
            v[u][m] = (ok[u] && f < nf) ? col[f] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    float2 dp[CB];
#pragma unroll
    for (int u = 0; u < CB; ++u) dp[u] = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int f = lane + 32 * m;
        const float4 q = f < nf ? scale4(qv[f], inv) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float2 qa = make_float2(q.x, q.y), qb = make_float2(q.z, q.w);
#pragma unroll
        for (int u = 0; u < CB; ++u) {
            dp[u] = __ffma2_rn(make_float2(v[u][m].x, v[u][m].y), qa, dp[u]);
            dp[u] = __ffma2_rn(make_float2(v[u][m].z, v[u][m].w), qb, dp[u]);
        }
    }
    float dj[CB];
#pragma unroll
    for (int u = 0; u < CB; ++u) dj[u] = warp_allsum(dp[u].x + dp[u].y);
    float2 sp2[CB];
#pragma unroll
    for (int u = 0; u < CB; ++u) sp2[u] = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int f = lane + 32 * m;
        if (f >= nf) continue;
        const float4 q = scale4(qv[f], inv);
        const float2 qa = make_float2(q.x, q.y), qb = make_float2(q.z, q.w);
#pragma unroll
        for (int u = 0; u < CB; ++u) {
            if (!ok[u]) continue;
            const float2 nd = make_float2(-dj[u], -dj[u]);
            const float2 wa = __ffma2_rn(nd, qa, make_float2(v[u][m].x, v[u][m].y));
            const float2 wb = __ffma2_rn(nd, qb, make_float2(v[u][m].z, v[u][m].w));
            reinterpret_cast<float4 *>(colp(jl[u]))[f] = make_float4(wa.x, wa.y, wb.x, wb.y);
            sp2[u] = __ffma2_rn(wa, wa, sp2[u]);
            sp2[u] = __ffma2_rn(wb, wb, sp2[u]);
        }
    }
    // lane u finishes column u: one square root for the batch
    float my_ss = 0.f, my_d = 0.f;
    int my_j = -1;
#pragma unroll
    for (int u = 0; u < CB; ++u) {
        const float t = warp_allsum(sp2[u].x + sp2[u].y);
        if (lane == u && ok[u]) {
            my_ss = t;
            my_d = dj[u];
            my_j = jb[u];
        }
    }
    if (my_j >= 0) {
        const float nv = sqrtf(my_ss);
        if (nv > best_v || (nv == best_v && my_j < best_j)) {
            best_v = nv;
            best_j = my_j;
        }
        Rk[my_j] = my_d;
    }
}

// largest (value, lowest index on ties) over the warp; every lane gets the result
__device__ __forceinline__ void warp_argmax(float &v, int &j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(DM_FULL, v, o);
        const int oj = __shfl_xor_sync(DM_FULL, j, o);
        if (ov > v || (ov == v && oj < j)) {
            v = ov;
            j = oj;
        }
    }
}

// P = [I, R11^-1 R12] in candidate order (rows t < rank of the node's slot), the node's
// skeleton and rank, from R (max_rank x cmax, global) and the pivot order; every thread of
// the CTA calls it. xs: `extra` floats of shared memory no longer in use.
__device__ void skel_write_p(const SkelArgs &a, int node, int c, int rank, const int *selpos, const int *piv,
                             const int *C, const float *R, float *xs, size_t extra) {
    float *Pn = a.P + (size_t)node * a.max_rank * a.ldp;
    const int ldas = (c + 3) & ~3;
    if ((size_t)rank * ldas + (size_t)rank * rank <= extra) {
        // in shared memory (A and Q are dead): Rs = R(0:rank, :) and a compact copy
        // R11[t][u] = R(t, piv[u]); each unselected column is solved in place, in the same
        // operation order as the global-memory form below; then coalesced row stores with the
        // identity columns
        float *Rs = xs, *R11 = xs + (size_t)rank * ldas;
        for (int e = threadIdx.x; e < rank * ldas; e += blockDim.x) {
            const int t = e / ldas, j = e - t * ldas;
            Rs[e] = j < c ? R[(size_t)t * a.cmax + j] : 0.f;
        }
        for (int e = threadIdx.x; e < rank * rank; e += blockDim.x) {
            const int t = e / rank, u = e - t * rank;
            R11[e] = R[(size_t)t * a.cmax + piv[u]];
        }
        __syncthreads();
        for (int j = threadIdx.x; j < c; j += blockDim.x) {
            if (selpos[j] >= 0) continue;
            for (int t = rank - 1; t >= 0; --t) {
                const float *r11 = R11 + (size_t)t * rank;
                float v = Rs[(size_t)t * ldas + j];
                for (int u = t + 1; u < rank; ++u) v = fmaf(-r11[u], Rs[(size_t)u * ldas + j], v);
                Rs[(size_t)t * ldas + j] = v / r11[t];
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < rank * c; e += blockDim.x) {
            const int t = e / c, j = e - t * c;
            const int sp_ = selpos[j];
            Pn[(size_t)t * a.ldp + j] = sp_ >= 0 ? (t == sp_ ? 1.f : 0.f) : Rs[(size_t)t * ldas + j];
        }
    } else for (int j = threadIdx.x; j < c; j += blockDim.x) {
        const int sp_ = selpos[j];
        if (sp_ >= 0) {
            for (int t = 0; t < rank; ++t) Pn[(size_t)t * a.ldp + j] = (t == sp_) ? 1.f : 0.f;
        } else {
            for (int t = rank - 1; t >= 0; --t) {
                float v = R[(size_t)t * a.cmax + j];
                for (int u = t + 1; u < rank; ++u) v = fmaf(-R[(size_t)t * a.cmax + piv[u]], Pn[(size_t)u * a.ldp + j], v);
                Pn[(size_t)t * a.ldp + j] = v / R[(size_t)t * a.cmax + piv[t]];
            }
        }
    }
    // zero the row padding so vectorised readers may overrun c up to ldp
    for (int t = 0; t < rank; ++t)
        for (int j = c + threadIdx.x; j < a.ldp; j += blockDim.x) Pn[(size_t)t * a.ldp + j] = 0.f;
    for (int t = threadIdx.x; t < a.max_rank; t += blockDim.x)
        a.skel[(int64_t)node * a.max_rank + t] = t < rank ? C[piv[t]] : -1;
    if (threadIdx.x == 0) a.ranks[node] = rank;
}

template <int M, int CB>
__global__ void __launch_bounds__(kSkelThreads, 2) skel_level_kernel(SkelArgs a) {
    // float4-accessed arrays first so that every one starts on a 16-byte boundary
    extern __shared__ float4 smem4[];
    float4 *qv4 = smem4;                                 // ldr / 4 (ldr a multiple of 4): pivot residual (then v)
    float4 *ccrd = qv4 + (a.ldr >> 2);                   // cmax: candidate coordinates (d <= 3) and s
    float *xr = reinterpret_cast<float *>(ccrd + a.cmax); // 4 x ldr: row x, y, z, s (d <= 3), one array each
    float *coef = xr + 4 * a.ldr;                        // max_rank: re-orthogonalisation coefficients
    int *C = reinterpret_cast<int *>(coef + a.max_rank); // cmax candidate positions
    int *Rw = C + a.cmax;                                // rmax row positions
    int *selpos = Rw + a.rmax;                           // cmax: -1 or pivot step
    int *piv = selpos + a.cmax;                          // max_rank
    __shared__ float wred[kSkelWarps];
    __shared__ float wbest_v[kSkelWarps];  // each warp's best remaining column norm and its index
    __shared__ int wbest_j[kSkelWarps];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int node = (1 << a.level) - 1 + (int)blockIdx.x;
    int64_t st, sz;
    dm_node_range(a.N, node, &st, &sz);
    float *R = a.R + (size_t)blockIdx.x * a.max_rank * a.cmax;
    float *Q = a.Q + (size_t)blockIdx.x * a.max_rank * a.ldr;

    // ---- candidates
    int c;
    if (a.level == a.L) {
        c = (int)sz;
        for (int j = threadIdx.x; j < c; j += blockDim.x) C[j] = (int)(st + j);
    } else {
        const int l = 2 * node + 1, r = 2 * node + 2;
        const int sl = a.ranks[l], sr = a.ranks[r];
        c = sl + sr;
        for (int j = threadIdx.x; j < c; j += blockDim.x)
            C[j] = j < sl ? a.skel[(int64_t)l * a.max_rank + j] : a.skel[(int64_t)r * a.max_rank + (j - sl)];
    }
    // ---- rows: every off-node position if few enough, else seeded draws with replacement
    const int64_t off = a.N - sz;
    const int rtarget = 2 * a.max_rank + 10;
    const int r = (int)(off <= rtarget ? off : rtarget);
    const uint64_t key = dm_stream_key(a.seed, DM_TAG_ROWS, (uint64_t)node);
    const bool small_d = a.d <= 3;
    for (int t = threadIdx.x; t < r; t += blockDim.x) {
        int64_t u = (off <= rtarget) ? (int64_t)t : (int64_t)dm_below(dm_rng(key, (uint64_t)t), (uint64_t)off);
        const int pos = (int)(u < st ? u : u + sz);
        Rw[t] = pos;
        if (small_d) {
            for (int k = 0; k < 3; ++k) xr[k * a.ldr + t] = k < a.d ? a.Xp[(int64_t)pos * a.d + k] : 0.f;
            xr[3 * a.ldr + t] = a.sp[pos];
        }
    }
    for (int j = threadIdx.x; j < c; j += blockDim.x) {
        selpos[j] = -1;
        if (small_d && !a.prefilled) {
            const int64_t cj = C[j];
            float4 v = make_float4(0.f, 0.f, 0.f, a.sp[cj]);
            if (a.d > 0) v.x = a.Xp[cj * a.d];
            if (a.d > 1) v.y = a.Xp[cj * a.d + 1];
            if (a.d > 2) v.z = a.Xp[cj * a.d + 2];
            ccrd[j] = v;
        }
    }
    // the sampled block lives in shared memory when it fits (internal levels: few candidates),
    // and rows of Q follow it there while they fit; a larger block keeps its leading columns
    // in shared memory (after min(kmax, 32) rows of Q) and the rest in the CTA's global slot
    const int nf = (r + 3) >> 2;  // float4 rows per column
    const int ldr = a.ldr;
    float *Ag = a.A + (size_t)blockIdx.x * a.cmax * ldr;
    const size_t extra = a.smem_extra > 0 ? (size_t)a.smem_extra / sizeof(float) : 0;  // floats
    float *xs = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(smem4) + a.smem_base);
    int kmax = a.max_rank;
    if (kmax > c) kmax = c;
    if (kmax > r) kmax = r;
    const int slots = (int)(extra / (size_t)ldr);  // columns or Q rows that fit in shared memory
    const int qkeep = kmax < 32 ? kmax : 32;
    const int ncs = c <= slots ? c : (slots > qkeep ? slots - qkeep : 0);
    float *Qs = xs + (size_t)ncs * ldr;
    int qcap = slots - ncs;
    if (qcap > a.max_rank) qcap = a.max_rank;
    auto colp = [&](int j) { return (j < ncs ? xs : Ag) + (size_t)j * ldr; };
    auto qrow = [&](int t) -> float4 * {
        return reinterpret_cast<float4 *>(t < qcap ? Qs + (size_t)t * ldr : Q + (size_t)t * ldr);
    };
    __syncthreads();

    // ---- sampled block A = K(R, C) (rows r..4 nf - 1 zero) and its column norms: warp per column;
    // warp w owns columns w, w + warps, ... here and in every column pass
    float best_v = -1.f;
    int best_j = 0x7fffffff;
    for (int j = warp; j < c; j += kSkelWarps) {
        float4 *col = reinterpret_cast<float4 *>(colp(j));
        float ss = 0.f;
        if (a.prefilled) {
            const float4 *src = reinterpret_cast<const float4 *>(Ag + (size_t)j * ldr);
            for (int f = lane; f < nf; f += 32) {
                const float4 v = src[f];
                if (j < ncs) col[f] = v;
                ss += dot4(v, v);
            }
        } else {
            const int64_t cj = C[j];
            float sj = 0.f, cx[3] = {0.f, 0.f, 0.f};
            if (small_d) {
                const float4 cc = ccrd[j];
                cx[0] = cc.x;
                cx[1] = cc.y;
                cx[2] = cc.z;
                sj = cc.w;
            }
            for (int f = lane; f < nf; f += 32) {
                float v[4];
                if (small_d) {
                    // rows 4f..4f+3 of each coordinate array: 16-byte loads, consecutive across lanes
                    const float4 rx = reinterpret_cast<const float4 *>(xr)[f];
                    const float4 ry = reinterpret_cast<const float4 *>(xr + ldr)[f];
                    const float4 rz = reinterpret_cast<const float4 *>(xr + 2 * ldr)[f];
                    const float4 rs = reinterpret_cast<const float4 *>(xr + 3 * ldr)[f];
                    const float px[4] = {rx.x, rx.y, rx.z, rx.w}, py[4] = {ry.x, ry.y, ry.z, ry.w},
                                pz[4] = {rz.x, rz.y, rz.z, rz.w}, ps[4] = {rs.x, rs.y, rs.z, rs.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float t0 = cx[0] - px[u], t1 = cx[1] - py[u], t2 = cx[2] - pz[u];
                        v[u] = (4 * f + u < r) ? ps[u] * sj * dm_ex2(-fmaf(t0, t0, fmaf(t1, t1, t2 * t2))) : 0.f;
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < 4; ++u) v[u] = (4 * f + u < r) ? kentry(a.Xp, a.sp, a.d, Rw[4 * f + u], cj) : 0.f;
                }
                const float4 w = make_float4(v[0], v[1], v[2], v[3]);
                col[f] = w;
                ss += dot4(w, w);
            }
        }
        ss = warp_allsum(ss);
        const float nv = sqrtf(ss);
        if (nv > best_v || (nv == best_v && j < best_j)) {
            best_v = nv;
            best_j = j;
        }
    }
    if (lane == 0) {
        wbest_v[warp] = best_v;
        wbest_j[warp] = best_j;
    }
    __syncthreads();

    const int nw = (nf + 31) >> 5;  // warps that own the pivot column's float4 rows
    const int nb = (((c + kSkelWarps - 1) / kSkelWarps) + CB - 1) / CB;  // column batches per warp
    int rank = 0;
    float nrm0 = 0.f;
    for (int k = 0; k < kmax; ++k) {
        // ---- pivot: largest residual norm among unselected columns, lowest index on ties
        // (every warp reduces the same per-warp candidates, so all agree without a barrier)
        float bv = lane < kSkelWarps ? wbest_v[lane] : -1.f;
        int bi = lane < kSkelWarps ? wbest_j[lane] : 0x7fffffff;
        warp_argmax(bv, bi);
        if (k == 0) nrm0 = bv;
        if (!(bv > a.tol * nrm0) || bv <= 0.f) break;
        const int p = bi;
        // ---- the pivot column, re-orthogonalised once against q_0..q_{k-1}: coefficients
        // q_t^T a_p, t = warp, warp + warps, ...
        float4 ap[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int f = lane + 32 * m;
            ap[m] = f < nf ? reinterpret_cast<const float4 *>(colp(p))[f] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int t = warp; t < k; t += kSkelWarps) {
            const float4 *qt = t < qcap ? reinterpret_cast<const float4 *>(Qs + (size_t)t * ldr)
                                        : reinterpret_cast<const float4 *>(Q + (size_t)t * ldr);
            float d = 0.f;
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const int f = lane + 32 * m;
                if (f < nf) d += dot4(qt[f], ap[m]);
            }
            d = warp_allsum(d);
            if (lane == 0) coef[t] = d;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            selpos[p] = k;
            piv[k] = p;
        }
        // fire-and-forget reductions: nothing waits on a global read before the barrier
        for (int t = threadIdx.x; t < k; t += blockDim.x) atomicAdd(R + (size_t)t * a.cmax + p, coef[t]);
        // ---- v = a_p - sum_t coef_t q_t on the warps that own its rows, |v|^2 partials
        if (warp < nw) {
            const int f = warp * 32 + lane;
            float4 v = ap[0];
#pragma unroll
            for (int m = 1; m < M; ++m)
                if (warp == m) v = ap[m];
            float ss = 0.f;
            if (f < nf) {
                auto sub = [&](const float4 qt, float ct) {
                    v.x = fmaf(-ct, qt.x, v.x);
                    v.y = fmaf(-ct, qt.y, v.y);
                    v.z = fmaf(-ct, qt.z, v.z);
                    v.w = fmaf(-ct, qt.w, v.w);
                };
                const int kq = k < qcap ? k : qcap;
                for (int t = 0; t < kq; ++t) sub(reinterpret_cast<const float4 *>(Qs + (size_t)t * ldr)[f], coef[t]);
                for (int t = kq; t < k; ++t) sub(reinterpret_cast<const float4 *>(Q + (size_t)t * ldr)[f], coef[t]);
                qv4[f] = v;
                ss = dot4(v, v);
            }
            ss = warp_allsum(ss);
            if (lane == 0) wred[warp] = ss;
        }
        __syncthreads();
        // ---- q_k = v / |v| (each thread forms the norm from the warp partials in one order)
        float ssv = 0.f;
        for (int w = 0; w < nw; ++w) ssv += wred[w];
        const float qn = sqrtf(ssv);
        const float inv = 1.f / qn;
        if (threadIdx.x == 0) R[(size_t)k * a.cmax + p] = qn;
        if (warp < nw) {
            const int f = warp * 32 + lane;
            if (f < nf) qrow(k)[f] = scale4(qv4[f], inv);
        }
        // ---- every other remaining column: R(k, j) = q_k^T a_j, a_j -= R(k, j) q_k, |a_j|
        float cv = -1.f;
        int cj = 0x7fffffff;
        for (int b = 0; b < nb; ++b)
            column_batch<M, CB>(xs, ncs, Ag, ldr, nf, c, 0, 1, b, qv4, inv, selpos, cv, cj, R + (size_t)k * a.cmax);
        warp_argmax(cv, cj);
        if (lane == 0) {
            wbest_v[warp] = cv;
            wbest_j[warp] = cj;
        }
        rank = k + 1;
        __syncthreads();
    }
    __syncthreads();

    skel_write_p(a, node, c, rank, selpos, piv, C, R, xs, extra);
}

// ---- Clustered form, for sampled blocks larger than one CTA's shared memory.
// A cluster of G CTAs per node (G = the cluster size) splits the candidates: CTA g keeps the
// columns j = g + G l, l < ceil(c / G), of the sampled block in its own shared memory, so the
// column passes stay on the SM, and its own copy of the leading rows of Q (rows past qcap in
// the node's global Q slot, written by CTA 0). A pivot step: every warp's best remaining
// column is published in its CTA's shared memory; one cluster barrier; every warp reads the
// G x 16 candidates and takes the same pivot (largest norm, lowest index on ties); the pivot
// column is copied from its owner's shared memory; each CTA re-orthogonalises it against its
// own Q copy and forms q_k with the same operations in the same order as the others (the same
// q_k everywhere, without a second exchange), then updates its own columns. The owner of the
// pivot records R(:, p); CTA 0 forms P after a final cluster barrier. Every CTA of a cluster
// takes the same decisions from the same data, so all reach every cluster barrier.
template <int M, int CB>
__global__ void __launch_bounds__(kSkelThreads, 1) skel_cluster_kernel(SkelArgs a) {
    cg::cluster_group cl = cg::this_cluster();
    const int G = (int)cl.num_blocks();
    const int g = (int)cl.block_rank();
    extern __shared__ float4 smem4[];
    float4 *qv4 = smem4;                                 // ldr / 4: the pivot column, then v
    float4 *ccrd = qv4 + (a.ldr >> 2);                   // cmax: candidate coordinates (d <= 3) and s
    float *xr = reinterpret_cast<float *>(ccrd + a.cmax); // 4 x ldr: row x, y, z, s (d <= 3)
    float *coef = xr + 4 * a.ldr;                        // max_rank
    int *C = reinterpret_cast<int *>(coef + a.max_rank); // cmax
    int *Rw = C + a.cmax;                                // rmax
    int *selpos = Rw + a.rmax;                           // cmax
    int *piv = selpos + a.cmax;                          // max_rank
    __shared__ float wred[kSkelWarps];
    __shared__ float wbest_v[2][kSkelWarps];  // per step parity: each warp's best column (read cluster-wide)
    __shared__ int wbest_j[2][kSkelWarps];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nl = (int)blockIdx.x / G;  // node within the level
    const int node = (1 << a.level) - 1 + nl;
    int64_t st, sz;
    dm_node_range(a.N, node, &st, &sz);
    float *R = a.R + (size_t)nl * a.max_rank * a.cmax;
    float *Q = a.Q + (size_t)nl * a.max_rank * a.ldr;

    int c;
    if (a.level == a.L) {
        c = (int)sz;
        for (int j = threadIdx.x; j < c; j += blockDim.x) C[j] = (int)(st + j);
    } else {
        const int l = 2 * node + 1, r = 2 * node + 2;
        const int sl = a.ranks[l], sr = a.ranks[r];
        c = sl + sr;
        for (int j = threadIdx.x; j < c; j += blockDim.x)
            C[j] = j < sl ? a.skel[(int64_t)l * a.max_rank + j] : a.skel[(int64_t)r * a.max_rank + (j - sl)];
    }
    const int64_t off = a.N - sz;
    const int rtarget = 2 * a.max_rank + 10;
    const int r = (int)(off <= rtarget ? off : rtarget);
    const uint64_t key = dm_stream_key(a.seed, DM_TAG_ROWS, (uint64_t)node);
    const bool small_d = a.d <= 3;
    for (int t = threadIdx.x; t < r; t += blockDim.x) {
        int64_t u = (off <= rtarget) ? (int64_t)t : (int64_t)dm_below(dm_rng(key, (uint64_t)t), (uint64_t)off);
        const int pos = (int)(u < st ? u : u + sz);
        Rw[t] = pos;
        if (small_d) {
            for (int k = 0; k < 3; ++k) xr[k * a.ldr + t] = k < a.d ? a.Xp[(int64_t)pos * a.d + k] : 0.f;
            xr[3 * a.ldr + t] = a.sp[pos];
        }
    }
    for (int j = threadIdx.x; j < c; j += blockDim.x) {
        selpos[j] = -1;
        if (small_d && !a.prefilled) {
            const int64_t cj = C[j];
            float4 v = make_float4(0.f, 0.f, 0.f, a.sp[cj]);
            if (a.d > 0) v.x = a.Xp[cj * a.d];
            if (a.d > 1) v.y = a.Xp[cj * a.d + 1];
            if (a.d > 2) v.z = a.Xp[cj * a.d + 2];
            ccrd[j] = v;
        }
    }
    // this CTA's columns; the share size (and so qcap) is the same in every CTA of the cluster
    const int cn = c > g ? (c - g + G - 1) / G : 0;
    const int cshare = (c + G - 1) / G;
    const int nf = (r + 3) >> 2;
    const int ldr = a.ldr;
    const float *Ag = a.A + (size_t)nl * a.cmax * ldr;
    const size_t extra = a.smem_extra > 0 ? (size_t)a.smem_extra / sizeof(float) : 0;
    float *xs = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(smem4) + a.smem_base);
    float *At = xs;  // the host sizes the launch so that the share always fits
    float *Qs = xs + (size_t)cshare * ldr;
    int qcap = (int)((extra - (size_t)cshare * ldr) / (size_t)ldr);
    if (qcap > a.max_rank) qcap = a.max_rank;
    __syncthreads();

    // ---- this CTA's columns of the sampled block and their norms (warp per column)
    float best_v = -1.f;
    int best_j = 0x7fffffff;
    for (int jl = warp; jl < cn; jl += kSkelWarps) {
        const int j = g + G * jl;
        float4 *col = reinterpret_cast<float4 *>(At + (size_t)jl * ldr);
        float ss = 0.f;
        if (a.prefilled) {
            const float4 *src = reinterpret_cast<const float4 *>(Ag + (size_t)j * ldr);
            for (int f = lane; f < nf; f += 32) {
                const float4 v = src[f];
                col[f] = v;
                ss += dot4(v, v);
            }
        } else {
            const int64_t cj = C[j];
            float sj = 0.f, cx[3] = {0.f, 0.f, 0.f};
            if (small_d) {
                const float4 cc = ccrd[j];
                cx[0] = cc.x;
                cx[1] = cc.y;
                cx[2] = cc.z;
                sj = cc.w;
            }
            for (int f = lane; f < nf; f += 32) {
                float v[4];
                if (small_d) {
                    const float4 rx = reinterpret_cast<const float4 *>(xr)[f];
                    const float4 ry = reinterpret_cast<const float4 *>(xr + ldr)[f];
                    const float4 rz = reinterpret_cast<const float4 *>(xr + 2 * ldr)[f];
                    const float4 rs = reinterpret_cast<const float4 *>(xr + 3 * ldr)[f];
                    const float px[4] = {rx.x, rx.y, rx.z, rx.w}, py[4] = {ry.x, ry.y, ry.z, ry.w},
                                pz[4] = {rz.x, rz.y, rz.z, rz.w}, ps[4] = {rs.x, rs.y, rs.z, rs.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float t0 = cx[0] - px[u], t1 = cx[1] - py[u], t2 = cx[2] - pz[u];
                        v[u] = (4 * f + u < r) ? ps[u] * sj * dm_ex2(-fmaf(t0, t0, fmaf(t1, t1, t2 * t2))) : 0.f;
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < 4; ++u) v[u] = (4 * f + u < r) ? kentry(a.Xp, a.sp, a.d, Rw[4 * f + u], cj) : 0.f;
                }
                const float4 w = make_float4(v[0], v[1], v[2], v[3]);
                col[f] = w;
                ss += dot4(w, w);
            }
        }
        ss = warp_allsum(ss);
        const float nv = sqrtf(ss);
        if (nv > best_v || (nv == best_v && j < best_j)) {
            best_v = nv;
            best_j = j;
        }
    }
    if (lane == 0) {
        wbest_v[0][warp] = best_v;
        wbest_j[0][warp] = best_j;
    }

    int kmax = a.max_rank;
    if (kmax > c) kmax = c;
    if (kmax > r) kmax = r;
    const int nw = (nf + 31) >> 5;  // warps that own the pivot column's float4 rows
    const int nb = (((cn + kSkelWarps - 1) / kSkelWarps) + CB - 1) / CB;  // column batches per warp
    int rank = 0;
    float nrm0 = 0.f;
    for (int k = 0; k < kmax; ++k) {
        // candidates of step k published in slot k & 1 of every CTA (the barrier also orders
        // this CTA's previous column pass before the reuse of qv4 below)
        cl.sync();
        float bv = -1.f;
        int bi = 0x7fffffff;
        for (int e = lane; e < G * kSkelWarps; e += 32) {
            const int rr = e / kSkelWarps, w = e - rr * kSkelWarps;
            const float v = *cl.map_shared_rank(&wbest_v[k & 1][w], rr);
            const int j = *cl.map_shared_rank(&wbest_j[k & 1][w], rr);
            if (v > bv || (v == bv && j < bi)) {
                bv = v;
                bi = j;
            }
        }
        warp_argmax(bv, bi);
        if (k == 0) nrm0 = bv;
        if (!(bv > a.tol * nrm0) || bv <= 0.f) break;
        const int p = bi, owner = p % G;
        // the pivot column from its owner's share (no CTA writes a selected column again)
        {
            const float4 *src =
                reinterpret_cast<const float4 *>(cl.map_shared_rank(At + (size_t)(p / G) * ldr, owner));
            for (int f = threadIdx.x; f < nf; f += blockDim.x) qv4[f] = src[f];
        }
        __syncthreads();
        float4 ap[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int f = lane + 32 * m;
            ap[m] = f < nf ? qv4[f] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int t = warp; t < k; t += kSkelWarps) {
            const float4 *qt = t < qcap ? reinterpret_cast<const float4 *>(Qs + (size_t)t * ldr)
                                        : reinterpret_cast<const float4 *>(Q + (size_t)t * ldr);
            float d = 0.f;
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const int f = lane + 32 * m;
                if (f < nf) d += dot4(qt[f], ap[m]);
            }
            d = warp_allsum(d);
            if (lane == 0) coef[t] = d;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            selpos[p] = k;
            piv[k] = p;
        }
        if (g == owner)
            for (int t = threadIdx.x; t < k; t += blockDim.x) atomicAdd(R + (size_t)t * a.cmax + p, coef[t]);
        if (warp < nw) {
            const int f = warp * 32 + lane;
            float4 v = ap[0];
#pragma unroll
            for (int m = 1; m < M; ++m)
                if (warp == m) v = ap[m];
            float ss = 0.f;
            if (f < nf) {
                auto sub = [&](const float4 qt, float ct) {
                    v.x = fmaf(-ct, qt.x, v.x);
                    v.y = fmaf(-ct, qt.y, v.y);
                    v.z = fmaf(-ct, qt.z, v.z);
                    v.w = fmaf(-ct, qt.w, v.w);
                };
                const int kq = k < qcap ? k : qcap;
                for (int t = 0; t < kq; ++t) sub(reinterpret_cast<const float4 *>(Qs + (size_t)t * ldr)[f], coef[t]);
                for (int t = kq; t < k; ++t) sub(reinterpret_cast<const float4 *>(Q + (size_t)t * ldr)[f], coef[t]);
                qv4[f] = v;
                ss = dot4(v, v);
            }
            ss = warp_allsum(ss);
            if (lane == 0) wred[warp] = ss;
        }
        __syncthreads();
        float ssv = 0.f;
        for (int w = 0; w < nw; ++w) ssv += wred[w];
        const float qn = sqrtf(ssv);
        const float inv = 1.f / qn;
        if (g == owner && threadIdx.x == 0) R[(size_t)k * a.cmax + p] = qn;
        if (warp < nw) {
            const int f = warp * 32 + lane;
            if (f < nf) {
                const float4 q = scale4(qv4[f], inv);
                if (k < qcap) reinterpret_cast<float4 *>(Qs + (size_t)k * ldr)[f] = q;
                else if (g == 0) reinterpret_cast<float4 *>(Q + (size_t)k * ldr)[f] = q;
            }
        }
        // ---- this CTA's remaining columns
        float cv = -1.f;
        int cj = 0x7fffffff;
        for (int b = 0; b < nb; ++b)
            column_batch<M, CB>(At, cn, At, ldr, nf, cn, g, G, b, qv4, inv, selpos, cv, cj, R + (size_t)k * a.cmax);
        warp_argmax(cv, cj);
        if (lane == 0) {
            wbest_v[(k + 1) & 1][warp] = cv;
            wbest_j[(k + 1) & 1][warp] = cj;
        }
        rank = k + 1;
    }
    // R complete in global memory, and no CTA reads another's shared memory after this barrier
    __threadfence();
    cl.sync();
    if (g != 0) return;
    skel_write_p(a, node, c, rank, selpos, piv, C, R, xs, extra);
}

// ---- near blocks K(I_a, I_a), row-major with leading dimension ldk, zero padded (d <= 3: the
// leaf's points and s are staged in shared memory; a thread per column, rows of the CTA's slice)
__global__ void pack_near_kernel(const float *__restrict__ Xp, const float *__restrict__ sp, int64_t N, int d, int L,
                                 int leaf_max, int ldk, float *__restrict__ Knear) {
    extern __shared__ float4 pts[];  // leaf_max: x, y, z, s
    const int leaf = blockIdx.x;
    int64_t st, sz;
    dm_node_range(N, (1 << L) - 1 + leaf, &st, &sz);
    if (d > 3) {  // generic dimension: entries straight from the point arrays
        float *blk = Knear + (size_t)leaf * leaf_max * ldk;
        const int rows_per = (leaf_max + gridDim.y - 1) / gridDim.y;
        const int r0 = blockIdx.y * rows_per, r1 = min(leaf_max, r0 + rows_per);
        for (int i = r0; i < r1; ++i)
            for (int j = threadIdx.x; j < ldk; j += blockDim.x)
                blk[(size_t)i * ldk + j] = (i < sz && j < sz) ? kentry(Xp, sp, d, st + i, st + j) : 0.f;
        return;
    }
    for (int j = threadIdx.x; j < (int)sz; j += blockDim.x) {
        const int64_t g = st + j;
        float4 v = make_float4(0.f, 0.f, 0.f, sp[g]);
        if (d > 0) v.x = Xp[g * d];
        if (d > 1) v.y = Xp[g * d + 1];
        if (d > 2) v.z = Xp[g * d + 2];
        pts[j] = v;
    }
    __syncthreads();
    float *blk = Knear + (size_t)leaf * leaf_max * ldk;
    const int rows_per = (leaf_max + gridDim.y - 1) / gridDim.y;
    const int r0 = blockIdx.y * rows_per;
    const int r1 = min(leaf_max, r0 + rows_per);
    for (int j = threadIdx.x; j < ldk; j += blockDim.x) {
        const bool cj = j < sz;
        const float4 pj = cj ? pts[j] : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i = r0; i < r1; ++i) {
            float v = 0.f;
            if (i < sz && cj) {
                const float4 pi = pts[i];  // broadcast
                const float t0 = pi.x - pj.x, t1 = pi.y - pj.y, t2 = pi.z - pj.z;
                v = pi.w * pj.w * dm_ex2(-fmaf(t2, t2, fmaf(t1, t1, t0 * t0)));
            }
            blk[(size_t)i * ldk + j] = v;
        }
    }
}

// ---- far blocks B_p = K(S_l, S_r) for the children of every internal node, row-major s_l x s_r
// (d <= 3, where an entry is a few flops; larger d goes through the coordinate-tiled fill)
__global__ void pack_far_kernel(const float *__restrict__ Xp, const float *__restrict__ sp, int d,
                                const int32_t *__restrict__ ranks, const int32_t *__restrict__ skel, int max_rank,
                                float *__restrict__ B) {
    const int node = blockIdx.x;
    const int l = 2 * node + 1, r = 2 * node + 2;
    const int sl = ranks[l], sr = ranks[r];
    float *Bn = B + (size_t)node * max_rank * max_rank;
    for (int e = threadIdx.x; e < sl * sr; e += blockDim.x) {
        const int ia = e / sr, ib = e % sr;
        Bn[e] = kentry(Xp, sp, d, skel[(int64_t)l * max_rank + ia], skel[(int64_t)r * max_rank + ib]);
    }
}

// PT[leaf][i][t] = P_leaf[t][i] (t < rank, zero up to ldt), the point-major copy the
// downward pass reads with contiguous 16-byte loads. Slices of 32 points go through a padded
// shared tile, so both the reads of P's rows and the writes of PT's rows are coalesced.
constexpr int kTrPts = 32;
constexpr int kTrMaxT = 256;  // ldt <= max_rank <= 256
__global__ void __launch_bounds__(256) transpose_leaf_kernel(DmHmat H, float *__restrict__ PT) {
    __shared__ float tile[kTrMaxT][kTrPts + 1];
    const int leaf = blockIdx.x;
    const int node = (1 << H.L) - 1 + leaf;
    int64_t st, sz;
    dm_node_range(H.N, node, &st, &sz);
    const int s = H.ranks[node];
    const int ldt = H.pt_ld[leaf];  // this leaf's row stride (its rank rounded up to 4)
    const float *Pn = H.P + (size_t)node * H.max_rank * H.ldp;
    float *out = PT + H.pt_off[leaf];
    // blockIdx.y picks the CTA's slices (one each when the grid covers the leaf)
    for (int i0 = (int)blockIdx.y * kTrPts; i0 < (int)sz; i0 += (int)gridDim.y * kTrPts) {
        const int np = (int)sz - i0 < kTrPts ? (int)sz - i0 : kTrPts;
        __syncthreads();
        for (int e = threadIdx.x; e < ldt * kTrPts; e += blockDim.x) {
            const int t = e / kTrPts, ii = e - t * kTrPts;
            tile[t][ii] = (t < s && ii < np) ? Pn[(size_t)t * H.ldp + i0 + ii] : 0.f;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < np * ldt; e += blockDim.x) {
            const int ii = e / ldt, t = e - ii * ldt;
            out[(size_t)(i0 + ii) * ldt + t] = tile[t][ii];
        }
    }
}

__global__ void permute_points_kernel(const float *__restrict__ Xs, const float *__restrict__ sf,
                                      const int32_t *__restrict__ perm, int64_t N, int d, float *__restrict__ Xp,
                                      float *__restrict__ sp) {
    int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (pos >= N) return;
    const int64_t i = perm[pos];
    for (int k = 0; k < d; ++k) Xp[pos * d + k] = Xs[i * d + k];
    sp[pos] = sf[i];
}

}  // namespace

namespace {

size_t fill_smem_bytes(int qn) {
    return sizeof(float) * (size_t)(kFillRows + 32 * qn) * (kFillK + 1) + sizeof(int) * (size_t)(kFillRows + 32 * qn);
}

template <int QN>
cudaError_t launch_fill_qn(dim3 grid, const SkelArgs &a, int mode, float *out, int leaf_max, int ldk, cudaStream_t st) {
    const size_t sm = fill_smem_bytes(QN);
    cudaError_t e = dm_allow_smem((const void *)fill_entries_kernel<QN>, sm);
    if (e != cudaSuccess) return e;
    fill_entries_kernel<QN><<<grid, 256, sm, st>>>(a, mode, out, leaf_max, ldk);
    dm_count_launches(1);
    return cudaGetLastError();
}

// grids (nodes x row tiles) below this many CTAs (two per SM) split their columns
constexpr unsigned kFillMinCtas = 2 * 152;

// The entry fill for blocks of up to `cols` columns: the fewest column groups per thread that
// cover them in one tile; a small grid (the upper tree levels, where one CTA per row tile
// would run its whole block alone on an SM) splits the columns into tiles of 64 (QN = 2,
// blockIdx.z).
cudaError_t launch_fill(int cols, dim3 grid, const SkelArgs &a, int mode, float *out, int leaf_max, int ldk,
                        cudaStream_t st) {
    if (cols > kSkelMaxCand || cols < 1) return cudaErrorInvalidValue;
    int qn = cols <= 128 ? 4 : cols <= 256 ? 8 : 16;
    if (grid.x * grid.y < kFillMinCtas) qn = 2;
    grid.z = (unsigned)((cols + 32 * qn - 1) / (32 * qn));
    switch (qn) {
        case 2: return launch_fill_qn<2>(grid, a, mode, out, leaf_max, ldk, st);
        case 4: return launch_fill_qn<4>(grid, a, mode, out, leaf_max, ldk, st);
        case 8: return launch_fill_qn<8>(grid, a, mode, out, leaf_max, ldk, st);
        default: return launch_fill_qn<16>(grid, a, mode, out, leaf_max, ldk, st);
    }
}

// The clustered ID runs an internal level whose sampled blocks may not fit one CTA's shared
// memory when its clusters fit one wave (nodes x G <= SMs): a cluster holds G SMs for the
// whole level, so it only pays where one CTA per node would leave SMs idle; the leaf level
// (many nodes, two CTAs per SM streaming their blocks through L2) keeps one CTA per node.
constexpr int kSkelClusterMaxG = 8;       // portable cluster size
constexpr int kSkelClusterMinQRows = 64;  // fewest Q rows a CTA keeps in shared memory (else all)

template <int M, int CB>
cudaError_t launch_skel_cluster(const SkelArgs &a, unsigned nodes, int G, size_t smem, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nodes * (unsigned)G);
    cfg.blockDim = dim3(kSkelThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = (unsigned)G;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, skel_cluster_kernel<M, CB>, a);
}

// how many clusters of G CTAs of `kern` with `smem` bytes each can be resident at once (0: none;
// cached per kernel, G and shared-memory size; one device per process in practice)
int skel_cluster_capacity(const void *kern, int G, size_t smem) {
    static std::mutex mu;
    static std::vector<std::pair<std::pair<const void *, int>, std::pair<size_t, int>>> seen;
    std::lock_guard<std::mutex> lk(mu);
    for (auto &e : seen)
        if (e.first.first == kern && e.first.second == G && e.second.first == smem) return e.second.second;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)G);
    cfg.blockDim = dim3(kSkelThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = (unsigned)G;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) n = 0;
    cudaGetLastError();
    seen.push_back({{kern, G}, {smem, n}});
    return n;
}

}  // namespace

size_t dm_skel_smem_bytes(int cmax, int rmax, int max_rank) {
    const size_t ldr = (size_t)((rmax + 3) & ~3);
    return sizeof(float) * ldr + sizeof(float) * (size_t)(4 * cmax + 4 * ldr + max_rank) +
           sizeof(int) * (size_t)(cmax + rmax + cmax + max_rank);
}

int dm_skel_max_candidates() { return kSkelMaxCand; }

cudaError_t dm_skeletonize(const float *Xp, const float *sp, int64_t N, int d, int L, const int32_t *perm,
                           double tol, int max_rank, int cmax, int ldp, uint64_t seed, int32_t *ranks,
                           int32_t *skel, float *P, DmSkelWork *w, cudaStream_t st) {
    (void)perm;
    SkelArgs a;
    a.Xp = Xp;
    a.sp = sp;
    a.N = N;
    a.d = d;
    a.L = L;
    a.tol = (float)tol;
    a.max_rank = max_rank;
    a.cmax = cmax;
    a.ldp = ldp;
    a.rmax = w->rmax;
    a.seed = seed;
    a.ranks = ranks;
    a.skel = skel;
    a.P = P;
    a.A = w->A;
    a.R = w->R;
    a.Q = w->Q;
    a.ldr = w->ldr;
    if (cmax > kSkelMaxCand || (w->ldr & 3) != 0 || w->ldr < w->rmax || w->rmax > 4 * 32 * kSkelMaxF4)
        return cudaErrorInvalidValue;
    const size_t smem = dm_skel_smem_bytes(cmax, w->rmax, max_rank);
    // float4 rows per lane: three (r <= 384, the default ranks) with three-column batches,
    // else five (r <= 640) with two
    const bool wide = w->rmax > 32 * 4 * 3;
    const void *kern = wide ? (const void *)skel_level_kernel<5, 2> : (const void *)skel_level_kernel<3, 3>;
    cudaError_t e = dm_allow_smem(kern, smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(ranks, 0, sizeof(int32_t), st);  // the root has no skeleton
    if (e != cudaSuccess) return e;
    a.prefilled = d > 3 ? 1 : 0;
    a.smem_base = (int)((smem + 15) & ~(size_t)15);
    int optin = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
    // dynamic bytes allowed = per-block opt-in limit minus the kernel's static shared memory
    const size_t dyn_max = ((size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0) & ~(size_t)15;
    const size_t smem_int = dyn_max > (size_t)a.smem_base ? dyn_max : smem;
    if ((e = dm_allow_smem(kern, smem_int)) != cudaSuccess) return e;
    // the leaf level (many CTAs) takes what still lets two CTAs share an SM (its register
    // footprint allows two), which holds the Q rows of the ranks seen in practice
    int sm_bytes = 0, reserved = 0;
    cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    const size_t half = (size_t)sm_bytes / 2;
    size_t smem_leaf = half > (size_t)reserved + fa.sharedSizeBytes ? (half - reserved - fa.sharedSizeBytes) & ~(size_t)15 : 0;
    if (smem_leaf > smem_int) smem_leaf = smem_int;
    if (smem_leaf < (size_t)a.smem_base) smem_leaf = smem;
    // the clustered form: its whole opt-in shared memory per CTA
    const void *ckern = wide ? (const void *)skel_cluster_kernel<5, 2> : (const void *)skel_cluster_kernel<3, 3>;
    cudaFuncAttributes fc;
    if ((e = cudaFuncGetAttributes(&fc, ckern)) != cudaSuccess) return e;
    const size_t smem_cl = ((size_t)optin > fc.sharedSizeBytes ? (size_t)optin - fc.sharedSizeBytes : 0) & ~(size_t)15;
    const bool cl_usable = smem_cl > (size_t)a.smem_base && dm_allow_smem(ckern, smem_cl) == cudaSuccess;
    cudaGetLastError();
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t colb = sizeof(float) * (size_t)w->ldr;  // one stored column of the block, one row of Q
    const int leaf_pts = (int)((N + (1ll << L) - 1) >> L);
    for (int lvl = L; lvl >= 1; --lvl) {
        a.level = lvl;
        if (a.prefilled) {
            // rows: at most 2 max_rank + 10 sampled; columns: the candidates, at most cmax
            const int rt = 2 * max_rank + 10;
            const dim3 grid(1u << lvl, (unsigned)((rt + kFillRows - 1) / kFillRows));
            if ((e = launch_fill(cmax, grid, a, 0, nullptr, 0, 0, st)) != cudaSuccess) return e;
        }
        // internal levels (few candidates per node, at most one CTA per SM) take the whole
        // shared memory, which holds the sampled block and Q
        const size_t lsm = lvl < L ? smem_int : smem_leaf;
        // candidates per node at this level: at most a leaf's points, or two children's ranks
        const int cb = lvl == L ? leaf_pts : (cmax < 2 * max_rank ? cmax : 2 * max_rank);
        int G = 0;
        if (cl_usable && lvl < L && (size_t)cb * colb > lsm - (size_t)a.smem_base) {
            // the smallest one-wave cluster (every cluster co-resident) whose CTAs hold their
            // share of the block and every row of Q, else the smallest that holds
            // kSkelClusterMinQRows of them
            const int kall = max_rank < cb ? max_rank : cb;
            const int kmin = kall < kSkelClusterMinQRows ? kall : kSkelClusterMinQRows;
            for (int pass = 0; pass < 2 && !G; ++pass) {
                const int kq = pass == 0 ? kall : kmin;
                for (int gg = 2; gg <= kSkelClusterMaxG && !G; gg *= 2) {
                    const size_t need = (size_t)((cb + gg - 1) / gg) * colb + (size_t)kq * colb;
                    if ((1ll << lvl) * gg <= nsm && need <= smem_cl - (size_t)a.smem_base &&
                        skel_cluster_capacity(ckern, gg, smem_cl) >= (1 << lvl))
                        G = gg;
                }
            }
        }
        if (G) {
            a.smem_extra = (int)(smem_cl - (size_t)a.smem_base);
            e = wide ? launch_skel_cluster<5, 2>(a, 1u << lvl, G, smem_cl, st)
                     : launch_skel_cluster<3, 3>(a, 1u << lvl, G, smem_cl, st);
        } else {
            a.smem_extra = lsm > (size_t)a.smem_base ? (int)(lsm - (size_t)a.smem_base) : 0;
            if (wide) skel_level_kernel<5, 2><<<1 << lvl, kSkelThreads, lsm, st>>>(a);
            else skel_level_kernel<3, 3><<<1 << lvl, kSkelThreads, lsm, st>>>(a);
            e = cudaGetLastError();
        }
        dm_count_launches(1);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t dm_pack(const DmHmat &H, float *Knear, float *B, bool pack_near, cudaStream_t st) {
    // d > 3: the coordinate-tiled entry fill (near blocks when the leaf fits one CTA's columns,
    // and the sibling blocks); d <= 3: the direct kernels below
    SkelArgs a{};
    a.Xp = H.Xs;
    a.sp = H.sp;
    a.N = H.N;
    a.d = H.d;
    a.L = H.L;
    a.max_rank = H.max_rank;
    a.ranks = const_cast<int32_t *>(H.ranks);  // read only
    a.skel = const_cast<int32_t *>(H.skel);
    const int near_cols = H.ldk > H.leaf_max ? H.ldk : H.leaf_max;
    cudaError_t e = cudaSuccess;
    if (pack_near && H.d > 3 && near_cols <= kSkelMaxCand) {
        const dim3 grid(1u << H.L, (unsigned)((H.leaf_max + kFillRows - 1) / kFillRows));
        if ((e = launch_fill(near_cols, grid, a, 1, Knear, H.leaf_max, H.ldk, st)) != cudaSuccess) return e;
    } else if (pack_near) {
        dim3 grid(1u << H.L, (unsigned)((H.leaf_max + 31) / 32));
        pack_near_kernel<<<grid, 128, sizeof(float4) * (size_t)H.leaf_max, st>>>(H.Xs, H.sp, H.N, H.d, H.L,
                                                                                  H.leaf_max, H.ldk, Knear);
        dm_count_launches(1);
    }
    if (H.L > 0 && H.d > 3 && H.max_rank <= kSkelMaxCand) {
        const dim3 grid((1u << H.L) - 1, (unsigned)((H.max_rank + kFillRows - 1) / kFillRows));
        if ((e = launch_fill(H.max_rank, grid, a, 2, B, 0, 0, st)) != cudaSuccess) return e;
    } else if (H.L > 0) {
        pack_far_kernel<<<(1 << H.L) - 1, 256, 0, st>>>(H.Xs, H.sp, H.d, H.ranks, H.skel, H.max_rank, B);
        dm_count_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t dm_transpose_leaf_bases(const DmHmat &H, float *PT, cudaStream_t st) {
    if (H.ldt > kTrMaxT) return cudaErrorInvalidValue;
    const dim3 grid(1u << H.L, (unsigned)((H.leaf_max + kTrPts - 1) / kTrPts));
    transpose_leaf_kernel<<<grid, 256, 0, st>>>(H, PT);
    dm_count_launches(1);
    return cudaGetLastError();
}

cudaError_t dm_permute_points(const float *Xs, const float *sf, const int32_t *perm, int64_t N, int d, float *Xp,
                              float *sp, cudaStream_t st) {
    permute_points_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(Xs, sf, perm, N, d, Xp, sp);
    dm_count_launches(1);
    return cudaGetLastError();
}
