// k_hmatvec.cu -- the hierarchical matvec y = K~ x of Eq. 2.18 (K~ = D + UV), chained
// form: used when the upper tree's skeleton vectors do not fit the shared memory of the
// cluster pass in k_htree.cu (very deep trees at high ranks).
//
//   near (D):  y~(I_a) = K(I_a, I_a) x~(I_a)                      every leaf a
//   N2S  (V):  w_a = P_a x~(I_a) (leaf),  w_a = P_a [w_l; w_r] (internal)
//   S2S  (UV): u_l = K(S_l, S_r) w_r,  u_r = K(S_l, S_r)^T w_l   every sibling pair
//   S2N  (U):  [u_l; u_r] += P_a^T u_a (internal),  y~(I_a) += P_a^T u_a (leaf)
//
// Two launches per right-hand side:
//  1. near_up_kernel: blocks [0, nleaves) do a leaf's N2S and then climb the tree
//     by "last arrival": each block that finishes a node bumps its parent's
//     counter with release semantics; the block that arrives second owns the
//     parent, runs the pair's S2S and the parent's N2S and climbs on. No block
//     ever waits, so there is no spin loop. The remaining blocks stream the leaf
//     blocks (cached: K(I_a, I_a) from HBM with 16-byte evict-first loads;
//     on the fly: entries recomputed from the staged points with MUFU ex2) and
//     write the near-field result, overlapping the latency-bound climb.
//  2. down_kernel: one block per leaf walks its ancestor chain top-down
//     (u_total = P_parent(:, child)^T u_total + u_child), applies P_leaf^T and
//     writes y = y~_near + y~_far, scattering back to the original point order.
#include "dm_internal.cuh"

namespace {

constexpr int kHThreads = 256;
constexpr int kDownThreads = 128;
constexpr int kDownSplit = 2;  // blocks per leaf in the downward pass
constexpr int kHWarps = kHThreads / 32;
constexpr int kCachedItemsPerLeaf = 4;  // near items (row ranges) per leaf block (cached)

__device__ __forceinline__ float4 ldcs4(const float *p) { return __ldcs(reinterpret_cast<const float4 *>(p)); }

// stage x~(I_a) (length m, zero padded to m4) into shared memory
__device__ __forceinline__ void stage_x(const DmHmat &H, const float *__restrict__ x, bool permuted, int64_t st,
                                        int m, int m4, float *sx) {
    for (int j = threadIdx.x; j < m4; j += blockDim.x) {
        float v = 0.f;
        if (j < m) v = permuted ? x[st + j] : x[H.perm[st + j]];
        sx[j] = v;
    }
}

// out[t] = P[t, 0:c] . v for t < s (warp per row; P rows zero padded to a multiple of 4)
__device__ __forceinline__ void gemv_rows(const float *__restrict__ P, int ldp, int s, int c, const float *v,
                                          float *out_global, float *out_smem) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c4 = (c + 3) >> 2;
    for (int t = warp; t < s; t += kHWarps) {
        const float4 *row = reinterpret_cast<const float4 *>(P + (size_t)t * ldp);
        float acc = 0.f;
        for (int q = lane; q < c4; q += 32) {
            float4 p = __ldg(row + q);
            float4 xv = *reinterpret_cast<const float4 *>(v + 4 * q);
            acc = fmaf(p.x, xv.x, acc);
            acc = fmaf(p.y, xv.y, acc);
            acc = fmaf(p.z, xv.z, acc);
            acc = fmaf(p.w, xv.w, acc);
        }
        acc = dm_warp_sum(acc);
        if (lane == 0) {
            if (out_global) out_global[t] = acc;
            if (out_smem) out_smem[t] = acc;
        }
    }
}

// out[t] = P[t, 0:c] . v for t < s, P in global memory (rows zero padded to a multiple of 4):
// a warp takes two rows at a time and issues all 16-byte loads of both rows (up to 512
// columns) before any arithmetic, so one memory round trip serves a pair of rows.
__device__ __forceinline__ void gemv2_rows_global(const float *__restrict__ P, int ldp, int s, int c, const float *v,
                                                  float *out_global) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c4 = (c + 3) >> 2;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 *v4 = reinterpret_cast<const float4 *>(v);
    for (int t = 2 * warp; t < s; t += 2 * kHWarps) {
        const bool two = t + 1 < s;
        const float4 *ra = reinterpret_cast<const float4 *>(P + (size_t)t * ldp);
        const float4 *rb = reinterpret_cast<const float4 *>(P + (size_t)(two ? t + 1 : t) * ldp);
        float acc_a = 0.f, acc_b = 0.f;
        for (int base = 0; base < c4; base += 128) {
            float4 ka[4], kb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q = base + lane + 32 * u;
                ka[u] = q < c4 ? __ldg(ra + q) : zero;
                kb[u] = (two && q < c4) ? __ldg(rb + q) : zero;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q = base + lane + 32 * u;
                const float4 xv = q < c4 ? v4[q] : zero;
                acc_a = fmaf(ka[u].x, xv.x, fmaf(ka[u].y, xv.y, fmaf(ka[u].z, xv.z, fmaf(ka[u].w, xv.w, acc_a))));
                acc_b = fmaf(kb[u].x, xv.x, fmaf(kb[u].y, xv.y, fmaf(kb[u].z, xv.z, fmaf(kb[u].w, xv.w, acc_b))));
            }
        }
        acc_a = dm_warp_sum(acc_a);
        acc_b = dm_warp_sum(acc_b);
        if (lane == 0) {
            out_global[t] = acc_a;
            if (two) out_global[t + 1] = acc_b;
        }
    }
}

// Leaf N2S, out[t] = P[t, 0:m] . v for t < s (rows zero padded to a multiple of 4): four
// threads per row and 64 rows per pass of the block, each thread with up to eight 16-byte loads
// in flight before its sums, so that a leaf's basis arrives in one or two memory round trips.
__device__ __forceinline__ void gemv_leaf(const float *__restrict__ P, int ldp, int s, int m, const float *v,
                                          float *out_global) {
    const int g = threadIdx.x & 3, row = threadIdx.x >> 2;
    const int q4 = (m + 3) >> 2;
    const float4 *v4 = reinterpret_cast<const float4 *>(v);
    for (int t0 = 0; t0 < s; t0 += kHThreads / 4) {
        const int t = t0 + row;
        const bool live = t < s;
        const float4 *pr = reinterpret_cast<const float4 *>(P + (size_t)(live ? t : 0) * ldp);
        float acc = 0.f;
        for (int base = g; base < q4; base += 32) {
            float4 pv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int q = base + 4 * u;
                pv[u] = (live && q < q4) ? __ldg(pr + q) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int q = base + 4 * u;
                if (q < q4) {
                    const float4 xv = v4[q];
                    acc = fmaf(pv[u].x, xv.x, fmaf(pv[u].y, xv.y, fmaf(pv[u].z, xv.z, fmaf(pv[u].w, xv.w, acc))));
                }
            }
        }
        acc += __shfl_xor_sync(DM_FULL, acc, 1);
        acc += __shfl_xor_sync(DM_FULL, acc, 2);
        if (live && g == 0) out_global[t] = acc;
    }
}

// out[t] = P[t, 0:c] . v for t < s from a shared-memory copy of P with row stride ld4 (multiple of 4)
__device__ __forceinline__ void gemv_rows_smem(const float *Ps, int ld4, int s, int c, const float *v, float *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c4 = (c + 3) >> 2;
    for (int t = warp; t < s; t += kHWarps) {
        const float4 *row = reinterpret_cast<const float4 *>(Ps + (size_t)t * ld4);
        float acc = 0.f;
        for (int q = lane; q < c4; q += 32) {
            const float4 p = row[q];
            const float4 xv = *reinterpret_cast<const float4 *>(v + 4 * q);
            acc = fmaf(p.x, xv.x, acc);
            acc = fmaf(p.y, xv.y, acc);
            acc = fmaf(p.z, xv.z, acc);
            acc = fmaf(p.w, xv.w, acc);
        }
        acc = dm_warp_sum(acc);
        if (lane == 0) out[t] = acc;
    }
}

// Top-down S2N of the internal levels, in the batched form (sweep_batch_kernel): after the
// climb every node's u holds its S2S part; its total incoming far-field vector is
// t_node = u_node + P_parent(:, node's columns)^T t_parent (level 1: u itself). A block owns
// the subtree under one node q of level lq: it forms t_q along q's ancestor chain in shared
// memory (reading the ancestors' u, writing none of them), stores t_q over u_q, then the
// levels below q down to L-1 in place, a warp per node. The leaves' totals are formed by
// their near items.
__device__ __forceinline__ void sweep_subtree(const DmHmat &H, int q, int lq, float *ta, float *tb, float *part) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int R = H.max_rank, RH4 = (H.rank_hi + 3) & ~3;
    {
        const int a1 = ((q + 1) >> (lq - 1)) - 1;  // q's ancestor at level 1
        for (int j = threadIdx.x; j < H.ranks[a1]; j += blockDim.x) ta[j] = __ldcg(H.uhat + (size_t)a1 * R + j);
        __syncthreads();
    }
    // the chain, levels 2..lq: two halves of the parent's rank over the two halves of the block
    const int half = threadIdx.x >> 7, jj = threadIdx.x & 127;
    for (int lvl = 2; lvl <= lq; ++lvl) {
        const int v = ((q + 1) >> (lq - lvl)) - 1, par = (v - 1) >> 1;
        const int sc = H.ranks[v], sp = H.ranks[par];
        const int off = (v == 2 * par + 2) ? H.ranks[2 * par + 1] : 0;
        const float *Pn = H.P + (size_t)par * R * H.ldp + off;
        const int th = (sp + 1) >> 1, t0 = half * th, t1 = min(sp, t0 + th);
        for (int j = jj; j < sc; j += 128) {
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
            int t = t0;
            for (; t + 4 <= t1; t += 4) {
                a0 = fmaf(__ldg(Pn + (size_t)t * H.ldp + j), ta[t], a0);
                a1 = fmaf(__ldg(Pn + (size_t)(t + 1) * H.ldp + j), ta[t + 1], a1);
                a2 = fmaf(__ldg(Pn + (size_t)(t + 2) * H.ldp + j), ta[t + 2], a2);
                a3 = fmaf(__ldg(Pn + (size_t)(t + 3) * H.ldp + j), ta[t + 3], a3);
            }
            for (; t < t1; ++t) a0 = fmaf(__ldg(Pn + (size_t)t * H.ldp + j), ta[t], a0);
            part[half * RH4 + j] = (a0 + a1) + (a2 + a3);
        }
        __syncthreads();
        for (int j = threadIdx.x; j < sc; j += blockDim.x)
            tb[j] = __ldcg(H.uhat + (size_t)v * R + j) + (part[j] + part[RH4 + j]);
        __syncthreads();
        float *tmp = ta;
        ta = tb;
        tb = tmp;
    }
    for (int j = threadIdx.x; j < H.ranks[q]; j += blockDim.x) __stcg(H.uhat + (size_t)q * R + j, ta[j]);
    __syncthreads();
    // the subtree's internal levels below q
    for (int lvl = lq + 1; lvl < H.L; ++lvl) {
        const int first = ((q + 1) << (lvl - lq)) - 1, count = 1 << (lvl - lq);
        for (int i = warp; i < count; i += kHWarps) {
            const int nd = first + i, par = (nd - 1) >> 1;
            const int sc = H.ranks[nd], sp = H.ranks[par];
            const int off = (nd == 2 * par + 2) ? H.ranks[2 * par + 1] : 0;
            const float *Pn = H.P + (size_t)par * R * H.ldp + off;
            const float *tp = H.uhat + (size_t)par * R;
            float *un = H.uhat + (size_t)nd * R;
            for (int j = lane; j < sc; j += 32) {
                float a0 = __ldcg(un + j), a1 = 0.f, a2 = 0.f, a3 = 0.f;
                int t = 0;
                for (; t + 4 <= sp; t += 4) {
                    a0 = fmaf(__ldg(Pn + (size_t)t * H.ldp + j), __ldcg(tp + t), a0);
                    a1 = fmaf(__ldg(Pn + (size_t)(t + 1) * H.ldp + j), __ldcg(tp + t + 1), a1);
                    a2 = fmaf(__ldg(Pn + (size_t)(t + 2) * H.ldp + j), __ldcg(tp + t + 2), a2);
                    a3 = fmaf(__ldg(Pn + (size_t)(t + 3) * H.ldp + j), __ldcg(tp + t + 3), a3);
                }
                for (; t < sp; ++t) a0 = fmaf(__ldg(Pn + (size_t)t * H.ldp + j), __ldcg(tp + t), a0);
                __stcg(un + j, (a0 + a1) + (a2 + a3));
            }
        }
        __syncthreads();  // this level's totals are the next level's parents
    }
}

// The climb by last arrival (see the file header) from `node`, whose weights this block has
// written: count the arrival at the parent; the second block to arrive owns the parent, runs
// the pair's S2S and the parent's N2S, and climbs on. With `owned`, the block already owns
// node's parent (both children written before this launch) and skips the first arrival.
// sw: shared memory for the children's weights, followed by the parent's operands when
// climb_smem.
__device__ __forceinline__ void climb_loop(const DmHmat &H, int node, int climb_smem, bool owned, float *sw) {
    __shared__ int s_go;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int RH = H.rank_hi, RH4 = (RH + 3) & ~3, C4 = (2 * RH + 3) & ~3;
    float *Bs = sw + C4;          // RH x RH4: parent's K(S_l, S_r)
    float *Ps = Bs + RH * RH4;    // RH x C4: parent's P
    for (;;) {
        const int parent = (node - 1) >> 1;
        const int l = 2 * parent + 1, r = 2 * parent + 2;
        const int sl = H.ranks[l], sr = H.ranks[r], sp = parent > 0 ? H.ranks[parent] : 0;
        const int c = sl + sr, c4 = (c + 3) & ~3;
        if (!owned) {
            // publish this node's weights, then count the arrival at the parent
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) {
                const unsigned old = atomicAdd(H.cnt + parent, 1u);
                s_go = (old == 1u);
                if (old == 1u) H.cnt[parent] = 0u;  // both children arrived: reset for the next call
                __threadfence();
            }
            __syncthreads();
            if (!s_go) return;  // the sibling's block climbs on
        }
        owned = false;
        node = parent;
        if (climb_smem) {
            // the parent's operands (asynchronous copies), in flight while the children's
            // weights are read
            const float *Bn = H.B + (size_t)parent * H.max_rank * H.max_rank;
            for (int e = threadIdx.x; e < sl * sr; e += blockDim.x) {
                const int ia = e / sr, ib = e % sr;
                dm_cp_async4(Bs + ia * RH4 + ib, Bn + e);
            }
            const float *Pn = H.P + (size_t)parent * H.max_rank * H.ldp;
            const int q4 = c4 >> 2;
            for (int e = threadIdx.x; e < sp * q4; e += blockDim.x) {
                const int t = e / q4, q = e % q4;
                dm_cp_async16(Ps + t * C4 + 4 * q, Pn + (size_t)t * H.ldp + 4 * q);  // rows zero padded to ldp
            }
        }
        for (int j = threadIdx.x; j < c4; j += blockDim.x) {
            float v = 0.f;
            if (j < sl) v = __ldcg(H.what + (size_t)l * H.max_rank + j);
            else if (j < c) v = __ldcg(H.what + (size_t)r * H.max_rank + (j - sl));
            sw[j] = v;
        }
        if (climb_smem) dm_cp_async_wait_all();
        __syncthreads();
        // S2S: u_l = B w_r (warp per row of B), u_r = B^T w_l (thread per column of B)
        if (climb_smem) {
            for (int a2 = warp; a2 < sl; a2 += kHWarps) {
                float acc = 0.f;
                for (int b2 = lane; b2 < sr; b2 += 32) acc = fmaf(Bs[a2 * RH4 + b2], sw[sl + b2], acc);
                acc = dm_warp_sum(acc);
                if (lane == 0) H.uhat[(size_t)l * H.max_rank + a2] = acc;
            }
            for (int b2 = threadIdx.x; b2 < sr; b2 += blockDim.x) {
                float acc = 0.f;
                for (int a2 = 0; a2 < sl; ++a2) acc = fmaf(Bs[a2 * RH4 + b2], sw[a2], acc);
                H.uhat[(size_t)r * H.max_rank + b2] = acc;
            }
        } else {
            const float *Bn = H.B + (size_t)node * H.max_rank * H.max_rank;
            for (int a2 = warp; a2 < sl; a2 += kHWarps) {
                float acc = 0.f;
                for (int b2 = lane; b2 < sr; b2 += 32) acc = fmaf(__ldg(Bn + (size_t)a2 * sr + b2), sw[sl + b2], acc);
                acc = dm_warp_sum(acc);
                if (lane == 0) H.uhat[(size_t)l * H.max_rank + a2] = acc;
            }
            for (int b2 = threadIdx.x; b2 < sr; b2 += blockDim.x) {
                float acc = 0.f;
                for (int a2 = 0; a2 < sl; ++a2) acc = fmaf(__ldg(Bn + (size_t)a2 * sr + b2), sw[a2], acc);
                H.uhat[(size_t)r * H.max_rank + b2] = acc;
            }
        }
        if (node == 0) return;
        // N2S of the internal node
        if (climb_smem) gemv_rows_smem(Ps, C4, sp, c, sw, H.what + (size_t)node * H.max_rank);
        else
            gemv_rows(H.P + (size_t)node * H.max_rank * H.ldp, H.ldp, sp, c, sw, H.what + (size_t)node * H.max_rank,
                      nullptr);
        __syncthreads();  // Bs/Ps are refilled for the next parent
    }
}

// Leaf N2S of leaf `leaf`, then the climb from it
__device__ __forceinline__ void climb_body(const DmHmat &H, int leaf, const float *__restrict__ x, int permuted,
                                           int climb_smem) {
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    const int nleaves = 1 << H.L;
    const int m4max = (H.leaf_max + 3) & ~3;
    const int node = nleaves - 1 + leaf;
    int64_t st, sz;
    dm_node_range(H.N, node, &st, &sz);
    const int m = (int)sz, m4 = (m + 3) & ~3;
    float *sx = sm;  // m4max
    stage_x(H, x, permuted != 0, st, m, m4, sx);
    __syncthreads();
    gemv_leaf(H.P + (size_t)node * H.max_rank * H.ldp, H.ldp, H.ranks[node], m, sx, H.what + (size_t)node * H.max_rank);
    if (H.L == 0) return;
    climb_loop(H, node, climb_smem, false, sm + m4max);
}

// body of the chained form's first launch for one problem: block `bid` of its grid (leaf climbs
// first, then near items)
__device__ __forceinline__ void near_up_body(const DmHmat &H, int bid, const float *__restrict__ x, int permuted,
                                             int near_mode, int near_rows, int climb_smem) {
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    const int nleaves = 1 << H.L;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m4max = (H.leaf_max + 3) & ~3;
    if (bid < nleaves) {
        climb_body(H, bid, x, permuted, climb_smem);
        return;
    }

    // ---------------------------------------------------- near field
    const int item = bid - nleaves;
    const int per_leaf = (H.leaf_max + near_rows - 1) / near_rows;
    const int leaf = item / per_leaf, chunk = item % per_leaf;
    int64_t st, sz;
    dm_node_range(H.N, nleaves - 1 + leaf, &st, &sz);
    const int m = (int)sz, m4 = (m + 3) & ~3;
    const int r0 = chunk * near_rows;
    if (r0 >= m) return;
    const int r1 = min(m, r0 + near_rows);
    if (near_mode == DM_NEAR_CACHED) {
        float *sx = sm;
        stage_x(H, x, permuted != 0, st, m, m4, sx);
        __syncthreads();
        const float *blk = H.Knear + (size_t)leaf * H.leaf_max * H.ldk;
        const int m4q = m4 >> 2;
        const float4 *sx4 = reinterpret_cast<const float4 *>(sx);
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        // two rows per warp pass; each lane issues all of its 16-byte loads of both rows
        // (up to 4 per row, rows of up to 512 floats) before any arithmetic
        for (int i = r0 + 2 * warp; i < r1; i += 2 * kHWarps) {
            const bool two = (i + 1) < r1;
            const float4 *ra = reinterpret_cast<const float4 *>(blk + (size_t)i * H.ldk);
            const float4 *rb = reinterpret_cast<const float4 *>(blk + (size_t)(two ? i + 1 : i) * H.ldk);
            float acc_a = 0.f, acc_b = 0.f;
            for (int base = 0; base < m4q; base += 128) {
                float4 ka[4], kb[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int q = base + lane + 32 * t;
                    ka[t] = q < m4q ? __ldcs(ra + q) : zero;
                    kb[t] = (two && q < m4q) ? __ldcs(rb + q) : zero;
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int q = base + lane + 32 * t;
                    const float4 xv = q < m4q ? sx4[q] : zero;
                    acc_a = fmaf(ka[t].x, xv.x, acc_a);
                    acc_a = fmaf(ka[t].y, xv.y, acc_a);
                    acc_a = fmaf(ka[t].z, xv.z, acc_a);
                    acc_a = fmaf(ka[t].w, xv.w, acc_a);
                    acc_b = fmaf(kb[t].x, xv.x, acc_b);
                    acc_b = fmaf(kb[t].y, xv.y, acc_b);
                    acc_b = fmaf(kb[t].z, xv.z, acc_b);
                    acc_b = fmaf(kb[t].w, xv.w, acc_b);
                }
            }
            acc_a = dm_warp_sum(acc_a);
            acc_b = dm_warp_sum(acc_b);
            if (lane == 0) {
                H.ynear[st + i] = acc_a;
                if (two) H.ynear[st + i + 1] = acc_b;
            }
        }
    } else {
        // on the fly: thread per row, entries s_i s_j 2^-|xs_i - xs_j|^2 from staged points
        const int d = H.d;
        float *sxs = sm;                 // m4max: s_j x_j
        float *spts = sm + m4max;        // m x d coordinates
        for (int j = threadIdx.x; j < m; j += blockDim.x) {
            const float xv = permuted ? x[st + j] : x[H.perm[st + j]];
            sxs[j] = H.sp[st + j] * xv;
        }
        for (int e = threadIdx.x; e < m * d; e += blockDim.x) spts[e] = H.Xs[st * d + e];
        __syncthreads();
        for (int i = r0 + (int)threadIdx.x; i < r1; i += blockDim.x) {
            float acc = 0.f;
            if (d == 3) {
                const float x0 = spts[i * 3], x1 = spts[i * 3 + 1], x2 = spts[i * 3 + 2];
#pragma unroll 4
                for (int j = 0; j < m; ++j) {
                    const float t0 = x0 - spts[j * 3], t1 = x1 - spts[j * 3 + 1], t2 = x2 - spts[j * 3 + 2];
                    const float r2 = fmaf(t0, t0, fmaf(t1, t1, t2 * t2));
                    acc = fmaf(dm_ex2(-r2), sxs[j], acc);
                }
            } else {
                for (int j = 0; j < m; ++j) {
                    float r2 = 0.f;
                    for (int k = 0; k < d; ++k) {
                        const float t = spts[i * d + k] - spts[j * d + k];
                        r2 = fmaf(t, t, r2);
                    }
                    acc = fmaf(dm_ex2(-r2), sxs[j], acc);
                }
            }
            H.ynear[st + i] = H.sp[st + i] * acc;
        }
    }
}

__global__ void __launch_bounds__(kHThreads) near_up_kernel(const __grid_constant__ DmHmat H,
                                                            const float *__restrict__ x, int permuted, int near_mode,
                                                            int near_rows, int climb_smem) {
    near_up_body(H, (int)blockIdx.x, x, permuted, near_mode, near_rows, climb_smem);
}

// Downward pass for one leaf. The ancestor chain (S2S parts u of the ancestors at
// levels 2..L and, per step, the slice of the parent's P that maps to the child) is
// fetched into shared memory in one batch of independent loads when it fits
// (`chain_in_smem`), then combined top-down: t = P_parent(:, child)^T t + u_child.
// The leaf's own S2N reads the point-major copy PT: one contiguous row per point.
__device__ __forceinline__ void down_body(const DmHmat &H, int bid, float *__restrict__ y, int permuted,
                                          int chain_in_smem) {
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    // kDownSplit blocks per leaf, each handling a contiguous quarter of its points
    const int leaf = bid / kDownSplit, part = bid % kDownSplit;
    const int nleaves = 1 << H.L;
    const int node_leaf = nleaves - 1 + leaf;
    int64_t st, sz;
    dm_node_range(H.N, node_leaf, &st, &sz);
    const int per = ((int)sz + kDownSplit - 1) / kDownSplit;
    const int i_lo = part * per, i_hi = min((int)sz, i_lo + per);
    if (i_lo >= i_hi) return;
    if (H.L == 0) {
        for (int i = i_lo + threadIdx.x; i < i_hi; i += blockDim.x) {
            const float v = H.ynear[st + i];
            if (permuted) y[st + i] = v;
            else y[H.perm[st + i]] = v;
        }
        return;
    }
    const int R = H.max_rank, RH = H.rank_hi, RH4 = (RH + 3) & ~3;
    float *ta = sm, *tb = sm + RH4;
    float *chain = sm + 2 * RH4;  // per level l >= 2: u_l (RH4) then the P slice (RH x RH4)
    const int stride = RH4 + RH * RH4;
    if (chain_in_smem) {
        for (int lvl = 2; lvl <= H.L; ++lvl) {
            const int parent = ((node_leaf + 1) >> (H.L - lvl + 1)) - 1;
            const int child = ((node_leaf + 1) >> (H.L - lvl)) - 1;
            const int off = (child == 2 * parent + 2) ? H.ranks[2 * parent + 1] : 0;
            const int sp = H.ranks[parent], sc = H.ranks[child];
            float *u = chain + (size_t)(lvl - 2) * stride;
            float *Ps = u + RH4;
            const float *Pn = H.P + (size_t)parent * R * H.ldp + off;
            const int tot = sp * sc;
            for (int e = threadIdx.x; e < tot; e += blockDim.x)
                dm_cp_async4(Ps + (e / sc) * RH4 + (e % sc), Pn + (size_t)(e / sc) * H.ldp + (e % sc));
            for (int e = threadIdx.x; e < sc; e += blockDim.x) dm_cp_async4(u + e, H.uhat + (size_t)child * R + e);
        }
        dm_cp_async_wait_all();
    }
    int node = ((node_leaf + 1) >> (H.L - 1)) - 1;
    int s = H.ranks[node];
    for (int j = threadIdx.x; j < RH4; j += blockDim.x) ta[j] = j < s ? H.uhat[(size_t)node * R + j] : 0.f;
    __syncthreads();
    for (int lvl = 2; lvl <= H.L; ++lvl) {
        const int child = ((node_leaf + 1) >> (H.L - lvl)) - 1;
        const int sc = H.ranks[child];
        if (chain_in_smem) {
            const float *u = chain + (size_t)(lvl - 2) * stride;
            const float *Ps = u + RH4;
            for (int j = threadIdx.x; j < RH4; j += blockDim.x) {
                float acc = 0.f;
                if (j < sc) {
                    float a0 = u[j], a1 = 0.f, a2 = 0.f, a3 = 0.f;  // four independent chains
                    int t = 0;
                    for (; t + 4 <= s; t += 4) {
                        a0 = fmaf(Ps[t * RH4 + j], ta[t], a0);
                        a1 = fmaf(Ps[(t + 1) * RH4 + j], ta[t + 1], a1);
                        a2 = fmaf(Ps[(t + 2) * RH4 + j], ta[t + 2], a2);
                        a3 = fmaf(Ps[(t + 3) * RH4 + j], ta[t + 3], a3);
                    }
                    for (; t < s; ++t) a0 = fmaf(Ps[t * RH4 + j], ta[t], a0);
                    acc = (a0 + a1) + (a2 + a3);
                }
                tb[j] = acc;
            }
        } else {
            const int off = (child == 2 * node + 2) ? H.ranks[2 * node + 1] : 0;
            const float *Pn = H.P + (size_t)node * R * H.ldp;
            for (int j = threadIdx.x; j < RH4; j += blockDim.x) {
                float acc = 0.f;
                if (j < sc) {
                    acc = H.uhat[(size_t)child * R + j];
                    for (int t = 0; t < s; ++t) acc = fmaf(__ldg(Pn + (size_t)t * H.ldp + off + j), ta[t], acc);
                }
                tb[j] = acc;
            }
        }
        __syncthreads();
        float *tmp = ta;
        ta = tb;
        tb = tmp;
        node = child;
        s = sc;
    }
    // leaf S2N: y_i = y_near_i + PT[i, :] . t, PT rows zero padded to pt_ld (>= rank, multiple of 4)
    const float4 *PT = reinterpret_cast<const float4 *>(dm_pt_row(H, leaf, 0));
    const int q4 = H.pt_ld[leaf] >> 2;
    const float4 *t4 = reinterpret_cast<const float4 *>(ta);
    for (int i = i_lo + threadIdx.x; i < i_hi; i += blockDim.x) {
        const float4 *row = PT + (size_t)i * q4;
        float a0 = H.ynear[st + i], a1 = 0.f;
        // batches of 8 independent 16-byte loads (ranks up to 32 in one round trip)
        for (int q0 = 0; q0 < q4; q0 += 8) {
            float4 p[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) p[u] = (q0 + u < q4) ? __ldg(row + q0 + u) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
                if (q0 + u < q4) {
                    const float4 v0 = t4[q0 + u];
                    a0 = fmaf(p[u].x, v0.x, fmaf(p[u].y, v0.y, fmaf(p[u].z, v0.z, fmaf(p[u].w, v0.w, a0))));
                }
                if (q0 + u + 1 < q4) {
                    const float4 v1 = t4[q0 + u + 1];
                    a1 = fmaf(p[u + 1].x, v1.x, fmaf(p[u + 1].y, v1.y, fmaf(p[u + 1].z, v1.z, fmaf(p[u + 1].w, v1.w, a1))));
                }
            }
        }
        const float acc = a0 + a1;
        if (permuted) y[st + i] = acc;
        else y[H.perm[st + i]] = acc;
    }
}

__global__ void __launch_bounds__(kDownThreads) down_kernel(const __grid_constant__ DmHmat H, float *__restrict__ y,
                                                             int permuted, int chain_in_smem) {
    down_body(H, (int)blockIdx.x, y, permuted, chain_in_smem);
}

// ---- batched form (many problems, three launches) ------------------------------------------
//  up_batch_kernel        map[block] = {problem, leaf}: leaf N2S and the climb by last arrival.
//  sweep_batch_kernel     map[block] = {problem, subtree}: the internal levels' totals top-down
//                         (sweep_subtree), 2^min(L-1, 4) blocks per tree of depth L >= 3.
//  near_s2n_batch_kernel  map[block] = {problem, item}, item = (leaf, chunk of item_rows rows):
//                         the near rows (cached blocks streamed, or recomputed) into shared
//                         memory, then the leaf's total incoming vector
//                         t = u_leaf + P_parent(:, leaf's columns)^T t_parent and
//                         y_i = near_i + PT[i, :] t for the item's rows, in the problem's y.
//                         Many items are resident per SM, so one item's latency-bound tail
//                         overlaps the others' streaming.
__global__ void __launch_bounds__(kHThreads) up_batch_kernel(const DmChainProblem *__restrict__ P,
                                                             const int2 *__restrict__ map,
                                                             const int *__restrict__ jv) {
    const int2 pb = map[blockIdx.x];
    const DmChainProblem &p = P[pb.x];
    climb_body(p.H, pb.y, p.x + (size_t)jv[pb.x] * p.xstep, p.permuted, p.climb_smem);
}

// the top-down sweep, map[block] = {problem, s}: the block owns the subtree under node
// 2^lq - 1 + s of level lq = min(L - 1, kSweepCut) (trees of depth L >= 3)
constexpr int kSweepCut = 4;
__global__ void __launch_bounds__(kHThreads) sweep_batch_kernel(const DmChainProblem *__restrict__ P,
                                                                const int2 *__restrict__ map) {
    extern __shared__ float4 smem4[];
    const int2 pb = map[blockIdx.x];
    const DmHmat &H = P[pb.x].H;
    const int lq = H.L - 1 < kSweepCut ? H.L - 1 : kSweepCut;
    const int RH4 = (H.rank_hi + 3) & ~3;
    float *ta = reinterpret_cast<float *>(smem4), *tb = ta + RH4, *part = tb + RH4;
    sweep_subtree(H, (1 << lq) - 1 + pb.y, lq, ta, tb, part);
}

struct BatchItem {
    int leaf, m, r0, nr;
    int64_t st;
};
__device__ __forceinline__ BatchItem batch_item(const DmHmat &H, int item, int rows) {
    const int per_leaf = (H.leaf_max + rows - 1) / rows;
    BatchItem it;
    it.leaf = item / per_leaf;
    const int chunk = item - it.leaf * per_leaf;
    int64_t sz;
    dm_node_range(H.N, (1 << H.L) - 1 + it.leaf, &it.st, &sz);
    it.m = (int)sz;
    it.r0 = chunk * rows;
    it.nr = it.r0 < it.m ? min(rows, it.m - it.r0) : 0;
    return it;
}

constexpr int kNearBatchThreads = 256;
__global__ void __launch_bounds__(kNearBatchThreads, 6) near_s2n_batch_kernel(const DmChainProblem *__restrict__ P,
                                                                              const int2 *__restrict__ map,
                                                                              const int *__restrict__ jv) {
    extern __shared__ float4 smem4[];
    const int2 pb = map[blockIdx.x];
    const DmChainProblem &p = P[pb.x];
    const DmHmat &H = p.H;
    const BatchItem q = batch_item(H, pb.y, p.near_rows);
    if (q.nr == 0) return;
    const int permuted = p.permuted;
    const float *__restrict__ x = p.x + (size_t)jv[pb.x] * p.xstep;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kNearBatchThreads / 32;
    const int m4 = (q.m + 3) & ~3;
    const int m4max = (H.leaf_max + 3) & ~3;
    const int RH4 = (H.rank_hi + 3) & ~3;
    float *sx = reinterpret_cast<float *>(smem4);  // m4max: x~(I_a), or s_j x_j when recomputed
    float *res = sx + m4max;                       // item_rows (multiple of 4): near results
    float *tl = res + ((p.near_rows + 3) & ~3);    // RH4: the leaf's total incoming vector
    float *tpar = tl + RH4;                        // RH4: the parent's total
    float *part = tpar + RH4;                      // 4 x RH4: partial sums of P_parent^T t_parent
    float *spts = part + 4 * RH4;                  // recomputed near field: m x d coordinates
    if (p.near_mode == DM_NEAR_CACHED) {
        for (int j = threadIdx.x; j < m4; j += kNearBatchThreads) {
            float v = 0.f;
            if (j < q.m) v = permuted ? x[q.st + j] : x[H.perm[q.st + j]];
            sx[j] = v;
        }
        __syncthreads();
        const float *blk = H.Knear + ((size_t)q.leaf * H.leaf_max + q.r0) * H.ldk;
        const int q4 = m4 >> 2;
        const float4 *x4 = reinterpret_cast<const float4 *>(sx);
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        // a warp per pair of rows; every 16-byte streaming load of both rows (up to 512
        // columns) issued before the sums
        for (int i = 2 * warp; i < q.nr; i += 2 * nw) {
            const bool two = i + 1 < q.nr;
            const float4 *ra = reinterpret_cast<const float4 *>(blk + (size_t)i * H.ldk);
            const float4 *rb = reinterpret_cast<const float4 *>(blk + (size_t)(two ? i + 1 : i) * H.ldk);
            float acc_a = 0.f, acc_b = 0.f;
            for (int base = 0; base < q4; base += 128) {
                float4 ka[4], kb[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int v = base + lane + 32 * t;
                    ka[t] = v < q4 ? __ldcs(ra + v) : zero;
                    kb[t] = (two && v < q4) ? __ldcs(rb + v) : zero;
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int v = base + lane + 32 * t;
                    const float4 xv = v < q4 ? x4[v] : zero;
                    acc_a = fmaf(ka[t].x, xv.x, fmaf(ka[t].y, xv.y, fmaf(ka[t].z, xv.z, fmaf(ka[t].w, xv.w, acc_a))));
                    acc_b = fmaf(kb[t].x, xv.x, fmaf(kb[t].y, xv.y, fmaf(kb[t].z, xv.z, fmaf(kb[t].w, xv.w, acc_b))));
                }
            }
            acc_a = dm_warp_sum(acc_a);
            acc_b = dm_warp_sum(acc_b);
            if (lane == 0) {
                res[i] = acc_a;
                if (two) res[i + 1] = acc_b;
            }
        }
    } else {
        // recomputed: thread per row, entries s_i s_j 2^-|xs_i - xs_j|^2 from staged points
        const int d = H.d;
        for (int j = threadIdx.x; j < q.m; j += kNearBatchThreads) {
            const float xv = permuted ? x[q.st + j] : x[H.perm[q.st + j]];
            sx[j] = H.sp[q.st + j] * xv;
        }
        for (int e = threadIdx.x; e < q.m * d; e += kNearBatchThreads) spts[e] = H.Xs[q.st * d + e];
        __syncthreads();
        for (int li = threadIdx.x; li < q.nr; li += kNearBatchThreads) {
            const int i = q.r0 + li;
            float acc = 0.f;
            for (int j = 0; j < q.m; ++j) {
                float r2 = 0.f;
                for (int k = 0; k < d; ++k) {
                    const float t = spts[i * d + k] - spts[j * d + k];
                    r2 = fmaf(t, t, r2);
                }
                acc = fmaf(dm_ex2(-r2), sx[j], acc);
            }
            res[li] = H.sp[q.st + i] * acc;
        }
    }
    // the leaf's total incoming vector
    const int node = (1 << H.L) - 1 + q.leaf;
    const int s = H.L > 0 ? H.ranks[node] : 0;
    const int s4 = (s + 3) & ~3;
    if (H.L >= 2) {
        const int par = (node - 1) >> 1, sp = H.ranks[par];
        const int off = (node == 2 * par + 2) ? H.ranks[2 * par + 1] : 0;
        const float *Pn = H.P + (size_t)par * H.max_rank * H.ldp + off;
        for (int t = threadIdx.x; t < sp; t += kNearBatchThreads) tpar[t] = __ldcg(H.uhat + (size_t)par * H.max_rank + t);
        __syncthreads();
        // four groups of 64 threads over quarters of the parent's rank
        const int g = threadIdx.x >> 6, j0 = threadIdx.x & 63;
        const int tq = (sp + 3) >> 2, t0 = g * tq, t1 = min(sp, t0 + tq);
        for (int j = j0; j < s; j += 64) {
            float a0 = 0.f, a1 = 0.f;
            int t = t0;
            for (; t + 2 <= t1; t += 2) {
                a0 = fmaf(__ldg(Pn + (size_t)t * H.ldp + j), tpar[t], a0);
                a1 = fmaf(__ldg(Pn + (size_t)(t + 1) * H.ldp + j), tpar[t + 1], a1);
            }
            if (t < t1) a0 = fmaf(__ldg(Pn + (size_t)t * H.ldp + j), tpar[t], a0);
            part[g * RH4 + j] = a0 + a1;
        }
        __syncthreads();
        const float *u = H.uhat + (size_t)node * H.max_rank;
        for (int j = threadIdx.x; j < s4; j += kNearBatchThreads)
            tl[j] = j < s ? __ldcg(u + j) + ((part[j] + part[RH4 + j]) + (part[2 * RH4 + j] + part[3 * RH4 + j])) : 0.f;
    } else if (H.L == 1) {
        const float *u = H.uhat + (size_t)node * H.max_rank;
        for (int j = threadIdx.x; j < s4; j += kNearBatchThreads) tl[j] = j < s ? __ldcg(u + j) : 0.f;
    }
    __syncthreads();
    // leaf S2N: PT rows are zero padded beyond the rank
    const float4 *t4 = reinterpret_cast<const float4 *>(tl);
    const int q4 = s4 >> 2;
    for (int li = threadIdx.x; li < q.nr; li += kNearBatchThreads) {
        const int i = q.r0 + li;
        float a0 = res[li], a1 = 0.f;
        if (q4 > 0) {
            const float4 *prow = reinterpret_cast<const float4 *>(dm_pt_row(H, q.leaf, i));
            for (int v = 0; v < q4; v += 2) {
                const float4 pa = __ldg(prow + v);
                const float4 ta = t4[v];
                a0 = fmaf(pa.x, ta.x, fmaf(pa.y, ta.y, fmaf(pa.z, ta.z, fmaf(pa.w, ta.w, a0))));
                if (v + 1 < q4) {
                    const float4 pv = __ldg(prow + v + 1);
                    const float4 tb = t4[v + 1];
                    a1 = fmaf(pv.x, tb.x, fmaf(pv.y, tb.y, fmaf(pv.z, tb.z, fmaf(pv.w, tb.w, a1))));
                }
            }
        }
        const float acc = a0 + a1;
        if (p.permuted) p.y[q.st + i] = acc;
        else p.y[H.perm[q.st + i]] = acc;
    }
}

}  // namespace

int dm_near_rows(int near_mode, int leaf_max) {
    if (near_mode == DM_NEAR_CACHED) return (leaf_max + kCachedItemsPerLeaf - 1) / kCachedItemsPerLeaf;
    const int chunks = (leaf_max + kHThreads - 1) / kHThreads;
    return (leaf_max + chunks - 1) / chunks;
}

DmChainShape dm_chain_shape(const DmHmat &H, int near_mode) {
    DmChainShape c;
    const int nleaves = 1 << H.L;
    c.near_rows = dm_near_rows(near_mode, H.leaf_max);
    const int per_leaf = (H.leaf_max + c.near_rows - 1) / c.near_rows;
    c.up_blocks = nleaves;
    c.near_blocks = nleaves * per_leaf;
    c.down_blocks = nleaves * kDownSplit;
    const int m4max = (H.leaf_max + 3) & ~3;
    const size_t RH = (size_t)H.rank_hi, RH4 = (RH + 3) & ~3, C4 = (2 * RH + 3) & ~3;
    // up items: staged x, children weights, and (when small enough) the parent's B and P
    const size_t climb_bytes = sizeof(float) * (RH * RH4 + RH * C4);
    c.climb_smem = climb_bytes <= 96 * 1024 ? 1 : 0;
    c.smem1 = sizeof(float) * ((size_t)m4max + C4 + 2 * (size_t)H.max_rank + 4) + (c.climb_smem ? climb_bytes : 0);
    if (near_mode != DM_NEAR_CACHED) {
        const size_t s2 = sizeof(float) * (size_t)(m4max + H.leaf_max * H.d);
        if (s2 > c.smem1) c.smem1 = s2;
    }
    // the ancestor chain fits in shared memory for the usual ranks; otherwise read it from L2
    const size_t chain = sizeof(float) * (2 * RH4 + (size_t)(H.L > 1 ? H.L - 1 : 0) * (RH4 + RH * RH4));
    c.chain_smem = chain <= 160 * 1024 ? 1 : 0;
    c.smem2 = c.chain_smem ? chain : sizeof(float) * 2 * RH4;
    return c;
}

cudaError_t dm_hmatvec_chain(const DmHmat &H, int near_mode, const float *x, float *y, bool permuted, cudaStream_t st) {
    const DmChainShape c = dm_chain_shape(H, near_mode);
    {
        cudaError_t e = dm_allow_smem((const void *)near_up_kernel, c.smem1);
        if (e != cudaSuccess) return e;
    }
    near_up_kernel<<<c.up_blocks + c.near_blocks, kHThreads, c.smem1, st>>>(H, x, permuted ? 1 : 0, near_mode,
                                                                             c.near_rows, c.climb_smem);
    dm_count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    {
        cudaError_t e2 = dm_allow_smem((const void *)down_kernel, c.smem2);
        if (e2 != cudaSuccess) return e2;
    }
    down_kernel<<<c.down_blocks, kDownThreads, c.smem2, st>>>(H, y, permuted ? 1 : 0, c.chain_smem);
    dm_count_launches(1);
    return cudaGetLastError();
}

DmBatchShape dm_batch_shape(const DmHmat &H, int near_mode) {
    DmBatchShape c;
    const int nleaves = 1 << H.L;
    c.item_rows = dm_near_item_rows(near_mode, H.leaf_max);
    c.items = nleaves * ((H.leaf_max + c.item_rows - 1) / c.item_rows);
    c.climbs = H.L > 0 ? nleaves : 0;
    c.sweeps = H.L >= 3 ? 1 << (H.L - 1 < kSweepCut ? H.L - 1 : kSweepCut) : 0;
    const int m4max = (H.leaf_max + 3) & ~3;
    const size_t RH = (size_t)H.rank_hi, RH4 = (RH + 3) & ~3, C4 = (2 * RH + 3) & ~3;
    const size_t climb_bytes = sizeof(float) * (RH * RH4 + RH * C4);
    c.climb_smem = climb_bytes <= 96 * 1024 ? 1 : 0;
    c.smem_up = sizeof(float) * ((size_t)m4max + C4) + (c.climb_smem ? climb_bytes : 0);
    c.smem_near = sizeof(float) * ((size_t)m4max + (size_t)((c.item_rows + 3) & ~3) + 6 * RH4);
    if (near_mode != DM_NEAR_CACHED) c.smem_near += sizeof(float) * (size_t)H.leaf_max * H.d;
    c.smem_sweep = sizeof(float) * 4 * RH4;
    return c;
}

cudaError_t dm_hmatvec_batch(const DmChainProblem *P, const int2 *map_up, int n_up, size_t smem_up,
                             const int2 *map_sweep, int n_sweep, size_t smem_sweep, const int2 *map_near, int n_near,
                             size_t smem_near, const int *jv, cudaStream_t st) {
    cudaError_t e;
    if (n_up > 0) {
        if ((e = dm_allow_smem((const void *)up_batch_kernel, smem_up)) != cudaSuccess) return e;
        up_batch_kernel<<<n_up, kHThreads, smem_up, st>>>(P, map_up, jv);
        dm_count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (n_sweep > 0) {
        if ((e = dm_allow_smem((const void *)sweep_batch_kernel, smem_sweep)) != cudaSuccess) return e;
        sweep_batch_kernel<<<n_sweep, kHThreads, smem_sweep, st>>>(P, map_sweep);
        dm_count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (n_near == 0) return cudaSuccess;
    if ((e = dm_allow_smem((const void *)near_s2n_batch_kernel, smem_near)) != cudaSuccess) return e;
    near_s2n_batch_kernel<<<n_near, kNearBatchThreads, smem_near, st>>>(P, map_near, jv);
    dm_count_launches(1);
    return cudaGetLastError();
}
