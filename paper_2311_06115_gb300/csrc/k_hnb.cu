// k_hnb.cu -- the hierarchical matvec Y = K~ X of Eq. 2.18 for a narrow block of NB <= 4
// right-hand sides, as the same three chained launches as the single-vector form in
// k_htree.cu (the operator of block Lanczos with small blocks):
//
//   A leaf_n2s_nb_kernel   block per leaf: W_a = P_a X(I_a, :)            (leaf N2S)
//   B tree_nb_kernel       one thread-block cluster: the whole upper tree (internal N2S,
//                          every S2S, internal S2N) with operands and NB-wide skeleton
//                          vectors in the cluster's shared memory
//   C near_nb_kernel       the stored leaf blocks streamed once for all NB columns, then
//                          the leaf S2N Y(I_a, :) += P_a^T U_a
//
// Every stored operand is read once per call for all NB columns, so the call costs about
// what a single-vector H-matvec costs (the near stream is bound by HBM, the tree pass by
// latency) while it applies the operator to NB vectors. Skeleton vectors are kept t-major,
// [rank][NB], so one 16-byte shared-memory load serves all columns of a row.
//
// The cluster is cut at level ls (2^ls CTAs, 8 or 16); CTA c owns the subtree under node
// 2^ls - 1 + c, and the 2^ls - 1 nodes above the cut go to the CTAs in an order that
// balances shared memory (largest node first to the least loaded CTA): the owner of every
// node is a table in the image. B and C are programmatic dependents of their predecessors.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "dm_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kNbLeafThreads = 256;
constexpr int kNbTreeThreads = 1024;
constexpr int kNbNearThreads = 256;
constexpr int kNbNearRowsTarget = 136;

__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <int NB>
__device__ __forceinline__ float col_dot4(const float4 k, const float4 *x4, int c, int q, int m4q) {
    const float4 v = x4[(size_t)c * m4q + q];
    return fmaf(k.x, v.x, fmaf(k.y, v.y, fmaf(k.z, v.z, k.w * v.w)));
}

// ------------------------------------------------------------------ A: leaf N2S

// W[leaf][t][c] = sum_j P_leaf[t][j] X[c][st + j]; x staged column by column ([NB][m4]); a warp
// per pair of basis rows with every 16-byte load of both rows issued before the sums.
template <int NB>
__global__ void __launch_bounds__(kNbLeafThreads) leaf_n2s_nb_kernel(const __grid_constant__ DmHmat H,
                                                                    const __grid_constant__ DmNbTree T,
                                                                    const float *__restrict__ x, int64_t ldx,
                                                                    int permuted) {
    grid_dep_launch();
    extern __shared__ float4 smem4[];
    float *sx = reinterpret_cast<float *>(smem4);
    const int nleaves = 1 << H.L;
    const int node = nleaves - 1 + blockIdx.x;
    const int s = H.ranks[node];
    const int row0 = blockIdx.y * 2 * (blockDim.x >> 5);
    if (row0 >= s) return;
    int64_t st, sz;
    dm_node_range(H.N, node, &st, &sz);
    const int m = (int)sz, m4 = (m + 3) & ~3, q4 = m4 >> 2;
    const float *P = H.P + (size_t)node * H.max_rank * H.ldp;
    float *out = T.what + (size_t)node * H.max_rank * NB;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    const int t0 = row0 + 2 * warp;
    float4 ka[4], kb[4];
    auto load_pair = [&](int t, int base) {
        const bool two = t + 1 < s;
        const float4 *ra = reinterpret_cast<const float4 *>(P + (size_t)t * H.ldp);
        const float4 *rb = reinterpret_cast<const float4 *>(P + (size_t)(two ? t + 1 : t) * H.ldp);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = base + lane + 32 * u;
            ka[u] = q < q4 ? __ldg(ra + q) : zero;
            kb[u] = (two && q < q4) ? __ldg(rb + q) : zero;
        }
    };
    if (t0 < s) load_pair(t0, 0);
    for (int e = threadIdx.x; e < NB * m4; e += blockDim.x) {
        const int c = e / m4, j = e - c * m4;
        float v = 0.f;
        if (j < m) v = x[(size_t)c * ldx + (permuted ? st + j : (int64_t)H.perm[st + j])];
        sx[e] = v;
    }
    __syncthreads();
    const float4 *x4 = reinterpret_cast<const float4 *>(sx);
    for (int t = t0; t < s; t += 2 * nw * (int)gridDim.y) {
        float acc_a[NB], acc_b[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) acc_a[c] = acc_b[c] = 0.f;
        for (int base = 0; base < q4; base += 128) {
            if (t != t0 || base != 0) load_pair(t, base);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q = base + lane + 32 * u;
                if (q < q4) {
#pragma unroll
                    for (int c = 0; c < NB; ++c) {
                        acc_a[c] += col_dot4<NB>(ka[u], x4, c, q, q4);
                        acc_b[c] += col_dot4<NB>(kb[u], x4, c, q, q4);
                    }
                }
            }
        }
#pragma unroll
        for (int c = 0; c < NB; ++c) {
            const float a = dm_warp_sum(acc_a[c]), b = dm_warp_sum(acc_b[c]);
            if (lane == 0) {
                out[(size_t)t * NB + c] = a;
                if (t + 1 < s) out[(size_t)(t + 1) * NB + c] = b;
            }
        }
    }
}

// ------------------------------------------------------------------ B: upper tree in one cluster

// out[(obase + o) NB + c] (=, or += when add) = sum_{k < nk} A(o, k) V[(vbase + k) NB + c]
// for o < nout, A(o, k) = sm[abase + o ao + k ak]; warps gw = 0..ngw-1 of a group; 8 outputs
// per warp pass, 4 lanes per output splitting k
template <int NB>
__device__ __forceinline__ void grp_gemm(const float *sm, int abase, int ao, int ak, int nout, int nk, int vbase,
                                         float *out, int obase, bool add, int gw, int ngw, int lane) {
    const int q = lane >> 2, ql = lane & 3;
    for (int o0 = gw * 8; o0 < nout; o0 += ngw * 8) {
        const int o = o0 + q;
        float acc[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) acc[c] = 0.f;
        if (o < nout) {
            const float *pa = sm + abase + o * ao;
            for (int k = ql; k < nk; k += 4) {
                const float a = pa[k * ak];
                const float *v = sm + vbase + k * NB;
                if constexpr (NB == 4) {
                    const float4 v4 = *reinterpret_cast<const float4 *>(v);
                    acc[0] = fmaf(a, v4.x, acc[0]);
                    acc[1] = fmaf(a, v4.y, acc[1]);
                    acc[2] = fmaf(a, v4.z, acc[2]);
                    acc[3] = fmaf(a, v4.w, acc[3]);
                } else {
#pragma unroll
                    for (int c = 0; c < NB; ++c) acc[c] = fmaf(a, v[c], acc[c]);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < NB; ++c) {
            acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 1);
            acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 2);
        }
        if (o < nout && ql == 0) {
            float *dst = out + (size_t)(obase + o * NB);
#pragma unroll
            for (int c = 0; c < NB; ++c) dst[c] = add ? dst[c] + acc[c] : acc[c];
        }
    }
}

// S2S of the pair in slot pr ([w_l | w_r | u_l | u_r], NB-wide rows): u_l = B w_r, u_r = B^T w_l
template <int NB>
__device__ __forceinline__ void grp_s2s_nb(const float *sm, int bo, int sl, int sr, int pr, float *out, int gw,
                                           int ngw, int lane) {
    const int rs = sr | 1, c = sl + sr;
    grp_gemm<NB>(sm, bo, rs, 1, sl, sr, pr + sl * NB, out, pr + c * NB, false, gw, ngw, lane);
    grp_gemm<NB>(sm, bo, 1, rs, sr, sl, pr, out, pr + (c + sl) * NB, false, gw, ngw, lane);
}

// Smem image of CTA c (floats): int4 lay[nnodes], int rk[nnodes] (padded to 4), int2 own[nnodes],
// int owner[nnodes] (padded to 4), then the nodes' operands and vector slots.
//   lay[n] = {P (column-major, stride s_n|1), B (row-major s_l x (s_r|1)), pair slot, scratch}
//   pair slot of an internal node at level >= ls: [w_l | w_r | u_l | u_r] of its children
//   scratch of a node above ls: a copy of its children's pair (they live in other CTAs)
//   own[n] = {w, u} offsets of node n's own vectors (in its owner's smem)
struct NbMeta {
    const int4 *lay;
    const int *rk;
    const int2 *own;
    const int *owner;
};
__device__ __forceinline__ NbMeta nb_meta(const float *sm, int nnodes) {
    NbMeta M;
    M.lay = reinterpret_cast<const int4 *>(sm);
    M.rk = reinterpret_cast<const int *>(M.lay + nnodes);
    M.own = reinterpret_cast<const int2 *>(M.rk + ((nnodes + 3) & ~3));
    M.owner = reinterpret_cast<const int *>(M.own + nnodes);
    return M;
}

template <int NB>
__global__ void __launch_bounds__(kNbTreeThreads) tree_nb_kernel(const __grid_constant__ DmHmat H,
                                                               const __grid_constant__ DmNbTree T) {
    grid_dep_launch();
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    cg::cluster_group cl = cg::this_cluster();
    const int ls = T.ls, L = H.L, nc = 1 << ls, R = H.max_rank;
    const int c = (int)cl.block_rank();
    const int g = nc - 1 + c;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nnodes = (2 << L) - 1;
    {
        const int o0 = T.img_off[c], len = T.img_off[c + 1] - o0;
        const float *src = T.img + o0;
        for (int i = 4 * threadIdx.x; i < len; i += 4 * blockDim.x) dm_cp_async16(sm + i, src + i);
    }
    grid_dep_wait();  // the leaves' weights come from the leaf N2S launch
    dm_cp_async_wait_all();
    __syncthreads();
    const NbMeta M = nb_meta(sm, nnodes);
    auto own_w = [&](int n) { return M.own[n].x; };
    auto own_u = [&](int n) { return M.own[n].y; };
    {
        // the leaves' weights (L2 reads: written by the leaf N2S launch): a lane's loads are all
        // issued before the first store, so one round trip serves the whole row
        const int first = ((g + 1) << (L - ls)) - 1, count = 1 << (L - ls);
        for (int i = warp; i < count; i += nw) {
            const int n = first + i, w = own_w(n), len = M.rk[n] * NB;
            const float *src = T.what + (size_t)n * R * NB;
            for (int base = lane; base < len; base += 256) {
                float t[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) t[u] = base + 32 * u < len ? __ldcg(src + base + 32 * u) : 0.f;
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (base + 32 * u < len) sm[w + base + 32 * u] = t[u];
            }
        }
    }
    __syncthreads();
    // upward pass inside the subtree: the N2S chain alone (w_n = P_n [w_l; w_r]); the S2S
    // products feed only the downward pass, so they leave the chain
    for (int lv = L - 1; lv >= ls; --lv) {
        const int first = ((g + 1) << (lv - ls)) - 1, count = 1 << (lv - ls);
        const int ngw = count >= nw ? 1 : nw / count;
        for (int i = warp / ngw; i < count; i += nw / ngw) {
            const int n = first + i, gw = warp % ngw;
            if (n == 0) continue;
            const int sl = M.rk[2 * n + 1], sr = M.rk[2 * n + 2], pr = M.lay[n].z;
            grp_gemm<NB>(sm, M.lay[n].x, 1, M.rk[n] | 1, M.rk[n], sl + sr, pr, sm, own_w(n), false, gw, ngw, lane);
        }
        __syncthreads();
    }
    // every S2S of the subtree at once: u_l = B w_r and u_r = B^T w_l of each child pair, two
    // independent products per node spread over all warps
    {
        const int nsub = (1 << (L - ls)) - 1;  // internal nodes of the subtree (levels ls .. L-1)
        const int tasks = 2 * nsub;
        const int ngw = tasks >= nw ? 1 : nw / tasks;
        for (int tk = warp / ngw; tk < tasks; tk += nw / ngw) {
            const int gw = warp % ngw, idx = tk >> 1;
            const int lvo = 31 - __clz(idx + 1);  // level of the node inside the subtree
            const int n = ((g + 1) << lvo) - 1 + (idx + 1 - (1 << lvo));
            const int sl = M.rk[2 * n + 1], sr = M.rk[2 * n + 2], pr = M.lay[n].z, bo = M.lay[n].y;
            const int rs = sr | 1, cc = sl + sr;
            if ((tk & 1) == 0) grp_gemm<NB>(sm, bo, rs, 1, sl, sr, pr + sl * NB, sm, pr + cc * NB, false, gw, ngw, lane);
            else grp_gemm<NB>(sm, bo, 1, rs, sr, sl, pr, sm, pr + (cc + sl) * NB, false, gw, ngw, lane);
        }
        __syncthreads();
    }
    // the levels above ls: each CTA takes the nodes it owns, one after the other
    if (nc > 1) {
        for (int lv = ls - 1; lv >= 0; --lv) {
            cl.sync();
            const int first = (1 << lv) - 1, count = 1 << lv;
            for (int n = first; n < first + count; ++n) {
                if (M.owner[n] != c) continue;
                const int l = 2 * n + 1, r = 2 * n + 2, sl = M.rk[l], sr = M.rk[r], cc = sl + sr;
                const int pr = M.lay[n].w;
                const float *wl = cl.map_shared_rank(sm + own_w(l), M.owner[l]);
                const float *wr = cl.map_shared_rank(sm + own_w(r), M.owner[r]);
                for (int j = threadIdx.x; j < cc * NB; j += blockDim.x)
                    sm[pr + j] = j < sl * NB ? wl[j] : wr[j - sl * NB];
                __syncthreads();
                grp_s2s_nb<NB>(sm, M.lay[n].y, sl, sr, pr, sm, warp, nw, lane);
                if (n > 0)
                    grp_gemm<NB>(sm, M.lay[n].x, 1, M.rk[n] | 1, M.rk[n], cc, pr, sm, own_w(n), false, warp, nw,
                                 lane);
                __syncthreads();
                float *ul = cl.map_shared_rank(sm + own_u(l), M.owner[l]);
                float *ur = cl.map_shared_rank(sm + own_u(r), M.owner[r]);
                for (int j = threadIdx.x; j < cc * NB; j += blockDim.x) {
                    const float v = sm[pr + cc * NB + j];
                    if (j < sl * NB) ul[j] = v;
                    else ur[j - sl * NB] = v;
                }
                __syncthreads();
            }
        }
        for (int lv = 1; lv < ls; ++lv) {
            cl.sync();
            const int first = (1 << lv) - 1, count = 1 << lv;
            for (int n = first; n < first + count; ++n) {
                if (M.owner[n] != c) continue;
                const int l = 2 * n + 1, r = 2 * n + 2, sl = M.rk[l], sr = M.rk[r], cc = sl + sr, s = M.rk[n];
                const int pr = M.lay[n].w;
                grp_gemm<NB>(sm, M.lay[n].x, s | 1, 1, cc, s, own_u(n), sm, pr + cc * NB, false, warp, nw, lane);
                __syncthreads();
                float *ul = cl.map_shared_rank(sm + own_u(l), M.owner[l]);
                float *ur = cl.map_shared_rank(sm + own_u(r), M.owner[r]);
                for (int j = threadIdx.x; j < cc * NB; j += blockDim.x) {
                    const float v = sm[pr + cc * NB + j];
                    if (j < sl * NB) ul[j] += v;
                    else ur[j - sl * NB] += v;
                }
                __syncthreads();
            }
        }
        cl.sync();
    }
    // downward pass inside the subtree: the pair's u += P^T u_n
    for (int lv = ls; lv < L; ++lv) {
        const int first = ((g + 1) << (lv - ls)) - 1, count = 1 << (lv - ls);
        const int ngw = count >= nw ? 1 : nw / count;
        for (int i = warp / ngw; i < count; i += nw / ngw) {
            const int n = first + i, gw = warp % ngw;
            if (n == 0) continue;
            const int sl = M.rk[2 * n + 1], sr = M.rk[2 * n + 2], cc = sl + sr, s = M.rk[n];
            grp_gemm<NB>(sm, M.lay[n].x, s | 1, 1, cc, s, own_u(n), sm, M.lay[n].z + cc * NB, true, gw, ngw, lane);
        }
        __syncthreads();
    }
    {
        const int first = ((g + 1) << (L - ls)) - 1, count = 1 << (L - ls);
        for (int i = warp; i < count; i += nw) {
            const int n = first + i, u = own_u(n), len = M.rk[n] * NB;
            for (int j = lane; j < len; j += 32) T.uhat[(size_t)n * R * NB + j] = sm[u + j];
        }
    }
}

// Image of CTA c: metadata, then every owned internal node's B and P (one warp per node).
__global__ void __launch_bounds__(512) tree_nb_image_kernel(const __grid_constant__ DmHmat H,
                                                          const __grid_constant__ DmNbTree T) {
    const int L = H.L, c = blockIdx.x;
    const int nnodes = (2 << L) - 1, ninternal = (1 << L) - 1;
    float *out = T.img + T.img_off[c];
    int4 *lay = reinterpret_cast<int4 *>(out);
    int *rk = reinterpret_cast<int *>(lay + nnodes);
    int2 *own = reinterpret_cast<int2 *>(rk + ((nnodes + 3) & ~3));
    int *owner = reinterpret_cast<int *>(own + nnodes);
    if (blockIdx.y == 0)
        for (int n = threadIdx.x; n < nnodes; n += blockDim.x) {
            lay[n] = T.lay[n];
            rk[n] = H.ranks[n];
            own[n] = T.own[n];
            owner[n] = T.owner[n];
        }
    const int lane = threadIdx.x & 31, nwt = (int)(blockDim.x >> 5) * (int)gridDim.y;
    const int warp = (int)blockIdx.y * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5);
    int mine = 0;
    for (int n = 0; n < ninternal; ++n) {
        if (T.owner[n] != c) continue;
        if ((mine++ % nwt) != warp) continue;
        const int4 ln = T.lay[n];
        const int s = H.ranks[n], sl = H.ranks[2 * n + 1], sr = H.ranks[2 * n + 2], cc = sl + sr;
        const float *Bg = H.B + (size_t)n * H.max_rank * H.max_rank;
        const int rs = sr | 1;
        for (int e = lane; e < sl * rs; e += 32) {
            const int a = e / rs, b = e - a * rs;
            out[ln.y + e] = b < sr ? Bg[a * sr + b] : 0.f;
        }
        if (n == 0) continue;
        const float *Pg = H.P + (size_t)n * H.max_rank * H.ldp;
        const int cs = s | 1;
        for (int e = lane; e < cc * cs; e += 32) {
            const int j = e / cs, t = e - j * cs;
            out[ln.x + e] = t < s ? Pg[(size_t)t * H.ldp + j] : 0.f;
        }
    }
}

// ------------------------------------------------------------------ C: near field + leaf S2N

template <int NB>
__global__ void __launch_bounds__(kNbNearThreads, 4) near_nb_kernel(const __grid_constant__ DmHmat H,
                                                                    const __grid_constant__ DmNbTree T,
                                                                    const float *__restrict__ x, int64_t ldx,
                                                                    float *__restrict__ y, int64_t ldy, int permuted,
                                                                    int rows, int far) {
    extern __shared__ float4 smem4[];
    const int per_leaf = (H.leaf_max + rows - 1) / rows;
    const int leaf = blockIdx.x / per_leaf, chunk = blockIdx.x - leaf * per_leaf;
    int64_t st, sz;
    dm_node_range(H.N, (1 << H.L) - 1 + leaf, &st, &sz);
    const int m = (int)sz, r0 = chunk * rows;
    const int nr = r0 < m ? min(rows, m - r0) : 0;
    if (nr == 0) return;
    const int m4 = (m + 3) & ~3, q4 = m4 >> 2;
    const int m4max = (H.leaf_max + 3) & ~3;
    float *sx = reinterpret_cast<float *>(smem4);  // NB x m4 (column stride m4)
    float *res = sx + NB * m4max;                  // rows x NB
    float *us = res + ((rows * NB + 3) & ~3);      // rank x NB (leaf S2N)
    for (int e = threadIdx.x; e < NB * m4; e += blockDim.x) {
        const int c = e / m4, j = e - c * m4;
        float v = 0.f;
        if (j < m) v = x[(size_t)c * ldx + (permuted ? st + j : (int64_t)H.perm[st + j])];
        sx[e] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float *blk = H.Knear + ((size_t)leaf * H.leaf_max + r0) * H.ldk;
    const float4 *x4 = reinterpret_cast<const float4 *>(sx);
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = 2 * warp; i < nr; i += 2 * nw) {
        const bool two = i + 1 < nr;
        const float4 *ra = reinterpret_cast<const float4 *>(blk + (size_t)i * H.ldk);
        const float4 *rb = reinterpret_cast<const float4 *>(blk + (size_t)(two ? i + 1 : i) * H.ldk);
        float4 ka[4], kb[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int v = lane + 32 * t;
            ka[t] = v < q4 ? __ldcs(ra + v) : zero;
            kb[t] = (two && v < q4) ? __ldcs(rb + v) : zero;
        }
        float acc_a[NB], acc_b[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) acc_a[c] = acc_b[c] = 0.f;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int v = lane + 32 * t;
            if (v < q4) {
#pragma unroll
                for (int c = 0; c < NB; ++c) {
                    acc_a[c] += col_dot4<NB>(ka[t], x4, c, v, q4);
                    acc_b[c] += col_dot4<NB>(kb[t], x4, c, v, q4);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < NB; ++c) {
            const float a = dm_warp_sum(acc_a[c]), b = dm_warp_sum(acc_b[c]);
            if (lane == 0) {
                res[i * NB + c] = a;
                if (two) res[(i + 1) * NB + c] = b;
            }
        }
    }
    const int node = (1 << H.L) - 1 + leaf;
    const int sr = far ? __ldg(H.ranks + node) : 0;
    if (far) {
        grid_dep_wait();  // the tree pass has written the leaves' u
        const float *u = T.uhat + (size_t)node * H.max_rank * NB;
        for (int e = threadIdx.x; e < sr * NB; e += blockDim.x) us[e] = __ldcg(u + e);
    }
    __syncthreads();
    for (int li = threadIdx.x; li < nr; li += blockDim.x) {
        const int i = r0 + li;
        float a[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) a[c] = res[li * NB + c];
        if (far) {
            const float4 *prow = reinterpret_cast<const float4 *>(dm_pt_row(H, leaf, i));
            const int t4 = (sr + 3) >> 2;
            for (int v = 0; v < t4; ++v) {
                const float4 p = __ldg(prow + v);
                const float pv[4] = {p.x, p.y, p.z, p.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int t = 4 * v + e;
                    if (t < sr) {
#pragma unroll
                        for (int c = 0; c < NB; ++c) a[c] = fmaf(pv[e], us[t * NB + c], a[c]);
                    }
                }
            }
        }
        const int64_t dst = permuted ? st + i : (int64_t)H.perm[st + i];
#pragma unroll
        for (int c = 0; c < NB; ++c) y[(size_t)c * ldy + dst] = a[c];
    }
}

template <typename... KArgs, typename... Args>
cudaError_t launch_nb(void (*kern)(KArgs...), dim3 grid, unsigned block, size_t smem, cudaStream_t st,
                      unsigned cluster, bool pdl, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    unsigned na = 0;
    if (pdl) {
        at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[na].val.programmaticStreamSerializationAllowed = 1;
        ++na;
    }
    if (cluster > 1) {
        at[na].id = cudaLaunchAttributeClusterDimension;
        at[na].val.clusterDim.x = cluster;
        at[na].val.clusterDim.y = 1;
        at[na].val.clusterDim.z = 1;
        ++na;
    }
    cfg.attrs = at;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <int NB>
const void *tree_nb_fn() {
    return (const void *)tree_nb_kernel<NB>;
}

template <int NB>
cudaError_t run_nb(const DmHmat &H, const DmNbTree &T, const float *x, int64_t ldx, float *y, int64_t ldy,
                   bool permuted, cudaStream_t st) {
    const int nleaves = 1 << H.L;
    const int pm = permuted ? 1 : 0;
    const int m4max = (H.leaf_max + 3) & ~3;
    cudaError_t e;
    const size_t smA = sizeof(float) * (size_t)NB * m4max;
    const int rows_per_cta = 2 * (kNbLeafThreads / 32);
    const unsigned gy = (unsigned)((H.rank_hi + rows_per_cta - 1) / rows_per_cta);
    if ((e = dm_allow_smem((const void *)leaf_n2s_nb_kernel<NB>, smA)) != cudaSuccess) return e;
    leaf_n2s_nb_kernel<NB><<<dim3((unsigned)nleaves, gy > 0 ? gy : 1u), kNbLeafThreads, smA, st>>>(H, T, x, ldx, pm);
    dm_count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = dm_allow_smem(tree_nb_fn<NB>(), (size_t)T.smem)) != cudaSuccess) return e;
    if (T.ls >= 4 &&
        (e = cudaFuncSetAttribute(tree_nb_fn<NB>(), cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) !=
            cudaSuccess)
        return e;
    e = launch_nb(tree_nb_kernel<NB>, dim3(1u << T.ls), kNbTreeThreads, (size_t)T.smem, st, 1u << T.ls, true, H, T);
    dm_count_launches(1);
    if (e != cudaSuccess) return e;
    // items (row chunks of the leaf blocks) that fit one wave beside the cluster: every item
    // resident at once, so no second partial wave of items
    int chunks = (H.leaf_max + kNbNearRowsTarget - 1) / kNbNearRowsTarget;
    {
        static int occ = 0, sms = 0;
        if (occ == 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const size_t sm_hi = sizeof(float) * ((size_t)NB * m4max + (size_t)(kNbNearRowsTarget * NB + 3) +
                                                  (size_t)H.max_rank * NB);
            if (dm_allow_smem((const void *)near_nb_kernel<NB>, sm_hi) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, near_nb_kernel<NB>, kNbNearThreads, sm_hi) !=
                    cudaSuccess)
                occ = 0;
            cudaGetLastError();
        }
        const int resident = occ * sms - (1 << T.ls);
        if (occ > 0 && resident > 0) {
            const int fit = resident / nleaves;
            if (fit >= 1 && fit < chunks) chunks = fit;
        }
    }
    const int rows = (H.leaf_max + chunks - 1) / chunks;
    const int n_items = nleaves * chunks;
    const size_t smC = sizeof(float) * ((size_t)NB * m4max + (size_t)((rows * NB + 3) & ~3) + (size_t)H.rank_hi * NB);
    if ((e = dm_allow_smem((const void *)near_nb_kernel<NB>, smC)) != cudaSuccess) return e;
    e = launch_nb(near_nb_kernel<NB>, dim3((unsigned)n_items), kNbNearThreads, smC, st, 1u, true, H, T, x, ldx, y, ldy,
                  pm, rows, 1);
    dm_count_launches(1);
    return e;
}

}  // namespace

// Host layout of the NB-wide cluster pass: the tree is cut at level ls (3, else 4 when the
// device runs 16-CTA clusters); subtree nodes belong to their level-ls ancestor's CTA, and
// the nodes above the cut go, largest first, to the CTA with the least shared memory in use.
bool dm_nb_tree_layout(const std::vector<int32_t> &rk, int L, int nb, int budget_floats, DmNbLayout &out) {
    if (L < 1) return false;
    for (int ls_want = 3; ls_want <= 4; ++ls_want) {
        const int ls = L - 1 < ls_want ? L - 1 : ls_want;
        if (ls_want == 4 && (ls < 4 || !dm_tree_cluster_supported(16))) break;
        const int nc = 1 << ls, nnodes = (1 << (L + 1)) - 1, ninternal = (1 << L) - 1;
        auto r4 = [](int64_t v) { return (v + 3) & ~int64_t(3); };
        // metadata: int4 lay, int rank (padded), int2 own, int owner (padded) per node
        const int64_t meta = r4(4 * (int64_t)nnodes + ((nnodes + 3) & ~3) + 2 * (int64_t)nnodes + ((nnodes + 3) & ~3));
        if (meta > budget_floats / 2) return false;
        std::vector<int64_t> used(nc, meta);
        std::vector<int> owner(nnodes, 0);
        // operands and vector slots an internal node brings to its owner: its children's pair
        // slot, B, P, and its own [w | u] when it sits at or above the cut
        auto node_floats = [&](int n) {
            const int sl = rk[2 * n + 1], sr = rk[2 * n + 2];
            int64_t f = r4((int64_t)2 * (sl + sr) * nb) + r4((int64_t)sl * (sr | 1));
            if (n > 0) f += r4((int64_t)(sl + sr) * (rk[n] | 1));
            if (n > 0 && dm_level_of(n) <= ls) f += r4((int64_t)2 * rk[n] * nb);
            return f;
        };
        for (int n = 0; n < nnodes; ++n) {
            const int lv = dm_level_of(n);
            owner[n] = lv >= ls ? ((n + 1) >> (lv - ls)) - nc : -1;
        }
        for (int n = 0; n < ninternal; ++n)
            if (owner[n] >= 0) used[owner[n]] += node_floats(n);
        std::vector<int> top;
        for (int n = 0; n < nc - 1; ++n) top.push_back(n);
        std::sort(top.begin(), top.end(), [&](int a, int b) { return node_floats(a) > node_floats(b); });
        for (int n : top) {
            int best = 0;
            for (int c = 1; c < nc; ++c)
                if (used[c] < used[best]) best = c;
            owner[n] = best;
            used[best] += node_floats(n);
        }
        // offsets
        std::vector<int64_t> cur(nc, meta);
        out.lay.assign(nnodes, make_int4(-1, -1, -1, -1));
        out.own.assign(nnodes, make_int2(-1, -1));
        for (int n = 0; n < ninternal; ++n) {
            const int c = owner[n], lv = dm_level_of(n);
            const int sl = rk[2 * n + 1], sr = rk[2 * n + 2];
            const int64_t pair = r4((int64_t)2 * (sl + sr) * nb);
            if (lv >= ls) {
                out.lay[n].z = (int)cur[c];
                cur[c] += pair;
                if (lv == ls && n > 0) {
                    out.lay[n].w = (int)cur[c];
                    out.own[n] = make_int2((int)cur[c], (int)(cur[c] + (int64_t)rk[n] * nb));
                    cur[c] += r4((int64_t)2 * rk[n] * nb);
                }
            } else {
                out.lay[n].w = (int)cur[c];  // scratch copy of the children's pair
                cur[c] += pair;
                if (n > 0) {
                    out.lay[n].z = (int)cur[c];
                    out.own[n] = make_int2((int)cur[c], (int)(cur[c] + (int64_t)rk[n] * nb));
                    cur[c] += r4((int64_t)2 * rk[n] * nb);
                }
            }
            out.lay[n].y = (int)cur[c];
            cur[c] += r4((int64_t)sl * (sr | 1));
            if (n > 0) {
                out.lay[n].x = (int)cur[c];
                cur[c] += r4((int64_t)(sl + sr) * (rk[n] | 1));
            }
        }
        // nodes below the cut keep their own [w | u] in their parent's pair slot
        for (int n = 1; n < nnodes; ++n) {
            const int lv = dm_level_of(n);
            if (lv > ls) {
                const int p = (n - 1) >> 1, sl = rk[2 * p + 1], sr = rk[2 * p + 2];
                const bool left = (n & 1) != 0;
                const int64_t w = out.lay[p].z + (left ? 0 : (int64_t)sl * nb);
                out.own[n] = make_int2((int)w, (int)(w + (int64_t)(sl + sr) * nb));
            }
        }
        bool fits = true;
        int64_t mx = 0;
        out.img_off.assign(nc + 1, 0);
        for (int c = 0; c < nc; ++c) {
            cur[c] = r4(cur[c]);
            if (cur[c] > budget_floats) fits = false;
            mx = cur[c] > mx ? cur[c] : mx;
            out.img_off[c + 1] = out.img_off[c] + (int)cur[c];
        }
        if (!fits) continue;
        out.owner = owner;
        out.ls = ls;
        out.smem = (int)(mx * 4);
        return true;
    }
    return false;
}

cudaError_t dm_nb_tree_image(const DmHmat &H, const DmNbTree &T, cudaStream_t st) {
    tree_nb_image_kernel<<<dim3(1u << T.ls, 8u), 512, 0, st>>>(H, T);
    dm_count_launches(1);
    return cudaGetLastError();
}

cudaError_t dm_hmatvec_nb(const DmHmat &H, const DmNbTree &T, int nb, const float *x, int64_t ldx, float *y,
                          int64_t ldy, bool permuted, cudaStream_t st) {
    if (nb != T.nb || H.L < 1) return cudaErrorInvalidValue;
    switch (nb) {
        case 2: return run_nb<2>(H, T, x, ldx, y, ldy, permuted, st);
        case 3: return run_nb<3>(H, T, x, ldx, y, ldy, permuted, st);
        case 4: return run_nb<4>(H, T, x, ldx, y, ldy, permuted, st);
        default: return cudaErrorInvalidValue;
    }
}
