// k_htree.cu -- the hierarchical matvec y = K~ x of Eq. 2.18 as three chained launches.
//
//   A leaf_n2s_kernel     block per leaf: w_a = P_a x~(I_a) (leaf N2S).
//   B tree_kernel         one thread-block cluster: the whole upper tree (internal N2S,
//                         every S2S, internal S2N) with its operands staged in the
//                         cluster's shared memory, ending with the incoming skeleton
//                         potential u_a of every leaf.
//   C near_cached_kernel  row chunks of the stored leaf blocks streamed with 16-byte
//     near_otf_kernel     evict-first loads (or entries recomputed from the points), then
//                         the leaf S2N y~(I_a) += P_a^T u_a, each row written once.
//
// B and C use programmatic dependent launch: B starts while A runs and stages its
// operands (they do not depend on x), then waits for A's results; C starts while B
// runs, streams its near rows, and waits for B only before the leaf S2N. The near
// stream (the bulk of the bytes) therefore overlaps the whole latency-bound tree pass.
//
// The tree is cut at level ls: CTA c of the cluster owns the subtree under node
// 2^ls - 1 + c; the 2^ls - 1 nodes above ls are spread one per CTA and level. Inside a
// subtree every level synchronises within the CTA; the levels above ls take one cluster
// barrier each, with the children's vectors reached in the other CTAs' shared memory.
#include <cooperative_groups.h>

#include "dm_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kLeafThreads = 256;
constexpr int kTreeThreads = 1024;
constexpr int kNearThreads = 256;      // on-the-fly near items (thread per row)
constexpr int kNearCachedThreads = 256;  // cached near items: 6 CTAs per SM at <= 40 registers
constexpr int kNearCachedMinBlocks = 6;
constexpr int kNearRowsTarget = 136;     // rows of a leaf block per cached near item (about one wave)

__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ------------------------------------------------------------------ A: leaf N2S

__global__ void __launch_bounds__(kLeafThreads) leaf_n2s_kernel(DmHmat H, const float *__restrict__ x,
                                                                 int permuted) {
    grid_dep_launch();  // the tree pass may start staging its operands now
    extern __shared__ float4 smem4[];
    float *sx = reinterpret_cast<float *>(smem4);
    const int nleaves = 1 << H.L;
    const int node = nleaves - 1 + blockIdx.x;
    // blockIdx.y splits the leaf's basis rows over several CTAs (2 rows per warp each), so
    // no warp walks more than one pair of rows: this launch is on the critical path of the
    // matvec (the tree pass waits for it)
    const int s = H.ranks[node];
    const int row0 = blockIdx.y * 2 * (blockDim.x >> 5);
    if (row0 >= s) return;
    int64_t st, sz;
    dm_node_range(H.N, node, &st, &sz);
    const int m = (int)sz, m4 = (m + 3) & ~3;
    const float *P = H.P + (size_t)node * H.max_rank * H.ldp;
    float *out = H.what + (size_t)node * H.max_rank;
    // warp per pair of rows; each lane issues all 16-byte loads of both rows before the sums.
    // The first pair's loads go out before x is staged (they do not depend on it), so the
    // basis rows and x arrive in one round trip.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int c4 = m4 >> 2;  // float4 per row (<= 128 for leaves of up to 512 points)
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    auto load_pair = [&](int t, float4 (&ka)[4], float4 (&kb)[4], int base) {
        const bool two = t + 1 < s;
        const float4 *ra = reinterpret_cast<const float4 *>(P + (size_t)t * H.ldp);
        const float4 *rb = reinterpret_cast<const float4 *>(P + (size_t)(two ? t + 1 : t) * H.ldp);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = base + lane + 32 * u;
            ka[u] = q < c4 ? __ldg(ra + q) : zero;
            kb[u] = (two && q < c4) ? __ldg(rb + q) : zero;
        }
    };
    const int t0 = row0 + 2 * warp;
    float4 ka0[4], kb0[4];
    if (t0 < s) load_pair(t0, ka0, kb0, 0);
    for (int j = threadIdx.x; j < m4; j += blockDim.x) {
        float v = 0.f;
        if (j < m) v = permuted ? x[st + j] : x[H.perm[st + j]];
        sx[j] = v;
    }
    __syncthreads();
    const float4 *v4 = reinterpret_cast<const float4 *>(sx);
    auto finish_pair = [&](int t, const float4 (&ka)[4], const float4 (&kb)[4], int base, float &acc_a,
                           float &acc_b) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = base + lane + 32 * u;
            const float4 xv = q < c4 ? v4[q] : zero;
            acc_a = fmaf(ka[u].x, xv.x, fmaf(ka[u].y, xv.y, fmaf(ka[u].z, xv.z, fmaf(ka[u].w, xv.w, acc_a))));
            acc_b = fmaf(kb[u].x, xv.x, fmaf(kb[u].y, xv.y, fmaf(kb[u].z, xv.z, fmaf(kb[u].w, xv.w, acc_b))));
        }
    };
    auto store_pair = [&](int t, float acc_a, float acc_b) {
        acc_a = dm_warp_sum(acc_a);
        acc_b = dm_warp_sum(acc_b);
        if (lane == 0) {
            out[t] = acc_a;
            if (t + 1 < s) out[t + 1] = acc_b;
        }
    };
    if (t0 < s) {  // the first pair: its first 128 float4 per row were loaded before the staging
        float acc_a = 0.f, acc_b = 0.f;
        finish_pair(t0, ka0, kb0, 0, acc_a, acc_b);
        for (int base = 128; base < c4; base += 128) {  // rows longer than 512 floats
            float4 ka[4], kb[4];
            load_pair(t0, ka, kb, base);
            finish_pair(t0, ka, kb, base, acc_a, acc_b);
        }
        store_pair(t0, acc_a, acc_b);
    }
    for (int t = t0 + 2 * nw * (int)gridDim.y; t < s; t += 2 * nw * (int)gridDim.y) {
        float acc_a = 0.f, acc_b = 0.f;
        for (int base = 0; base < c4; base += 128) {
            float4 ka[4], kb[4];
            load_pair(t, ka, kb, base);
            finish_pair(t, ka, kb, base, acc_a, acc_b);
        }
        store_pair(t, acc_a, acc_b);
    }
}

// ------------------------------------------------------------------ B: upper tree in one cluster

// CTA of the cluster that owns node n: a subtree node belongs to the CTA of its level-ls
// ancestor; the top nodes are spread one per CTA and level (odd multiples of powers of two)
__host__ __device__ __forceinline__ int tree_owner(int n, int ls) {
    const int lv = dm_level_of(n), nc = 1 << ls;
    if (lv >= ls) return ((n + 1) >> (lv - ls)) - nc;
    const int i = n - ((1 << lv) - 1);
    return (2 * i + 1) * (nc >> (lv + 1));
}

// All operands and vectors of the tree pass live in the CTA's shared memory and are addressed
// by float offsets from its base `sm`: B of node n at lay[n].y (row-major, row stride s_r|1),
// P of node n at lay[n].x (column-major, column stride s_n|1). The children of an internal
// node share one slot [w_l | w_r | u_l | u_r]: at lay[n].z for a subtree node, at lay[n].w
// (a scratch copy) for a node above ls. A node at level ls has its own [w | u] at lay[n].w, a
// node above ls its own [w | u] at lay[n].z.

// out[obase + o] (=, or += when add) = sum_{k < nk} sm[abase + o ao + k ak] sm[vbase + k] for
// o < nout, by warps gw = 0..ngw-1 of a group: 8 outputs per warp pass, 4 lanes per output
__device__ __forceinline__ void grp_gemv(const float *sm, int abase, int ao, int ak, int nout, int nk, int vbase,
                                         float *out, int obase, bool add, int gw, int ngw, int lane) {
    const int q = lane >> 2, ql = lane & 3, ak4 = 4 * ak;
    for (int o0 = gw * 8; o0 < nout; o0 += ngw * 8) {
        const int o = o0 + q;
        float a0 = 0.f, a1 = 0.f;
        if (o < nout) {
            const float *pa = sm + abase + o * ao + ql * ak;
            const float *pv = sm + vbase + ql;
            int k = ql;
            for (; k + 4 < nk; k += 8) {
                a0 = fmaf(pa[0], pv[0], a0);
                a1 = fmaf(pa[ak4], pv[4], a1);
                pa += 2 * ak4;
                pv += 8;
            }
            if (k < nk) a0 = fmaf(pa[0], pv[0], a0);
        }
        float v = a0 + a1;
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        if (o < nout && ql == 0) out[obase + o] = add ? out[obase + o] + v : v;
    }
}

// S2S of the pair in slot `pr` ([w_l | w_r | u_l | u_r]): u_l = B w_r, u_r = B^T w_l
__device__ __forceinline__ void grp_s2s(const float *sm, int bo, int sl, int sr, int pr, float *out, int gw, int ngw,
                                        int lane) {
    const int rs = sr | 1, c = sl + sr;
    grp_gemv(sm, bo, rs, 1, sl, sr, pr + sl, out, pr + c, false, gw, ngw, lane);
    grp_gemv(sm, bo, 1, rs, sr, sl, pr, out, pr + c + sl, false, gw, ngw, lane);
}

// first node and node count of level lv inside the subtree under g (g at level ls)
__device__ __forceinline__ void level_nodes(int g, int ls, int lv, int *first, int *count) {
    *first = ((g + 1) << (lv - ls)) - 1;
    *count = 1 << (lv - ls);
}

// Build each CTA's shared-memory image in global memory once per compression: metadata
// (layout int4, rank, own w/u offsets per node), then every owned internal node's B and P in the layout
// the tree pass reads. Block c writes CTA c's image; the tree pass stages it with 16-byte
// copies.
__global__ void __launch_bounds__(512) tree_image_kernel(const __grid_constant__ DmHmat H, float *img,
                                                         const int *img_off) {
    const int ls = H.tree_ls, L = H.L, c = blockIdx.x;  // image c; blockIdx.y: a share of its nodes
    const int nnodes = (2 << L) - 1, ninternal = (1 << L) - 1;
    float *out = img + img_off[c];
    int4 *lay = reinterpret_cast<int4 *>(out);
    int *rk = reinterpret_cast<int *>(lay + nnodes);
    int2 *own = reinterpret_cast<int2 *>(rk + ((nnodes + 3) & ~3));
    if (blockIdx.y == 0)
        for (int n = threadIdx.x; n < nnodes; n += blockDim.x) {
            lay[n] = H.tlay[n];
            rk[n] = H.ranks[n];
            own[n] = H.town[n];
        }
    // a warp per owned node, the warps of all gridDim.y blocks of this image taking the owned
    // nodes in turn (the copies are independent: their global-memory latencies overlap)
    const int lane = threadIdx.x & 31, nw = (int)(blockDim.x >> 5) * (int)gridDim.y;
    const int warp = (int)blockIdx.y * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5);
    int mine = 0;  // owned nodes seen so far: the warp takes every nw-th
    for (int n = 0; n < ninternal; ++n) {
        if (tree_owner(n, ls) != c) continue;
        if ((mine++ % nw) != warp) continue;
        const int4 ln = H.tlay[n];
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

__global__ void __launch_bounds__(kTreeThreads) tree_kernel(const __grid_constant__ DmHmat H) {
    grid_dep_launch();  // the near stream does not depend on this pass until its leaf S2N
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    cg::cluster_group cl = cg::this_cluster();
    const int ls = H.tree_ls, L = H.L, nc = 1 << ls, R = H.max_rank;
    const int c = (int)cl.block_rank();
    const int g = nc - 1 + c;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nnodes = (2 << L) - 1;
    const int4 *lay = reinterpret_cast<const int4 *>(smem4);
    const int *rk = reinterpret_cast<const int *>(lay + nnodes);
    const int2 *own = reinterpret_cast<const int2 *>(rk + ((nnodes + 3) & ~3));
    auto own_w = [&](int n) { return own[n].x; };  // own w and u of node n (root excluded)
    auto own_u = [&](int n) { return own[n].y; };

    // 1. stage this CTA's image (metadata and operands; independent of x, so it overlaps the
    //    leaf N2S launch): contiguous 16-byte copies
    {
        const int o0 = H.timg_off[c], len = H.timg_off[c + 1] - o0;
        const float *src = H.timg + o0;
        for (int i = 4 * threadIdx.x; i < len; i += 4 * blockDim.x) dm_cp_async16(sm + i, src + i);
    }
    // 2. the leaves' weights come from the leaf N2S launch
    grid_dep_wait();
    dm_cp_async_wait_all();
    __syncthreads();
    {
        // a lane's loads are all issued before the first store (one round trip per row)
        int first, count;
        level_nodes(g, ls, L, &first, &count);
        for (int i = warp; i < count; i += nw) {
            const int n = first + i, w = own_w(n), len = rk[n];
            const float *src = H.what + (size_t)n * R;
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
    // 3. upward pass inside the subtree: the N2S chain alone (a level's nodes share the CTA's
    //    warps); the S2S products feed only the downward pass, so they leave the chain and run
    //    afterwards, every child pair of the subtree at once
    for (int lv = L - 1; lv >= ls; --lv) {
        int first, count;
        level_nodes(g, ls, lv, &first, &count);
        const int ngw = count >= nw ? 1 : nw / count;
        for (int i = warp / ngw; i < count; i += nw / ngw) {
            const int n = first + i, gw = warp % ngw;
            if (n == 0) continue;
            const int sl = rk[2 * n + 1], sr = rk[2 * n + 2], pr = lay[n].z;
            grp_gemv(sm, lay[n].x, 1, rk[n] | 1, rk[n], sl + sr, pr, sm, own_w(n), false, gw, ngw, lane);
        }
        __syncthreads();
    }
    {
        const int nsub = (1 << (L - ls)) - 1;  // internal nodes of the subtree (levels ls .. L-1)
        const int tasks = 2 * nsub;             // u_l = B w_r and u_r = B^T w_l of each pair
        const int ngw = tasks >= nw ? 1 : nw / tasks;
        for (int tk = warp / ngw; tk < tasks; tk += nw / ngw) {
            const int gw = warp % ngw, idx = tk >> 1;
            const int lvo = 31 - __clz(idx + 1);
            const int n = ((g + 1) << lvo) - 1 + (idx + 1 - (1 << lvo));
            const int sl = rk[2 * n + 1], sr = rk[2 * n + 2], pr = lay[n].z, bo = lay[n].y;
            const int rs = sr | 1, c = sl + sr;
            if ((tk & 1) == 0) grp_gemv(sm, bo, rs, 1, sl, sr, pr + sl, sm, pr + c, false, gw, ngw, lane);
            else grp_gemv(sm, bo, 1, rs, sr, sl, pr, sm, pr + c + sl, false, gw, ngw, lane);
        }
        __syncthreads();
    }
    // 4. the levels above ls: one node per CTA and level, all warps on it; the children's w
    //    are copied from the other CTAs' shared memory into the node's pair scratch
    if (nc > 1) {
        auto top_node = [&](int lv) {
            const int span = nc >> (lv + 1);
            if (c % span != 0 || ((c / span) & 1) == 0) return -1;
            return (1 << lv) - 1 + (c / span - 1) / 2;
        };
        for (int lv = ls - 1; lv >= 0; --lv) {
            cl.sync();
            const int n = top_node(lv);
            if (n >= 0) {
                const int l = 2 * n + 1, r = 2 * n + 2, sl = rk[l], sr = rk[r], cc = sl + sr;
                const int ol = tree_owner(l, ls), orr = tree_owner(r, ls);
                const int pr = lay[n].w;
                const float *wl = cl.map_shared_rank(sm + own_w(l), ol);
                const float *wr = cl.map_shared_rank(sm + own_w(r), orr);
                for (int j = threadIdx.x; j < cc; j += blockDim.x) sm[pr + j] = j < sl ? wl[j] : wr[j - sl];
                __syncthreads();
                grp_s2s(sm, lay[n].y, sl, sr, pr, sm, warp, nw, lane);
                if (n > 0) grp_gemv(sm, lay[n].x, 1, rk[n] | 1, rk[n], cc, pr, sm, own_w(n), false, warp, nw, lane);
                __syncthreads();
                float *ul = cl.map_shared_rank(sm + own_u(l), ol), *ur = cl.map_shared_rank(sm + own_u(r), orr);
                for (int j = threadIdx.x; j < cc; j += blockDim.x) {
                    const float v = sm[pr + cc + j];
                    if (j < sl) ul[j] = v;
                    else ur[j - sl] = v;
                }
            }
        }
        for (int lv = 1; lv < ls; ++lv) {
            cl.sync();
            const int n = top_node(lv);
            if (n >= 0) {
                const int l = 2 * n + 1, r = 2 * n + 2, sl = rk[l], sr = rk[r], cc = sl + sr, s = rk[n];
                const int pr = lay[n].w;  // the children's shares of P^T u_n go to the u part
                grp_gemv(sm, lay[n].x, s | 1, 1, cc, s, own_u(n), sm, pr + cc, false, warp, nw, lane);
                __syncthreads();
                float *ul = cl.map_shared_rank(sm + own_u(l), tree_owner(l, ls));
                float *ur = cl.map_shared_rank(sm + own_u(r), tree_owner(r, ls));
                for (int j = threadIdx.x; j < cc; j += blockDim.x) {
                    const float v = sm[pr + cc + j];
                    if (j < sl) ul[j] += v;
                    else ur[j - sl] += v;
                }
            }
        }
        cl.sync();
    }
    // 5. downward pass inside the subtree (the root has no P): the pair's u += P^T u_n
    for (int lv = ls; lv < L; ++lv) {
        int first, count;
        level_nodes(g, ls, lv, &first, &count);
        const int ngw = count >= nw ? 1 : nw / count;
        for (int i = warp / ngw; i < count; i += nw / ngw) {
            const int n = first + i, gw = warp % ngw;
            if (n == 0) continue;
            const int sl = rk[2 * n + 1], sr = rk[2 * n + 2], cc = sl + sr, s = rk[n];
            grp_gemv(sm, lay[n].x, s | 1, 1, cc, s, own_u(n), sm, lay[n].z + cc, true, gw, ngw, lane);
        }
        __syncthreads();
    }
    // 6. the leaves' potentials
    {
        int first, count;
        level_nodes(g, ls, L, &first, &count);
        for (int i = warp; i < count; i += nw) {
            const int n = first + i, u = own_u(n);
            for (int j = lane; j < rk[n]; j += 32) H.uhat[(size_t)n * R + j] = sm[u + j];
        }
    }
}

// ------------------------------------------------------------------ C: near field + leaf S2N

// geometry of near item `item` (leaf, chunk of `rows` rows): leaf index, leaf start, leaf
// size, first row, rows in the chunk (0 for an empty tail chunk of a shorter leaf)
struct NearItem {
    int leaf, m, r0, nr;
    int64_t st;
};
__device__ __forceinline__ NearItem near_item(const DmHmat &H, int item, int rows) {
    const int per_leaf = (H.leaf_max + rows - 1) / rows;
    NearItem it;
    it.leaf = item / per_leaf;
    const int chunk = item - it.leaf * per_leaf;
    int64_t sz;
    dm_node_range(H.N, (1 << H.L) - 1 + it.leaf, &it.st, &sz);
    it.m = (int)sz;
    it.r0 = chunk * rows;
    it.nr = it.r0 < it.m ? min(rows, it.m - it.r0) : 0;
    return it;
}

// Cached near field, one block per item (rows of one leaf block): x~(I_a) staged in shared
// memory, a warp per pair of rows with every 16-byte streaming load of both rows issued before
// the sums (rows of up to 512 floats), then the leaf S2N after waiting for the tree pass.
// Blocks use little shared memory and few registers, so all items are resident at once.
__global__ void __launch_bounds__(kNearCachedThreads, kNearCachedMinBlocks) near_cached_kernel(const __grid_constant__ DmHmat H,
                                                                    const float *__restrict__ x,
                                                                    float *__restrict__ y, int permuted, int rows,
                                                                    int far) {
    extern __shared__ float4 smem4[];
    const NearItem q = near_item(H, blockIdx.x, rows);
    if (q.nr == 0) return;
    float *sx = reinterpret_cast<float *>(smem4);
    const int m4max = (H.leaf_max + 3) & ~3;
    float *res = sx + m4max;
    const int m4 = (q.m + 3) & ~3;
    for (int j = threadIdx.x; j < m4; j += blockDim.x) {
        float v = 0.f;
        if (j < q.m) v = permuted ? x[q.st + j] : x[H.perm[q.st + j]];
        sx[j] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float *blk = H.Knear + ((size_t)q.leaf * H.leaf_max + q.r0) * H.ldk;
    const int q4 = m4 >> 2;
    const float4 *x4 = reinterpret_cast<const float4 *>(sx);
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = 2 * warp; i < q.nr; i += 2 * nw) {
        const bool two = i + 1 < q.nr;
        const float4 *ra = reinterpret_cast<const float4 *>(blk + (size_t)i * H.ldk);
        const float4 *rb = reinterpret_cast<const float4 *>(blk + (size_t)(two ? i + 1 : i) * H.ldk);
        float4 ka[4], kb[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int v = lane + 32 * t;
            ka[t] = v < q4 ? __ldcs(ra + v) : zero;
            kb[t] = (two && v < q4) ? __ldcs(rb + v) : zero;
        }
        float acc_a = 0.f, acc_b = 0.f;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int v = lane + 32 * t;
            const float4 xv = v < q4 ? x4[v] : zero;
            acc_a = fmaf(ka[t].x, xv.x, fmaf(ka[t].y, xv.y, fmaf(ka[t].z, xv.z, fmaf(ka[t].w, xv.w, acc_a))));
            acc_b = fmaf(kb[t].x, xv.x, fmaf(kb[t].y, xv.y, fmaf(kb[t].z, xv.z, fmaf(kb[t].w, xv.w, acc_b))));
        }
        acc_a = dm_warp_sum(acc_a);
        acc_b = dm_warp_sum(acc_b);
        if (lane == 0) {
            res[i] = acc_a;
            if (two) res[i + 1] = acc_b;
        }
    }
    __syncthreads();
    if (far) grid_dep_wait();  // the tree pass has written the leaves' u
    const int node = (1 << H.L) - 1 + q.leaf;
    const int sr = far ? __ldg(H.ranks + node) : 0;
    const float *u = H.uhat + (size_t)node * H.max_rank;
    for (int li = threadIdx.x; li < q.nr; li += blockDim.x) {
        const int i = q.r0 + li;
        float a0 = res[li], a1 = 0.f;
        if (far) {
            const float4 *prow = reinterpret_cast<const float4 *>(dm_pt_row(H, q.leaf, i));
            const int t4 = (sr + 3) >> 2;  // PT rows are zero beyond the rank
            for (int v = 0; v < t4; ++v) {
                const float4 p = __ldg(prow + v);
                const int j = 4 * v;
                const float u0 = __ldcg(u + j);
                const float u1 = j + 1 < sr ? __ldcg(u + j + 1) : 0.f;
                const float u2 = j + 2 < sr ? __ldcg(u + j + 2) : 0.f;
                const float u3 = j + 3 < sr ? __ldcg(u + j + 3) : 0.f;
                if (v & 1) a1 = fmaf(p.x, u0, fmaf(p.y, u1, fmaf(p.z, u2, fmaf(p.w, u3, a1))));
                else a0 = fmaf(p.x, u0, fmaf(p.y, u1, fmaf(p.z, u2, fmaf(p.w, u3, a0))));
            }
        }
        const float val = a0 + a1;
        if (permuted) y[q.st + i] = val;
        else y[H.perm[q.st + i]] = val;
    }
}

// On-the-fly near field (thread per row; entries s_i s_j 2^-|xs_i - xs_j|^2 from the staged
// points), then the leaf S2N after waiting for the tree pass. One block per item.
__global__ void __launch_bounds__(kNearThreads) near_otf_kernel(const __grid_constant__ DmHmat H,
                                                                 const float *__restrict__ x, float *__restrict__ y,
                                                                 int permuted, int rows, int far) {
    extern __shared__ float4 smem4[];
    const NearItem q = near_item(H, blockIdx.x, rows);
    if (q.nr == 0) return;
    const int m4max = (H.leaf_max + 3) & ~3, d = H.d;
    float *sx = reinterpret_cast<float *>(smem4);  // m4max: s_j x_j
    float *spts = sx + m4max;                      // m x d points
    for (int j = threadIdx.x; j < q.m; j += blockDim.x) {
        const float xv = permuted ? x[q.st + j] : x[H.perm[q.st + j]];
        sx[j] = H.sp[q.st + j] * xv;
    }
    for (int e = threadIdx.x; e < q.m * d; e += blockDim.x) spts[e] = H.Xs[q.st * d + e];
    __syncthreads();
    float acc = 0.f;
    const int li = threadIdx.x, i = q.r0 + li;
    if (li < q.nr) {
        if (d == 3) {
            const float x0 = spts[i * 3], x1 = spts[i * 3 + 1], x2 = spts[i * 3 + 2];
#pragma unroll 4
            for (int j = 0; j < q.m; ++j) {
                const float t0 = x0 - spts[j * 3], t1 = x1 - spts[j * 3 + 1], t2 = x2 - spts[j * 3 + 2];
                acc = fmaf(dm_ex2(-fmaf(t0, t0, fmaf(t1, t1, t2 * t2))), sx[j], acc);
            }
        } else {
            for (int j = 0; j < q.m; ++j) {
                float r2 = 0.f;
                for (int k = 0; k < d; ++k) {
                    const float t = spts[i * d + k] - spts[j * d + k];
                    r2 = fmaf(t, t, r2);
                }
                acc = fmaf(dm_ex2(-r2), sx[j], acc);
            }
        }
        acc *= H.sp[q.st + i];
    }
    if (far) grid_dep_wait();
    if (li >= q.nr) return;
    if (far) {
        const int node = (1 << H.L) - 1 + q.leaf;
        const int sr = __ldg(H.ranks + node);
        const float *u = H.uhat + (size_t)node * H.max_rank;
        const float *prow = dm_pt_row(H, q.leaf, i);
        for (int j = 0; j < sr; ++j) acc = fmaf(__ldg(prow + j), __ldcg(u + j), acc);
    }
    if (permuted) y[q.st + i] = acc;
    else y[H.perm[q.st + i]] = acc;
}

template <typename... KArgs, typename... Args>
cudaError_t launch_ex(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                      unsigned cluster, bool pdl, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
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

}  // namespace

bool dm_tree_cluster_supported(int ctas) {
    static int cached[2] = {-1, -1};  // 8, 16 CTAs (one device per process in practice)
    const int slot = ctas > 8 ? 1 : 0;
    if (cached[slot] >= 0) return cached[slot] != 0;
    int ok = 0;
    const size_t smem = (size_t)kTreeSmemBudget;
    if (dm_allow_smem((const void *)tree_kernel, smem) == cudaSuccess &&
        (ctas <= 8 || cudaFuncSetAttribute((const void *)tree_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                           1) == cudaSuccess)) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)ctas);
        cfg.blockDim = dim3(kTreeThreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at;
        at.id = cudaLaunchAttributeClusterDimension;
        at.val.clusterDim.x = (unsigned)ctas;
        at.val.clusterDim.y = 1;
        at.val.clusterDim.z = 1;
        cfg.attrs = &at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, (const void *)tree_kernel, &cfg) == cudaSuccess && n > 0) ok = 1;
    }
    cudaGetLastError();
    cached[slot] = ok;
    return ok != 0;
}

cudaError_t dm_tree_image(const DmHmat &H, cudaStream_t st) {
    if (!H.tree_ok) return cudaSuccess;
    tree_image_kernel<<<dim3(1u << H.tree_ls, 8u), 512, 0, st>>>(H, H.timg, H.timg_off);
    dm_count_launches(1);
    return cudaGetLastError();
}

int dm_near_item_rows(int near_mode, int leaf_max) {
    if (near_mode == DM_NEAR_CACHED) {
        const int chunks = (leaf_max + kNearRowsTarget - 1) / kNearRowsTarget;
        return (leaf_max + chunks - 1) / chunks;
    }
    const int chunks = (leaf_max + kNearThreads - 1) / kNearThreads;
    return (leaf_max + chunks - 1) / chunks;
}

cudaError_t dm_hmatvec(const DmHmat &H, int near_mode, const float *x, float *y, bool permuted, cudaStream_t st) {
    if (H.L > 0 && !H.tree_ok) return dm_hmatvec_chain(H, near_mode, x, y, permuted, st);
    const int nleaves = 1 << H.L;
    const bool far = H.L > 0;
    const int pm = permuted ? 1 : 0;
    cudaError_t e;
    if (far) {
        const size_t smA = sizeof(float) * (size_t)((H.leaf_max + 3) & ~3);
        const int rows_per_cta = 2 * (kLeafThreads / 32);
        const unsigned gy = (unsigned)((H.rank_hi + rows_per_cta - 1) / rows_per_cta);
        leaf_n2s_kernel<<<dim3((unsigned)nleaves, gy > 0 ? gy : 1u), kLeafThreads, smA, st>>>(H, x, pm);
        dm_count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = dm_allow_smem((const void *)tree_kernel, (size_t)H.tree_smem)) != cudaSuccess) return e;
        e = launch_ex(tree_kernel, 1u << H.tree_ls, kTreeThreads, (size_t)H.tree_smem, st, 1u << H.tree_ls, true, H);
        dm_count_launches(1);
        if (e != cudaSuccess) return e;
    }
    const int rows = dm_near_item_rows(near_mode, H.leaf_max);
    const int n_items = nleaves * ((H.leaf_max + rows - 1) / rows);
    const int m4max = (H.leaf_max + 3) & ~3;
    if (near_mode == DM_NEAR_CACHED) {
        const size_t smC = sizeof(float) * ((size_t)m4max + (size_t)((rows + 3) & ~3));
        if ((e = dm_allow_smem((const void *)near_cached_kernel, smC)) != cudaSuccess) return e;
        e = launch_ex(near_cached_kernel, (unsigned)n_items, kNearCachedThreads, smC, st, 1u, far, H, x, y, pm, rows,
                      far ? 1 : 0);
    } else {
        const size_t smC = sizeof(float) * ((size_t)m4max + (size_t)H.leaf_max * H.d);
        if ((e = dm_allow_smem((const void *)near_otf_kernel, smC)) != cudaSuccess) return e;
        e = launch_ex(near_otf_kernel, (unsigned)n_items, kNearThreads, smC, st, 1u, far, H, x, y, pm, rows,
                      far ? 1 : 0);
    }
    dm_count_launches(1);
    return e;
}
