// k_hmatvec.cu -- the hierarchical matvec y = K~ x of Eq. 2.18 (K~ = D + UV).
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
constexpr int kHWarps = kHThreads / 32;
constexpr int kCachedRowsPerItem = 32;   // rows of one leaf block per near item (cached)

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

__global__ void __launch_bounds__(kHThreads) near_up_kernel(DmHmat H, const float *__restrict__ x, int permuted,
                                                            int near_mode, int near_rows) {
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    __shared__ int s_go;
    const int nleaves = 1 << H.L;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m4max = (H.leaf_max + 3) & ~3;

    if ((int)blockIdx.x < nleaves) {
        // ------------------------------------------------ leaf N2S, then climb
        const int leaf = blockIdx.x;
        int node = nleaves - 1 + leaf;
        int64_t st, sz;
        dm_node_range(H.N, node, &st, &sz);
        const int m = (int)sz, m4 = (m + 3) & ~3;
        float *sx = sm;                          // m4max
        float *sw = sm + m4max;                  // 2 * max_rank (+pad): children weights
        stage_x(H, x, permuted != 0, st, m, m4, sx);
        __syncthreads();
        const int s_leaf = H.ranks[node];
        gemv_rows(H.P + (size_t)node * H.max_rank * H.ldp, H.ldp, s_leaf, m, sx,
                  H.what + (size_t)node * H.max_rank, nullptr);
        if (H.L == 0) return;
        for (;;) {
            // publish this node's weights, then count the arrival at the parent
            __threadfence();
            __syncthreads();
            const int parent = (node - 1) >> 1;
            if (threadIdx.x == 0) {
                const unsigned old = atomicAdd(H.cnt + parent, 1u);
                s_go = (old == 1u);
                if (old == 1u) H.cnt[parent] = 0u;  // both children arrived: reset for the next call
                __threadfence();
            }
            __syncthreads();
            if (!s_go) return;
            node = parent;
            const int l = 2 * node + 1, r = 2 * node + 2;
            const int sl = H.ranks[l], sr = H.ranks[r];
            const int c = sl + sr, c4 = (c + 3) & ~3;
            for (int j = threadIdx.x; j < c4; j += blockDim.x) {
                float v = 0.f;
                if (j < sl) v = __ldcg(H.what + (size_t)l * H.max_rank + j);
                else if (j < c) v = __ldcg(H.what + (size_t)r * H.max_rank + (j - sl));
                sw[j] = v;
            }
            __syncthreads();
            // S2S: u_l = B w_r (warp per row of B), u_r = B^T w_l (thread per column of B)
            const float *Bn = H.B + (size_t)node * H.max_rank * H.max_rank;
            for (int a = warp; a < sl; a += kHWarps) {
                float acc = 0.f;
                for (int b = lane; b < sr; b += 32) acc = fmaf(__ldg(Bn + (size_t)a * sr + b), sw[sl + b], acc);
                acc = dm_warp_sum(acc);
                if (lane == 0) H.uhat[(size_t)l * H.max_rank + a] = acc;
            }
            for (int b = threadIdx.x; b < sr; b += blockDim.x) {
                float acc = 0.f;
                for (int a = 0; a < sl; ++a) acc = fmaf(__ldg(Bn + (size_t)a * sr + b), sw[a], acc);
                H.uhat[(size_t)r * H.max_rank + b] = acc;
            }
            if (node == 0) return;
            // N2S of the internal node
            gemv_rows(H.P + (size_t)node * H.max_rank * H.ldp, H.ldp, H.ranks[node], c, sw,
                      H.what + (size_t)node * H.max_rank, nullptr);
        }
    }

    // ---------------------------------------------------- near field
    const int item = blockIdx.x - nleaves;
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
        // two rows per warp pass for memory-level parallelism
        for (int i = r0 + 2 * warp; i < r1; i += 2 * kHWarps) {
            const bool two = (i + 1) < r1;
            const float *ra = blk + (size_t)i * H.ldk;
            const float *rb = blk + (size_t)(two ? i + 1 : i) * H.ldk;
            float acc_a = 0.f, acc_b = 0.f;
            for (int q = lane; q < m4q; q += 32) {
                const float4 ka = ldcs4(ra + 4 * q);
                const float4 kb = ldcs4(rb + 4 * q);
                const float4 xv = *reinterpret_cast<const float4 *>(sx + 4 * q);
                acc_a = fmaf(ka.x, xv.x, acc_a);
                acc_a = fmaf(ka.y, xv.y, acc_a);
                acc_a = fmaf(ka.z, xv.z, acc_a);
                acc_a = fmaf(ka.w, xv.w, acc_a);
                acc_b = fmaf(kb.x, xv.x, acc_b);
                acc_b = fmaf(kb.y, xv.y, acc_b);
                acc_b = fmaf(kb.z, xv.z, acc_b);
                acc_b = fmaf(kb.w, xv.w, acc_b);
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

__global__ void __launch_bounds__(kHThreads) down_kernel(DmHmat H, float *__restrict__ y, int permuted) {
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    float *ta = sm, *tb = sm + H.max_rank;
    const int leaf = blockIdx.x;
    const int nleaves = 1 << H.L;
    const int node_leaf = nleaves - 1 + leaf;
    int64_t st, sz;
    dm_node_range(H.N, node_leaf, &st, &sz);
    const int m = (int)sz;
    if (H.L == 0) {
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const float v = H.ynear[st + i];
            if (permuted) y[st + i] = v;
            else y[H.perm[st + i]] = v;
        }
        return;
    }
    // ancestor at level 1 .. L of this leaf: node(l) = ((node_leaf + 1) >> (L - l)) - 1
    int node = ((node_leaf + 1) >> (H.L - 1)) - 1;
    int s = H.ranks[node];
    for (int j = threadIdx.x; j < s; j += blockDim.x) ta[j] = H.uhat[(size_t)node * H.max_rank + j];
    __syncthreads();
    for (int lvl = 2; lvl <= H.L; ++lvl) {
        const int child = ((node_leaf + 1) >> (H.L - lvl)) - 1;
        const int off = (child == 2 * node + 2) ? H.ranks[2 * node + 1] : 0;
        const int sc = H.ranks[child];
        const float *Pn = H.P + (size_t)node * H.max_rank * H.ldp;
        for (int j = threadIdx.x; j < sc; j += blockDim.x) {
            float acc = H.uhat[(size_t)child * H.max_rank + j];
            for (int t = 0; t < s; ++t) acc = fmaf(__ldg(Pn + (size_t)t * H.ldp + off + j), ta[t], acc);
            tb[j] = acc;
        }
        __syncthreads();
        float *tmp = ta;
        ta = tb;
        tb = tmp;
        node = child;
        s = sc;
    }
    // leaf S2N and output
    const float *Pl = H.P + (size_t)node_leaf * H.max_rank * H.ldp;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        float acc = H.ynear[st + i];
        for (int t = 0; t < s; ++t) acc = fmaf(__ldg(Pl + (size_t)t * H.ldp + i), ta[t], acc);
        if (permuted) y[st + i] = acc;
        else y[H.perm[st + i]] = acc;
    }
}

}  // namespace

int dm_near_rows(int near_mode, int leaf_max) {
    if (near_mode == DM_NEAR_CACHED) return kCachedRowsPerItem;
    const int chunks = (leaf_max + kHThreads - 1) / kHThreads;
    return (leaf_max + chunks - 1) / chunks;
}

cudaError_t dm_hmatvec(const DmHmat &H, int near_mode, const float *x, float *y, bool permuted, cudaStream_t st) {
    const int nleaves = 1 << H.L;
    const int rows = dm_near_rows(near_mode, H.leaf_max);
    const int per_leaf = (H.leaf_max + rows - 1) / rows;
    const int m4max = (H.leaf_max + 3) & ~3;
    size_t smem1 = sizeof(float) * (size_t)(m4max + 2 * H.max_rank + 4);
    if (near_mode != DM_NEAR_CACHED) {
        size_t s2 = sizeof(float) * (size_t)(m4max + H.leaf_max * H.d);
        if (s2 > smem1) smem1 = s2;
    }
    static thread_local size_t configured = 0;
    if (smem1 > 48 * 1024 && smem1 > configured) {
        cudaError_t e = cudaFuncSetAttribute(near_up_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1);
        if (e != cudaSuccess) return e;
        configured = smem1;
    }
    near_up_kernel<<<nleaves + nleaves * per_leaf, kHThreads, smem1, st>>>(H, x, permuted ? 1 : 0, near_mode, rows);
    dm_count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    down_kernel<<<nleaves, kHThreads, sizeof(float) * 2 * H.max_rank, st>>>(H, y, permuted ? 1 : 0);
    dm_count_launches(1);
    return cudaGetLastError();
}
