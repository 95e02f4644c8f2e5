// k_hblock.cu -- the hierarchical matvec Y = K~ X for a block of nb right-hand sides
// (Eq. 2.18 applied to several vectors at once: the matmat of the LinearOperator in
// Section 3.3, and the operator of block Lanczos).
//
// Every operand is read once per block instead of once per vector, which turns the
// near field -- the bulk of the bytes -- from a matrix-vector stream into a small GEMM per
// leaf, C_a = K(I_a, I_a) X(I_a, :). Vectors live in a padded leaf layout: column c of a
// block holds leaf a's entries at [a * ldk, a * ldk + m_a), zero up to (a + 1) * ldk, so
// every leaf segment starts on a 16-byte boundary.
//
//   permute_in   X(orig order) -> Xb (padded leaf layout)
//   leaf N2S     W_a = P_a Xb(I_a)                              (block per leaf)
//   up(lv)       S2S U_l = B W_r, U_r = B^T W_l; N2S W_n = P_n [W_l; W_r]  (block per node)
//   down(lv)     [U_l; U_r] += P_n^T U_n                        (block per node)
//   near         Yb(I_a) = K(I_a, I_a) Xb(I_a)                  (register-tiled FP32 GEMM)
//   s2n_out      Y = Yb(I_a) + P_a^T U_a, scattered to the output layout
//
// The near GEMM does not depend on the tree passes, so it runs on a second stream while
// the latency-bound chain of tree launches proceeds; s2n_out joins the two.
#include "dm_internal.cuh"

namespace {

constexpr int kBlkThreads = 256;
constexpr int kTreeLvThreads = 512;  // leaf N2S and the per-level tree kernels (latency bound: more warps)
constexpr int kColTile = 32;  // right-hand sides per block of the tree kernels (a lane each)

// start and size of leaf `a`
__device__ __forceinline__ void leaf_range(const DmHmat &H, int a, int64_t *st, int *m) {
    int64_t s0, sz;
    dm_node_range(H.N, (1 << H.L) - 1 + a, &s0, &sz);
    *st = s0;
    *m = (int)sz;
}

// ------------------------------------------------------------------ layout changes

// Xb[c][a ldk + j] = x[c ldin + perm[st_a + j]] (perm == nullptr: x is in position order);
// a CTA per (leaf a, column c), zero padding past the leaf
__global__ void blk_permute_in_kernel(const __grid_constant__ DmHmat H, const float *__restrict__ x, int64_t ldin,
                                      const int32_t *__restrict__ perm, int nb, float *__restrict__ Xb,
                                      int64_t ldx) {
    const int a = blockIdx.x, c = blockIdx.y;
    int64_t st;
    int m;
    leaf_range(H, a, &st, &m);
    const float *xc = x + (size_t)c * ldin;
    float *out = Xb + (size_t)c * ldx + (size_t)a * H.ldk;
    for (int j = threadIdx.x; j < H.ldk; j += blockDim.x) {
        float v = 0.f;
        if (j < m) v = xc[perm ? perm[st + j] : st + j];
        out[j] = v;
    }
}

// ------------------------------------------------------------------ tree passes

constexpr int kVs = kColTile + 1;  // shared-memory row stride of staged vectors (conflict-free)

// out[o][lane] (= or +=) sum_k A(o, k) V[k][lane] for o < nout, where A(o, k) = A[o ao + k ak]
// (global memory) and V is nk x kColTile in shared memory (row stride kVs). A warp takes four
// output rows at a time: its lanes load 32 consecutive A(o, k) of each of the four rows at
// once and broadcast them by shuffles, so the four accumulation chains run side by side and
// a row costs nk / 32 memory round trips shared with three others.
__device__ __forceinline__ void blk_gemm_rows(const float *__restrict__ A, int ao, int ak, int nout, int nk,
                                              const float *V, float *out, int ldo, bool add, int ncol) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o0 = 4 * warp; o0 < nout; o0 += 4 * nw) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k0 = 0; k0 < nk; k0 += 32) {
            const int kk = k0 + lane;
            float av[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                av[q] = (o0 + q < nout && kk < nk) ? __ldg(A + (size_t)(o0 + q) * ao + (size_t)kk * ak) : 0.f;
            const int kn = nk - k0 < 32 ? nk - k0 : 32;
            for (int t = 0; t < kn; ++t) {
                const float v = V[(k0 + t) * kVs + lane];
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] = fmaf(__shfl_sync(DM_FULL, av[q], t), v, acc[q]);
            }
        }
        if (lane < ncol) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (o0 + q < nout) {
                    float *dst = out + (size_t)(o0 + q) * ldo + lane;
                    *dst = add ? *dst + acc[q] : acc[q];
                }
            }
        }
    }
}

// leaf N2S: W_a[t][c] = sum_j P_a[t][j] Xb[c][a ldk + j]; grid (nleaves, column groups)
__global__ void __launch_bounds__(kTreeLvThreads) blk_leaf_n2s_kernel(const __grid_constant__ DmHmat H,
                                                                   const float *__restrict__ Xb, int64_t ldx,
                                                                   int nb, float *__restrict__ Wb) {
    extern __shared__ float sm[];
    const int a = blockIdx.x, c0 = blockIdx.y * kColTile, ncol = min(kColTile, nb - c0);
    const int node = (1 << H.L) - 1 + a;
    int64_t st;
    int m;
    leaf_range(H, a, &st, &m);
    // coalesced along the leaf's positions j, transposed into rows of kVs floats
    for (int e = threadIdx.x; e < m * kColTile; e += blockDim.x) {
        const int c = e / m, j = e - c * m;
        sm[j * kVs + c] = c < ncol ? Xb[(size_t)(c0 + c) * ldx + (size_t)a * H.ldk + j] : 0.f;
    }
    __syncthreads();
    const int s = H.ranks[node];
    blk_gemm_rows(H.P + (size_t)node * H.max_rank * H.ldp, H.ldp, 1, s, m, sm,
                  Wb + (size_t)node * H.max_rank * nb + c0, nb, false, ncol);
}

// one level of the upward pass (nodes of level lv): S2S of the children pair, then the
// node's own N2S (not at the root)
__global__ void __launch_bounds__(kTreeLvThreads) blk_up_kernel(const __grid_constant__ DmHmat H, int lv, int nb,
                                                             float *__restrict__ Wb, float *__restrict__ Ub) {
    extern __shared__ float sm[];
    const int n = (1 << lv) - 1 + blockIdx.x, c0 = blockIdx.y * kColTile, ncol = min(kColTile, nb - c0);
    const int l = 2 * n + 1, r = 2 * n + 2;
    const int sl = H.ranks[l], sr = H.ranks[r], cc = sl + sr;
    const size_t R = (size_t)H.max_rank * nb;
    for (int e = threadIdx.x; e < cc * kColTile; e += blockDim.x) {
        const int k = e / kColTile, c = e - k * kColTile;
        float v = 0.f;
        if (c < ncol) v = k < sl ? Wb[l * R + (size_t)k * nb + c0 + c] : Wb[r * R + (size_t)(k - sl) * nb + c0 + c];
        sm[k * kVs + c] = v;
    }
    __syncthreads();
    const float *Bn = H.B + (size_t)n * H.max_rank * H.max_rank;  // s_l x s_r, row-major
    // U_l = B W_r, U_r = B^T W_l (written, not accumulated: the downward pass adds later)
    blk_gemm_rows(Bn, sr, 1, sl, sr, sm + sl * kVs, Ub + l * R + c0, nb, false, ncol);
    blk_gemm_rows(Bn, 1, sr, sr, sl, sm, Ub + r * R + c0, nb, false, ncol);
    if (n > 0)
        blk_gemm_rows(H.P + (size_t)n * H.max_rank * H.ldp, H.ldp, 1, H.ranks[n], cc, sm, Wb + n * R + c0, nb,
                      false, ncol);
}

// one level of the downward pass (nodes of level lv >= 1): [U_l; U_r] += P_n^T U_n
__global__ void __launch_bounds__(kTreeLvThreads) blk_down_kernel(const __grid_constant__ DmHmat H, int lv, int nb,
                                                               float *__restrict__ Ub) {
    extern __shared__ float sm[];
    const int n = (1 << lv) - 1 + blockIdx.x, c0 = blockIdx.y * kColTile, ncol = min(kColTile, nb - c0);
    const int l = 2 * n + 1, r = 2 * n + 2;
    const int s = H.ranks[n], sl = H.ranks[l], sr = H.ranks[r];
    const size_t R = (size_t)H.max_rank * nb;
    for (int e = threadIdx.x; e < s * kColTile; e += blockDim.x) {
        const int t = e / kColTile, c = e - t * kColTile;
        sm[t * kVs + c] = c < ncol ? Ub[n * R + (size_t)t * nb + c0 + c] : 0.f;
    }
    __syncthreads();
    const float *Pn = H.P + (size_t)n * H.max_rank * H.ldp;  // s x (s_l + s_r), row-major
    blk_gemm_rows(Pn, 1, H.ldp, sl, s, sm, Ub + l * R + c0, nb, true, ncol);
    blk_gemm_rows(Pn + sl, 1, H.ldp, sr, s, sm, Ub + r * R + c0, nb, true, ncol);
}

// ------------------------------------------------------------------ near field (FP32 GEMM)

// Work item = (leaf, chunk of RT rows) x (CT columns). 256 threads, each a 4 x 4 register
// tile: rows rg + q RT/4 (q < 4), columns 4 cg .. 4 cg + 3. The K-dimension runs over the
// leaf's columns in steps of 32, double buffered: the stored block rows (cached) arrive by
// 16-byte cp.async with zero fill past the block; on-the-fly entries are computed into the
// same buffer from the points.
constexpr int kNearKStep = 32;
constexpr int kKsStride = kNearKStep + 4;  // 36 floats: 16-byte rows, conflict-free for the row mapping

__device__ __forceinline__ void cp_async16_zfill(void *smem, const void *gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <int CT>
__global__ void __launch_bounds__(kBlkThreads) blk_near_kernel(const __grid_constant__ DmHmat H, int onthefly,
                                                               const float *__restrict__ Xb, int64_t ldx, int nb,
                                                               float *__restrict__ Yb, int chunks) {
    constexpr int RT = 4096 / CT;  // rows per item
    constexpr int NCG = CT / 4;    // column groups
    extern __shared__ float4 smem4[];
    float *Ks = reinterpret_cast<float *>(smem4);  // [2][RT][kKsStride]
    float *Xs = Ks + 2 * RT * kKsStride;           // [2][kNearKStep][CT]
    const int a = blockIdx.x / chunks, chunk = blockIdx.x - a * chunks;
    const int c0 = blockIdx.y * CT, ncol = min(CT, nb - c0);
    int64_t st;
    int m;
    leaf_range(H, a, &st, &m);
    const int r0 = chunk * RT;
    if (r0 >= m) return;
    const int nr = min(RT, m - r0);
    const int m4 = (m + 3) & ~3;
    const int nsteps = (m4 + kNearKStep - 1) / kNearKStep;
    const int tid = threadIdx.x, cg = tid % NCG, rg = tid / NCG;
    const float *blk = H.Knear + ((size_t)a * H.leaf_max + r0) * H.ldk;
    const float *xseg = Xb + (size_t)a * H.ldk;

    auto stage = [&](int step, int buf) {
        const int j0 = step * kNearKStep;
        float *ks = Ks + buf * RT * kKsStride;
        float *xs = Xs + buf * kNearKStep * CT;
        if (!onthefly) {
            // RT rows x 8 float4 per row
            for (int e = tid; e < RT * (kNearKStep / 4); e += kBlkThreads) {
                const int r = e >> 3, q = e & 7, j = j0 + 4 * q;
                const bool ok = r < nr && j < m4;
                cp_async16_zfill(ks + r * kKsStride + 4 * q, ok ? blk + (size_t)r * H.ldk + j : blk, ok);
            }
        } else {
            const int d = H.d;
            for (int e = tid; e < RT * kNearKStep; e += kBlkThreads) {
                const int r = e / kNearKStep, jj = e - r * kNearKStep, j = j0 + jj;
                float v = 0.f;
                if (r < nr && j < m) {
                    const float *xi = H.Xs + (size_t)(st + r0 + r) * d, *xj = H.Xs + (size_t)(st + j) * d;
                    float r2 = 0.f;
                    for (int k = 0; k < d; ++k) {
                        const float t = __ldg(xi + k) - __ldg(xj + k);
                        r2 = fmaf(t, t, r2);
                    }
                    v = __ldg(H.sp + st + r0 + r) * __ldg(H.sp + st + j) * dm_ex2(-r2);
                }
                ks[r * kKsStride + jj] = v;
            }
        }
        // X: kNearKStep rows x CT columns, transposed from the column-major block (4-byte copies)
        for (int e = tid; e < kNearKStep * CT; e += kBlkThreads) {
            const int c = e / kNearKStep, jj = e - c * kNearKStep, j = j0 + jj;
            const bool ok = c < ncol && j < m4;
            const unsigned s = (unsigned)__cvta_generic_to_shared(xs + jj * CT + c);
            const float *src = ok ? xseg + (size_t)(c0 + c) * ldx + j : xseg;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(src), "r"(ok ? 4 : 0)
                         : "memory");
        }
        cp_async_commit();
    };

    float acc[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[q][u] = 0.f;

    stage(0, 0);
    for (int step = 0; step < nsteps; ++step) {
        const int buf = step & 1;
        if (step + 1 < nsteps) {
            stage(step + 1, buf ^ 1);
            cp_async_wait1();
        } else {
            cp_async_wait0();
        }
        __syncthreads();
        const float *ks = Ks + buf * RT * kKsStride;
        const float *xs = Xs + buf * kNearKStep * CT;
#pragma unroll 8
        for (int jj = 0; jj < kNearKStep; ++jj) {
            const float4 xv = *reinterpret_cast<const float4 *>(xs + jj * CT + 4 * cg);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float kv = ks[(rg + q * (RT / 4)) * kKsStride + jj];
                acc[q][0] = fmaf(kv, xv.x, acc[q][0]);
                acc[q][1] = fmaf(kv, xv.y, acc[q][1]);
                acc[q][2] = fmaf(kv, xv.z, acc[q][2]);
                acc[q][3] = fmaf(kv, xv.w, acc[q][3]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = rg + q * (RT / 4);
        if (r >= nr) continue;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int c = 4 * cg + u;
            if (c < ncol) Yb[(size_t)(c0 + c) * ldx + (size_t)a * H.ldk + r0 + r] = acc[q][u];
        }
    }
}

// leaf S2N and output: y[c][out(i)] = Yb[c][a ldk + i] + sum_t PT_a[i][t] U_a[t][c]
// out(i) = perm[st + i] (original order), st + i (position order, posout), or the padded
// position a ldk + i (may alias Yb); column stride ldo. A thread per row i of the leaf, 32
// accumulators (the column group); U_a is staged in shared memory and read as broadcasts,
// so the reads of Yb and the position-order writes are coalesced along the rows.
__global__ void __launch_bounds__(kBlkThreads) blk_s2n_out_kernel(const __grid_constant__ DmHmat H,
                                                                  const float *Yb, int64_t ldx, int nb,
                                                                  const float *__restrict__ Ub, int far,
                                                                  const int32_t *__restrict__ perm, int posout,
                                                                  float *y, int64_t ldo) {
    extern __shared__ float sm[];
    const int a = blockIdx.x, c0 = blockIdx.y * kColTile, ncol = min(kColTile, nb - c0);
    const int node = (1 << H.L) - 1 + a;
    int64_t st;
    int m;
    leaf_range(H, a, &st, &m);
    const int s = far ? H.ranks[node] : 0;
    const size_t R = (size_t)H.max_rank * nb;
    for (int e = threadIdx.x; e < s * kColTile; e += blockDim.x) {
        const int t = e / kColTile, c = e - t * kColTile;
        sm[t * kColTile + c] = c < ncol ? Ub[node * R + (size_t)t * nb + c0 + c] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        float acc[kColTile];
#pragma unroll
        for (int c = 0; c < kColTile; ++c) acc[c] = 0.f;
        const float *pt = dm_pt_row(H, a, i);
        for (int t = 0; t < s; ++t) {
            const float p = __ldg(pt + t);
            const float4 *u4 = reinterpret_cast<const float4 *>(sm + t * kColTile);
#pragma unroll
            for (int q = 0; q < kColTile / 4; ++q) {
                const float4 u = u4[q];
                acc[4 * q] = fmaf(p, u.x, acc[4 * q]);
                acc[4 * q + 1] = fmaf(p, u.y, acc[4 * q + 1]);
                acc[4 * q + 2] = fmaf(p, u.z, acc[4 * q + 2]);
                acc[4 * q + 3] = fmaf(p, u.w, acc[4 * q + 3]);
            }
        }
        const int64_t dst = perm ? (int64_t)perm[st + i] : (posout ? st + i : (int64_t)a * H.ldk + i);
#pragma unroll
        for (int c = 0; c < kColTile; ++c) {
            if (c < ncol) {
                const size_t cc = (size_t)(c0 + c);
                y[cc * ldo + dst] = Yb[cc * ldx + (size_t)a * H.ldk + i] + acc[c];
            }
        }
    }
}

template <int CT>
cudaError_t launch_near(const DmHmat &H, int onthefly, const float *Xb, int64_t ldx, int nb, float *Yb,
                        cudaStream_t st) {
    constexpr int RT = 4096 / CT;
    const int chunks = (H.leaf_max + RT - 1) / RT;
    const size_t smem = sizeof(float) * (2 * (size_t)RT * kKsStride + 2 * (size_t)kNearKStep * CT);
    cudaError_t e = dm_allow_smem((const void *)blk_near_kernel<CT>, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((1 << H.L) * chunks), (unsigned)((nb + CT - 1) / CT));
    blk_near_kernel<CT><<<grid, kBlkThreads, smem, st>>>(H, onthefly, Xb, ldx, nb, Yb, chunks);
    dm_count_launches(1);
    return cudaGetLastError();
}

}  // namespace

int64_t dm_block_ldx(const DmHmat &H) { return (int64_t)(1 << H.L) * H.ldk; }

cudaError_t dm_hmatvec_block(const DmHmat &H, int near_mode, int near_prec, const DmBlockWork &W, int nb,
                             const float *x, int64_t ldin, const int32_t *perm_in, bool x_padded, float *y,
                             int64_t ldo, int y_layout, cudaStream_t st) {
    if (nb < 1 || nb > W.nb_max) return cudaErrorInvalidValue;
    const int nleaves = 1 << H.L;
    const int64_t ldx = W.ldx;
    const float *Xb = x;
    cudaError_t e;
    if (!x_padded) {
        blk_permute_in_kernel<<<dim3((unsigned)nleaves, (unsigned)nb), 128, 0, st>>>(H, x, ldin, perm_in, nb, W.Xb,
                                                                                   ldx);
        dm_count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        Xb = W.Xb;
    }
    // near field on the side stream (it reads only Xb and writes only Yb)
    cudaStream_t sn = W.side ? W.side : st;
    if (W.side) {
        if ((e = cudaEventRecord(W.fork, st)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(sn, W.fork, 0)) != cudaSuccess) return e;
    }
    const int onthefly = near_mode == DM_NEAR_CACHED ? 0 : 1;
    if (near_prec != DM_PREC_FP32 && !onthefly)
        e = dm_launch_near_tc(H, Xb, ldx, nb, W.Yb, H.err, near_prec == DM_PREC_TF32X3, sn);
    else if (nb <= 16) e = launch_near<16>(H, onthefly, Xb, ldx, nb, W.Yb, sn);
    else if (nb <= 32) e = launch_near<32>(H, onthefly, Xb, ldx, nb, W.Yb, sn);
    else e = launch_near<64>(H, onthefly, Xb, ldx, nb, W.Yb, sn);
    if (e != cudaSuccess) return e;
    if (W.side) {
        if ((e = cudaEventRecord(W.join, sn)) != cudaSuccess) return e;
    }
    const bool far = H.L > 0;
    const unsigned cgroups = (unsigned)((nb + kColTile - 1) / kColTile);
    if (far) {
        const size_t sm_leaf = sizeof(float) * (size_t)H.leaf_max * kVs;
        if ((e = dm_allow_smem((const void *)blk_leaf_n2s_kernel, sm_leaf)) != cudaSuccess) return e;
        blk_leaf_n2s_kernel<<<dim3(nleaves, cgroups), kTreeLvThreads, sm_leaf, st>>>(H, Xb, ldx, nb, W.Wb);
        dm_count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const size_t sm_pair = sizeof(float) * 2 * (size_t)H.max_rank * kVs;
        if ((e = dm_allow_smem((const void *)blk_up_kernel, sm_pair)) != cudaSuccess) return e;
        for (int lv = H.L - 1; lv >= 0; --lv) {
            blk_up_kernel<<<dim3(1u << lv, cgroups), kTreeLvThreads, sm_pair, st>>>(H, lv, nb, W.Wb, W.Ub);
            dm_count_launches(1);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        const size_t sm_one = sizeof(float) * (size_t)H.max_rank * kVs;
        if ((e = dm_allow_smem((const void *)blk_down_kernel, sm_one)) != cudaSuccess) return e;
        for (int lv = 1; lv < H.L; ++lv) {
            blk_down_kernel<<<dim3(1u << lv, cgroups), kTreeLvThreads, sm_one, st>>>(H, lv, nb, W.Ub);
            dm_count_launches(1);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    if (W.side) {
        if ((e = cudaStreamWaitEvent(st, W.join, 0)) != cudaSuccess) return e;
    }
    const size_t sm_one = sizeof(float) * (size_t)H.max_rank * kColTile;
    if ((e = dm_allow_smem((const void *)blk_s2n_out_kernel, sm_one)) != cudaSuccess) return e;
    blk_s2n_out_kernel<<<dim3(nleaves, cgroups), kBlkThreads, sm_one, st>>>(
        H, W.Yb, ldx, nb, W.Ub, far ? 1 : 0, y_layout == DM_BLK_ORIGINAL ? H.perm : nullptr,
        y_layout == DM_BLK_POSITION ? 1 : 0, y, ldo);
    dm_count_launches(1);
    return cudaGetLastError();
}
