// k_bstep.cu -- one step of block Lanczos (Section 2.3.1 applied to a block of B <= 4
// vectors) in one cooperative launch: classical Gram-Schmidt twice against the basis, then
// CholeskyQR twice for the new block, with the coefficients in FP64.
//
// With Z = K~ V_j (B columns, position order) and the basis V[:, 0:ncols):
//   A  H0 = V^T Z                                      (FP32 partial sums, FP64 atomics)
//   B  Z' = Z - V H0;  H1 = V^T Z';  G1 = Z'^T Z'
//   C  Z'' = Z' - V H1;  G'' = G1 - H1^T H1 (= Z''^T Z'', as V^T Z' = H1);  R1 = chol(G'');
//      Q = Z'' R1^-1;  G2 = Q^T Q
//   D  R2 = chol(G2);  V[:, out:out+B) = Q R2^-1;  T(0:ncols, out-B:out) = H0 + H1;  B_j = R2 R1
// Passes are separated by bounded grid barriers (every block resident: one 512-thread block
// per SM). Each block owns a contiguous range of rows and keeps its rows of Z', Q in shared
// memory across the barriers. Accumulators are cleared by the kernel after their last
// reader has passed a barrier (H0 in C, H1 and G1 in D); G2 alternates between two buffers by
// step parity, the next one cleared in A.
#include "dm_internal.cuh"

namespace {

constexpr int kBsThreads = 512;
constexpr int kBsWarps = kBsThreads / 32;
// the FP64 coefficient sums go to kHCopies copies (block g to copy g mod kHCopies), so no
// address takes more than a few atomics from each group of blocks; readers add the copies
constexpr int kHCopies = 8;

struct BStepArgs {
    float *V;
    int64_t ldv;
    int ncols;       // basis columns to orthogonalise against
    int out;         // first column of V written (ncols for a step, 0 for the start block)
    const float *Z;  // B columns, stride ldv, zero past N
    double *H0, *H1; // kHCopies x (ncols x B, row-major), zero on entry; copy c at c * hstride
    int64_t hstride;
    double *G1;      // B x B (zero on entry)
    double *G2;      // two B x B buffers; this step uses parity `par`, clears the other
    int par;
    double *T;       // projected matrix, column-major m_max x m_max (nullptr: no entries)
    int ldT;
    double *Bj;      // B x B: R2 R1 (row-major)
    int *flag;       // raised when a block lost rank
    unsigned *bar;
    unsigned bar_base;
    int *err;
    int64_t per;     // rows per block (multiple of 4)
};

// Cholesky G = R^T R of a B x B FP64 matrix (row-major) and R^-1, with reciprocal square
// roots instead of divisions; a pivot that is not positive (a rank-deficient block) raises
// *flag and is replaced by a tiny positive value.
template <int B>
__device__ void chol_small(const double (&G)[B][B], double (&R)[B][B], double (&Ri)[B][B], int *flag) {
    double tr = 0.0;
    for (int i = 0; i < B; ++i) tr += G[i][i];
    const double tiny = 1e-300 + 1e-28 * tr;
    double inv[B];
    for (int i = 0; i < B; ++i)
        for (int j = 0; j < B; ++j) R[i][j] = Ri[i][j] = 0.0;
    for (int j = 0; j < B; ++j) {
        double d = G[j][j];
        for (int k = 0; k < j; ++k) d -= R[k][j] * R[k][j];
        if (!(d > tiny)) {
            if (flag) *flag = 1;
            d = tiny;
        }
        inv[j] = dm_rsqrt_fp64(d);
        R[j][j] = d * inv[j];
        for (int i = j + 1; i < B; ++i) {
            double t = G[j][i];
            for (int k = 0; k < j; ++k) t -= R[k][j] * R[k][i];
            R[j][i] = t * inv[j];
        }
    }
    for (int i = 0; i < B; ++i) {
        Ri[i][i] = inv[i];
        for (int q = i - 1; q >= 0; --q) {
            double t = 0.0;
            for (int k = q + 1; k <= i; ++k) t += R[q][k] * Ri[k][i];
            Ri[q][i] = -t * inv[q];
        }
    }
}

// acc[r][c] (global FP64) += sum over this block's rows of V[r][i] S[c][i] for r < ncols:
// a warp per basis column, lanes over row quads, then a warp sum per column c
template <int B>
__device__ __forceinline__ void project_rows(const float *__restrict__ V, int64_t ldv, int ncols, int64_t r0,
                                             int nq, const float4 *S, double *acc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = warp; r < ncols; r += kBsWarps) {
        const float4 *vr = reinterpret_cast<const float4 *>(V + (size_t)r * ldv + r0);
        float s[B];
#pragma unroll
        for (int c = 0; c < B; ++c) s[c] = 0.f;
#pragma unroll 4
        for (int q = lane; q < nq; q += 32) {
            const float4 v = __ldcg(vr + q);
#pragma unroll
            for (int c = 0; c < B; ++c) {
                const float4 z = S[c * nq + q];
                s[c] = fmaf(v.x, z.x, fmaf(v.y, z.y, fmaf(v.z, z.z, fmaf(v.w, z.w, s[c]))));
            }
        }
#pragma unroll
        for (int c = 0; c < B; ++c) {
            const float t = dm_warp_sum(s[c]);
            if (lane == 0) atomicAdd(acc + (size_t)r * B + c, (double)t);
        }
    }
}

// S[c][q] -= sum_r V[r][q] h[r][c] for this block's row quads: the basis columns split into
// rs slices so all threads work (thread = (slice, quad)), partial sums combined in `part`
template <int B>
__device__ __forceinline__ void update_rows(const float *__restrict__ V, int64_t ldv, int ncols, int64_t r0, int nq,
                                            const float *hs, float4 *S, float4 *part) {
    const int rs = nq > 0 ? (blockDim.x / nq > 0 ? (int)(blockDim.x / nq) : 1) : 1;
    const int64_t ld4 = ldv >> 2;
    const float4 *v0 = reinterpret_cast<const float4 *>(V + r0);
    for (int t = threadIdx.x; t < rs * nq; t += blockDim.x) {
        const int sl = t / nq, q = t - sl * nq;
        float4 a[B];
#pragma unroll
        for (int c = 0; c < B; ++c) a[c] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
        for (int r = sl; r < ncols; r += rs) {
            const float4 v = __ldcg(v0 + (size_t)r * ld4 + q);
#pragma unroll
            for (int c = 0; c < B; ++c) {
                const float h = hs[r * B + c];
                a[c].x = fmaf(v.x, h, a[c].x);
                a[c].y = fmaf(v.y, h, a[c].y);
                a[c].z = fmaf(v.z, h, a[c].z);
                a[c].w = fmaf(v.w, h, a[c].w);
            }
        }
#pragma unroll
        for (int c = 0; c < B; ++c) part[((size_t)sl * B + c) * nq + q] = a[c];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < B * nq; e += blockDim.x) {
        const int c = e / nq, q = e - c * nq;
        float4 z = S[e];
        for (int sl = 0; sl < rs; ++sl) {
            const float4 p = part[((size_t)sl * B + c) * nq + q];
            z.x -= p.x;
            z.y -= p.y;
            z.z -= p.z;
            z.w -= p.w;
        }
        S[e] = z;
    }
    __syncthreads();
}

// acc (global B x B, FP64) += S^T S over this block's rows
template <int B>
__device__ __forceinline__ void gram_rows(const float4 *S, int nq, double *acc, float *red) {
    float g[B * B];
#pragma unroll
    for (int e = 0; e < B * B; ++e) g[e] = 0.f;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        float4 z[B];
#pragma unroll
        for (int c = 0; c < B; ++c) z[c] = S[c * nq + q];
#pragma unroll
        for (int c = 0; c < B; ++c)
#pragma unroll
            for (int d = c; d < B; ++d)
                g[c * B + d] += z[c].x * z[d].x + z[c].y * z[d].y + z[c].z * z[d].z + z[c].w * z[d].w;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int e = 0; e < B * B; ++e) {
        const float t = dm_warp_sum(g[e]);
        if (lane == 0) red[warp * B * B + e] = t;
    }
    __syncthreads();
    if (threadIdx.x < B * B) {
        const int c = threadIdx.x / B, d = threadIdx.x % B;
        if (d >= c) {
            double s = 0.0;
            for (int w = 0; w < kBsWarps; ++w) s += (double)red[w * B * B + threadIdx.x];
            atomicAdd(acc + c * B + d, s);
            if (d != c) atomicAdd(acc + d * B + c, s);
        }
    }
}

template <int B>
__global__ void __launch_bounds__(kBsThreads, 1) bstep_kernel(const __grid_constant__ BStepArgs a) {
    extern __shared__ float4 bs4[];
    __shared__ float red[kBsWarps * B * B];
    __shared__ double s_R1[B][B], s_R1i[B][B], s_M[B][B];
    const unsigned G = gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * a.per;
    const int64_t r1 = r0 + a.per < a.ldv ? r0 + a.per : a.ldv;
    const int nq = r1 > r0 ? (int)((r1 - r0) >> 2) : 0;
    float4 *S = bs4;                                          // B x nq: Z, then Z', Z'', Q
    float4 *part = S + (size_t)B * (a.per >> 2);              // update partials: B x (blockDim) float4
    float *hs = reinterpret_cast<float *>(part + (size_t)B * kBsThreads);  // ncols x B coefficients
    double *G2 = a.G2 + (size_t)a.par * B * B;
    double *G2n = a.G2 + (size_t)(a.par ^ 1) * B * B;

    // ---- A: stage Z; H0 = V^T Z
    for (int e = threadIdx.x; e < B * nq; e += blockDim.x) {
        const int c = e / nq, q = e - c * nq;
        S[e] = __ldcg(reinterpret_cast<const float4 *>(a.Z + (size_t)c * a.ldv + r0) + q);
    }
    if (blockIdx.x == 0 && threadIdx.x < B * B) G2n[threadIdx.x] = 0.0;
    __syncthreads();
    const int copy = blockIdx.x % kHCopies;
    if (a.ncols > 0) project_rows<B>(a.V, a.ldv, a.ncols, r0, nq, S, a.H0 + copy * a.hstride);
    if (!grid_barrier(a.bar, a.bar_base + G, a.err)) return;

    // ---- B: Z' = Z - V H0; H1 = V^T Z'; G1 = Z'^T Z'
    if (a.ncols > 0) {
        for (int e = threadIdx.x; e < a.ncols * B; e += blockDim.x) {
            double t = 0.0;
#pragma unroll
            for (int u = 0; u < kHCopies; ++u) t += __ldcg(a.H0 + u * a.hstride + e);
            hs[e] = (float)t;
        }
        __syncthreads();
        update_rows<B>(a.V, a.ldv, a.ncols, r0, nq, hs, S, part);
        project_rows<B>(a.V, a.ldv, a.ncols, r0, nq, S, a.H1 + copy * a.hstride);
    }
    gram_rows<B>(S, nq, a.G1, red);
    if (!grid_barrier(a.bar, a.bar_base + 2 * G, a.err)) return;

    // ---- C: Z'' = Z' - V H1; R1 = chol(G1 - H1^T H1); Q = Z'' R1^-1; G2 = Q^T Q
    double *h1d = reinterpret_cast<double *>(hs + ((a.ncols * B + 1) & ~1));  // ncols x B, FP64
    if (a.ncols > 0) {
        for (int e = threadIdx.x; e < a.ncols * B; e += blockDim.x) {
            double t = 0.0;
#pragma unroll
            for (int u = 0; u < kHCopies; ++u) t += __ldcg(a.H1 + u * a.hstride + e);
            h1d[e] = t;
            hs[e] = (float)t;
        }
        __syncthreads();
        update_rows<B>(a.V, a.ldv, a.ncols, r0, nq, hs, S, part);
        // H0 has been read by every block (pass B): block 0 moves it into T and clears it
        if (blockIdx.x == 0)
            for (int e = threadIdx.x; e < a.ncols * B; e += blockDim.x) {
                const int r = e / B, c = e - r * B;
                double t = 0.0;
#pragma unroll
                for (int u = 0; u < kHCopies; ++u) {
                    t += __ldcg(a.H0 + u * a.hstride + e);
                    a.H0[u * a.hstride + e] = 0.0;
                }
                if (a.T) a.T[(size_t)(a.out - B + c) * a.ldT + r] = t;
            }
    }
    if (threadIdx.x < B * B) {
        const int c = threadIdx.x / B, d = threadIdx.x % B;
        double g = __ldcg(a.G1 + threadIdx.x);
        for (int r = 0; r < a.ncols; ++r) g -= h1d[r * B + c] * h1d[r * B + d];
        s_M[c][d] = g;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double R[B][B], Ri[B][B];
        chol_small<B>(s_M, R, Ri, blockIdx.x == 0 ? a.flag : nullptr);
        for (int i = 0; i < B; ++i)
            for (int j = 0; j < B; ++j) {
                s_R1[i][j] = R[i][j];
                s_R1i[i][j] = Ri[i][j];
            }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        float4 z[B], o[B];
#pragma unroll
        for (int c = 0; c < B; ++c) z[c] = S[c * nq + q];
#pragma unroll
        for (int c = 0; c < B; ++c) {
            o[c] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int r = 0; r <= c; ++r) {
                const float w = (float)s_R1i[r][c];
                o[c].x = fmaf(z[r].x, w, o[c].x);
                o[c].y = fmaf(z[r].y, w, o[c].y);
                o[c].z = fmaf(z[r].z, w, o[c].z);
                o[c].w = fmaf(z[r].w, w, o[c].w);
            }
        }
#pragma unroll
        for (int c = 0; c < B; ++c) S[c * nq + q] = o[c];
    }
    __syncthreads();
    gram_rows<B>(S, nq, G2, red);
    if (!grid_barrier(a.bar, a.bar_base + 3 * G, a.err)) return;

    // ---- D: R2 = chol(G2); V[:, out:out+B) = Q R2^-1; T entries; B_j = R2 R1
    if (threadIdx.x < B * B) s_M[threadIdx.x / B][threadIdx.x % B] = __ldcg(G2 + threadIdx.x);
    __syncthreads();
    __shared__ double s_R2i[B][B];
    if (threadIdx.x == 0) {
        double R[B][B], Ri[B][B];
        chol_small<B>(s_M, R, Ri, blockIdx.x == 0 ? a.flag : nullptr);
        for (int i = 0; i < B; ++i)
            for (int j = 0; j < B; ++j) s_R2i[i][j] = Ri[i][j];
        if (blockIdx.x == 0)
            for (int i = 0; i < B; ++i)
                for (int j = 0; j < B; ++j) {
                    double t = 0.0;
                    for (int k = i; k <= j; ++k) t += R[i][k] * s_R1[k][j];
                    a.Bj[i * B + j] = t;
                }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        float4 z[B];
#pragma unroll
        for (int c = 0; c < B; ++c) z[c] = S[c * nq + q];
#pragma unroll
        for (int c = 0; c < B; ++c) {
            float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int r = 0; r <= c; ++r) {
                const float w = (float)s_R2i[r][c];
                o.x = fmaf(z[r].x, w, o.x);
                o.y = fmaf(z[r].y, w, o.y);
                o.z = fmaf(z[r].z, w, o.z);
                o.w = fmaf(z[r].w, w, o.w);
            }
            reinterpret_cast<float4 *>(a.V + (size_t)(a.out + c) * a.ldv + r0)[q] = o;
        }
    }
    // H1 and G1 have been read by every block (pass C): block 0 adds H1 into T, clears both
    if (blockIdx.x == 0) {
        for (int e = threadIdx.x; e < a.ncols * B; e += blockDim.x) {
            const int r = e / B, c = e - r * B;
            if (a.T) a.T[(size_t)(a.out - B + c) * a.ldT + r] += h1d[e];
            for (int u = 0; u < kHCopies; ++u) a.H1[u * a.hstride + e] = 0.0;
        }
        if (threadIdx.x < B * B) a.G1[threadIdx.x] = 0.0;
    }
}

template <int B>
cudaError_t launch_bstep(BStepArgs &a, int G, cudaStream_t st) {
    const size_t smem = sizeof(float) * ((size_t)B * a.per + (size_t)4 * B * kBsThreads +
                                         (size_t)3 * ((a.ncols > 0 ? a.ncols : 1) * B + 2));
    cudaError_t e = dm_allow_smem((const void *)bstep_kernel<B>, smem);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&a};
    e = cudaLaunchCooperativeKernel((const void *)bstep_kernel<B>, dim3((unsigned)G), dim3(kBsThreads), args, smem, st);
    dm_count_launches(1);
    return e;
}

}  // namespace

int dm_bstep_max_b() { return 4; }

int dm_bstep_hcopies() { return kHCopies; }

cudaError_t dm_bstep(int b, float *V, int64_t ldv, int ncols, int out, const float *Z, double *H0, double *H1,
                     int64_t hstride, double *G1, double *G2, int par, double *T, int ldT, double *Bj, int *flag,
                     unsigned *bar, unsigned bar_base, int *err, int blocks, cudaStream_t st) {
    BStepArgs a;
    a.hstride = hstride;
    a.V = V;
    a.ldv = ldv;
    a.ncols = ncols;
    a.out = out;
    a.Z = Z;
    a.H0 = H0;
    a.H1 = H1;
    a.G1 = G1;
    a.G2 = G2;
    a.par = par & 1;
    a.T = T;
    a.ldT = ldT;
    a.Bj = Bj;
    a.flag = flag;
    a.bar = bar;
    a.bar_base = bar_base;
    a.err = err;
    a.per = ((ldv + blocks - 1) / blocks + 3) & ~int64_t(3);
    switch (b) {
        case 2: return launch_bstep<2>(a, blocks, st);
        case 3: return launch_bstep<3>(a, blocks, st);
        case 4: return launch_bstep<4>(a, blocks, st);
        default: return cudaErrorInvalidValue;
    }
}
