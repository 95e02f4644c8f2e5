// k_blanczos.cu -- block Lanczos: the Lanczos method of Section 2.3.1 run on a block of b
// vectors at a time, so that every H-matvec applies the operator to b right-hand sides
// (one pass over the stored blocks instead of b).
//
// Step j (V_j = the j-th block of b orthonormal columns, position order):
//   Z = K~ V_j                                    block H-matvec
//   H = V^T Z, Z -= V H, twice (CGS2)             all (j+1) b basis columns; FP32 partial
//                                                 sums reduced in FP64; T(:, block j) = H1 + H2
//   Z = V_{j+1} B_j by CholQR2                    Gram in FP64, Cholesky in FP64
//                                                 (B_j^T enters T through step j+1's H)
// T = V^T K~ V is block tridiagonal up to rounding; it is kept dense (upper triangle) and
// the Rayleigh-Ritz step reduces it to a tridiagonal matrix by Householder reflections in
// FP64, so the FP64 Sturm-sequence solver and inverse iteration of the single-vector path
// give its eigenpairs. A Ritz pair (theta, y) has residual |A V y - theta V y| = |B_j y_j|
// (y_j = the last b entries of y).
#include "dm_internal.cuh"

namespace {

constexpr int kBlThreads = 256;
constexpr int kBlMaxB = 16;

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// start block: column c uniform in [-1, 1] from the stream (seed, V0 tag, 1 + c), indexed
// by original point index (independent of the tree permutation)
__global__ void bl_start_kernel(const int32_t *__restrict__ perm, int64_t N, int b, uint64_t seed, float *Z,
                                int64_t ldz) {
    const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (pos >= N) return;
    const uint64_t key = dm_stream_key(seed, DM_TAG_V0, 1 + (uint64_t)c);
    Z[(size_t)c * ldz + pos] = (float)(2.0 * dm_unit(dm_rng(key, (uint64_t)perm[pos])) - 1.0);
}

// part[p][r][c] = sum over this block's rows of A[r][i] Z[c][i]   (r < ncols, c < b)
__global__ void __launch_bounds__(kBlThreads) bl_proj_kernel(const float *__restrict__ A, int64_t lda, int ncols,
                                                             const float *__restrict__ Z, int64_t ldz, int b,
                                                             int64_t N, int64_t per, float *__restrict__ part,
                                                             int ldpart) {
    extern __shared__ float zs[];  // b x per
    const int64_t r0 = blockIdx.x * per;
    const int nrows = (int)(r0 >= N ? 0 : (N - r0 < per ? N - r0 : per));
    for (int e = threadIdx.x; e < b * nrows; e += blockDim.x) {
        const int c = e / nrows, i = e - c * nrows;
        zs[c * per + i] = Z[(size_t)c * ldz + r0 + i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float *out = part + (size_t)blockIdx.x * ldpart * b;
    for (int r = warp; r < ncols; r += nw) {
        float acc[kBlMaxB];
#pragma unroll
        for (int c = 0; c < kBlMaxB; ++c) acc[c] = 0.f;
        const float *ar = A + (size_t)r * lda + r0;
        for (int i = lane; i < nrows; i += 32) {
            const float v = __ldcg(ar + i);
#pragma unroll
            for (int c = 0; c < kBlMaxB; ++c)
                if (c < b) acc[c] = fmaf(v, zs[c * per + i], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < kBlMaxB; ++c) {
            if (c < b) {
                const float s = dm_warp_sum(acc[c]);
                if (lane == 0) out[(size_t)r * b + c] = s;
            }
        }
    }
}

// H[r][c] = sum_p part[p][r][c] (FP64); with T: T(row0 + r, col0 + c) += H[r][c].
// A warp per output: the lanes split the partial sums, then a warp reduction.
__global__ void bl_reduce_kernel(const float *__restrict__ part, int nparts, int ldpart, int ncols, int b,
                                 double *__restrict__ H, double *T, int ldT, int row0, int col0) {
    const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (e >= ncols * b) return;
    const int r = e / b, c = e - r * b;
    double s = 0.0;
    for (int p = lane; p < nparts; p += 32) s += (double)part[((size_t)p * ldpart + r) * b + c];
    s = dm_warp_sum_d(s);
    if (lane == 0) {
        H[e] = s;
        if (T) T[(size_t)(col0 + c) * ldT + row0 + r] += s;
    }
}

// Z[c][i] -= sum_r A[r][i] H[r][c]   (thread per row)
__global__ void __launch_bounds__(kBlThreads) bl_update_kernel(const float *__restrict__ A, int64_t lda, int ncols,
                                                               float *__restrict__ Z, int64_t ldz, int b, int64_t N,
                                                               const double *__restrict__ H) {
    extern __shared__ float hs[];  // ncols x b
    for (int e = threadIdx.x; e < ncols * b; e += blockDim.x) hs[e] = (float)H[e];
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    float acc[kBlMaxB];
#pragma unroll
    for (int c = 0; c < kBlMaxB; ++c) acc[c] = 0.f;
    for (int r = 0; r < ncols; ++r) {
        const float v = __ldcg(A + (size_t)r * lda + i);
#pragma unroll
        for (int c = 0; c < kBlMaxB; ++c)
            if (c < b) acc[c] = fmaf(v, hs[r * b + c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < kBlMaxB; ++c)
        if (c < b) Z[(size_t)c * ldz + i] -= acc[c];
}

// Cholesky G = R^T R (FP64; b <= 16) by one warp in shared memory: lane i owns column i of
// R (Cholesky) and of R^-1 (triangular inverse), and row i of the product. Rinv = R^-1;
// Bacc = R (first) or R Bacc. A pivot that is not positive (a rank-deficient block: the
// Krylov space is exhausted) raises *flag and is replaced by a tiny positive value.
__global__ void __launch_bounds__(32) bl_chol_kernel(const double *__restrict__ G, int b,
                                                     double *__restrict__ Rinv, double *__restrict__ Bacc,
                                                     int first, int *flag) {
    __shared__ double R[kBlMaxB][kBlMaxB + 1], Ri[kBlMaxB][kBlMaxB + 1], Bo[kBlMaxB][kBlMaxB + 1];
    const int i = threadIdx.x;
    double tr = 0.0;
    for (int q = 0; q < b; ++q) tr += G[q * b + q];
    const double tiny = 1e-300 + 1e-28 * tr;
    if (i < b)
        for (int q = 0; q < b; ++q) {
            R[q][i] = 0.0;
            Ri[q][i] = 0.0;
            Bo[q][i] = Bacc[q * b + i];
        }
    __syncwarp();
    for (int j = 0; j < b; ++j) {
        // lane j: the pivot; then lanes i > j: R[j][i]
        if (i == j) {
            double sd = G[j * b + j];
            for (int k = 0; k < j; ++k) sd -= R[k][j] * R[k][j];
            if (!(sd > tiny)) {
                *flag = 1;
                sd = tiny;
            }
            R[j][j] = sqrt(sd);
        }
        __syncwarp();
        if (i > j && i < b) {
            double t = G[j * b + i];
            for (int k = 0; k < j; ++k) t -= R[k][j] * R[k][i];
            R[j][i] = t / R[j][j];
        }
        __syncwarp();
    }
    // column i of R^-1: Ri[i][i] = 1 / R[i][i], then rows q = i-1 .. 0
    if (i < b) {
        Ri[i][i] = 1.0 / R[i][i];
        for (int q = i - 1; q >= 0; --q) {
            double t = 0.0;
            for (int k = q + 1; k <= i; ++k) t += R[q][k] * Ri[k][i];
            Ri[q][i] = -t / R[q][q];
        }
    }
    __syncwarp();
    if (i < b) {
        for (int q = 0; q < b; ++q) Rinv[q * b + i] = Ri[q][i];
        // row i of R (first) or R Bacc
        for (int q = 0; q < b; ++q) {
            double t;
            if (first) t = R[i][q];
            else {
                t = 0.0;
                for (int k = i; k < b; ++k) t += R[i][k] * Bo[k][q];
            }
            Bacc[i * b + q] = t;
        }
    }
}

// out[c][i] = sum_{r <= c} Z[r][i] Rinv[r][c]   (thread per row)
__global__ void bl_scale_kernel(const float *__restrict__ Z, int64_t ldz, int b, int64_t N,
                                const double *__restrict__ Rinv, float *__restrict__ out, int64_t ldo) {
    __shared__ float ri[kBlMaxB * kBlMaxB];
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) ri[e] = (float)Rinv[e];
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    float z[kBlMaxB];
#pragma unroll
    for (int c = 0; c < kBlMaxB; ++c) z[c] = c < b ? Z[(size_t)c * ldz + i] : 0.f;
#pragma unroll
    for (int c = 0; c < kBlMaxB; ++c) {
        if (c >= b) continue;
        float s = 0.f;
#pragma unroll
        for (int r = 0; r < kBlMaxB; ++r)
            if (r <= c) s = fmaf(z[r], ri[r * b + c], s);
        out[(size_t)c * ldo + i] = s;
    }
}

// ---- Householder tridiagonalisation of the symmetric T (upper triangle, m x m) in FP64,
// one CTA of 1024 threads: W = Q^T T Q with alpha = diag, beta = subdiagonal; the reflector
// of step k (I - hb_k v v^T, v on rows k+1..m-1) is left in column k of W below the diagonal.
// Per step: the column norm and the dot p.v in one warp (no block-wide reduction), the
// product p = W_sub v with a warp per row (lanes over the row, a shuffle sum), the rank-2
// update over all threads; four barriers per step.
constexpr int kTrThreads = 1024;
constexpr int kTrSmemMax = 144;  // largest m whose working matrix fits in shared memory

__global__ void __launch_bounds__(kTrThreads) bl_tridiag_kernel(const double *__restrict__ T, int ldT, int m,
                                                                double *Wg, int ldwg, double *__restrict__ alpha,
                                                                double *__restrict__ beta,
                                                                double *__restrict__ hb, int in_smem) {
    extern __shared__ double sv[];  // v (m), p (m), scalars (4), then the m x m working matrix
    double *v = sv, *p = sv + m, *sc = sv + 2 * m;
    double *W = in_smem ? sv + 2 * m + 4 : Wg;
    const int ldw = in_smem ? m : ldwg;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int r = e % m, c = e / m;
        W[(size_t)c * ldw + r] = r <= c ? T[(size_t)c * ldT + r] : T[(size_t)r * ldT + c];
    }
    __syncthreads();
    for (int k = 0; k + 2 < m; ++k) {
        const int n = m - k - 1;  // trailing size
        double *col = W + (size_t)k * ldw + (k + 1);
        if (warp == 0) {
            double ss = 0.0;
            for (int i = lane; i < n; i += 32) {
                const double x = col[i];
                v[i] = x;
                ss = fma(x, x, ss);
            }
            ss = dm_warp_sum_d(ss);
            if (lane == 0) {
                const double x0 = col[0];
                const double xn = sqrt(ss);
                const double al = x0 >= 0.0 ? -xn : xn;
                const double vnorm2 = ss - x0 * x0 + (x0 - al) * (x0 - al);
                const double bk = vnorm2 > 0.0 ? 2.0 / vnorm2 : 0.0;
                v[0] = x0 - al;
                alpha[k] = W[(size_t)k * ldw + k];
                beta[k] = vnorm2 > 0.0 ? al : x0;
                hb[k] = bk;
                sc[0] = bk;
            }
        }
        __syncthreads();
        const double bk = sc[0];
        if (bk != 0.0) {
            // p = bk W_sub v: eight lanes per row i (W symmetric: column k+1+i of the
            // sub-block), three shuffle steps; few FP64 instructions per row (the FP64 pipe
            // of this part is narrow, so shuffle-and-add trees are kept short)
            for (int base = 4 * warp; base < n; base += 4 * nw) {  // warp-uniform bound
                const int i = base + (lane >> 3), l8 = lane & 7;
                double s = 0.0;
                if (i < n) {
                    const double *wr = W + (size_t)(k + 1 + i) * ldw + (k + 1);
                    for (int j = l8; j < n; j += 8) s = fma(wr[j], v[j], s);
                }
                s += __shfl_xor_sync(0xffffffffu, s, 1);
                s += __shfl_xor_sync(0xffffffffu, s, 2);
                s += __shfl_xor_sync(0xffffffffu, s, 4);
                if (i < n && l8 == 0) p[i] = bk * s;
            }
            __syncthreads();
            if (warp == 0) {
                double pv = 0.0;
                for (int i = lane; i < n; i += 32) pv = fma(p[i], v[i], pv);
                const double K = 0.5 * bk * dm_warp_sum_d(pv);
                for (int i = lane; i < n; i += 32) p[i] -= K * v[i];  // w
            }
            __syncthreads();
            for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
                const int i = e % n, j = e / n;
                double *wij = W + (size_t)(k + 1 + j) * ldw + (k + 1 + i);
                *wij = fma(-v[i], p[j], fma(-p[i], v[j], *wij));
            }
        }
        // keep the reflector in column k below the diagonal
        for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = v[i];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (m >= 2) {
            alpha[m - 2] = W[(size_t)(m - 2) * ldw + (m - 2)];
            beta[m - 2] = W[(size_t)(m - 2) * ldw + (m - 1)];
            hb[m - 2] = 0.0;
        }
        alpha[m - 1] = W[(size_t)(m - 1) * ldw + (m - 1)];
        beta[m - 1] = 0.0;
    }
    if (in_smem) {
        // the reflectors (below the diagonal) for the back-transformation
        __syncthreads();
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int r = e % m, c = e / m;
            if (r > c) Wg[(size_t)c * ldwg + r] = W[(size_t)c * ldw + r];
        }
    }
}

// Eigenvectors of T from those of the tridiagonal (Y, columns of length m): y <- Q y with
// Q = H_0 H_1 ... H_{m-3}; then the residual bound |B_j y_j| (y_j = last b entries) and
// the FP32 copy Yf (m x k, row-major) for the Ritz-vector product. A warp per vector, the
// reflectors staged in shared memory once per CTA (from global memory when they do not fit).
constexpr int kBtWarps = 8;
__global__ void __launch_bounds__(32 * kBtWarps) bl_backtransform_kernel(const double *__restrict__ W, int ldw,
                                                                         const double *__restrict__ hb, int m, int k,
                                                                         double *__restrict__ Y, int ldy,
                                                                         float *__restrict__ Yf,
                                                                         const double *__restrict__ Bj, int b,
                                                                         double *__restrict__ resid, int staged) {
    extern __shared__ double bsm[];  // staged: reflectors (m x m, column-major); then kBtWarps x m vectors
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double *Wr = staged ? bsm : W;
    const int ldr = staged ? m : ldw;
    double *ys = bsm + (staged ? (size_t)m * m : 0) + (size_t)warp * m;
    if (staged) {
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int r = e % m, c = e / m;
            bsm[e] = r > c ? W[(size_t)c * ldw + r] : 0.0;
        }
    }
    const int iv = blockIdx.x * kBtWarps + warp;
    if (iv < k)
        for (int i = lane; i < m; i += 32) ys[i] = Y[(size_t)iv * ldy + i];
    __syncthreads();
    if (iv >= k) return;
    for (int kk = m - 3; kk >= 0; --kk) {
        const double bk = hb[kk];
        if (bk == 0.0) continue;
        const int n = m - kk - 1;
        const double *v = Wr + (size_t)kk * ldr + (kk + 1);
        double s = 0.0;
        for (int i = lane; i < n; i += 32) s = fma(v[i], ys[kk + 1 + i], s);
        const double f = bk * dm_warp_sum_d(s);
        for (int i = lane; i < n; i += 32) ys[kk + 1 + i] -= f * v[i];
        __syncwarp();
    }
    for (int i = lane; i < m; i += 32) {
        Y[(size_t)iv * ldy + i] = ys[i];
        Yf[(size_t)i * k + iv] = (float)ys[i];
    }
    __syncwarp();
    if (lane == 0) {
        double rr = 0.0;
        for (int r = 0; r < b; ++r) {
            double t = 0.0;
            for (int c = r; c < b; ++c) t += Bj[r * b + c] * ys[m - b + c];
            rr += t * t;
        }
        resid[iv] = sqrt(rr);
    }
}

}  // namespace

int dm_block_lanczos_max_b() { return kBlMaxB; }

cudaError_t dm_bl_random_block(DmLanczos &Lz, DmBlockLanczos &B, const int32_t *perm, uint64_t seed,
                               cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(B.T, 0, sizeof(double) * (size_t)Lz.m_max * Lz.m_max, st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(B.flag, 0, sizeof(int), st)) != cudaSuccess) return e;
    bl_start_kernel<<<dim3(nblk(Lz.N, 256), (unsigned)B.b), 256, 0, st>>>(perm, Lz.N, B.b, seed, B.Z, Lz.ldv);
    dm_count_launches(1);
    return cudaGetLastError();
}

cudaError_t dm_bl_start(DmLanczos &Lz, DmBlockLanczos &B, const int32_t *perm, uint64_t seed, cudaStream_t st) {
    cudaError_t e = dm_bl_random_block(Lz, B, perm, seed, st);
    if (e != cudaSuccess) return e;
    // V_0 = Z R^-1 by CholQR2 (no T entries)
    return dm_bl_cholqr(Lz, B, 0, false, st);
}

// ncols columns of A (stride lda) against the b columns of Z: H (FP64, ncols x b); with
// to_T, T(row0.., col0..) += H.
static cudaError_t project(DmLanczos &Lz, DmBlockLanczos &B, const float *A, int ncols, const float *Z,
                           bool to_T, int col0, cudaStream_t st) {
    const int64_t per = (Lz.N + B.nparts - 1) / B.nparts;
    const size_t sm = sizeof(float) * (size_t)B.b * per;
    cudaError_t e = dm_allow_smem((const void *)bl_proj_kernel, sm);
    if (e != cudaSuccess) return e;
    bl_proj_kernel<<<B.nparts, kBlThreads, sm, st>>>(A, Lz.ldv, ncols, Z, Lz.ldv, B.b, Lz.N, per, B.part,
                                                     B.ldpart);
    dm_count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    bl_reduce_kernel<<<nblk((int64_t)ncols * B.b, 8), 256, 0, st>>>(B.part, B.nparts, B.ldpart, ncols, B.b, B.H,
                                                                     to_T ? B.T : nullptr, Lz.m_max, 0, col0);
    dm_count_launches(1);
    return cudaGetLastError();
}

cudaError_t dm_bl_cholqr(DmLanczos &Lz, DmBlockLanczos &B, int j, bool next_block, cudaStream_t st) {
    // Z = V_{j+1} B_j: two rounds of (Gram, Cholesky, Z R^-1); the second writes V block j+1
    const int b = B.b;
    float *Vn = Lz.V + (size_t)(next_block ? (j + 1) : 0) * b * Lz.ldv;
    cudaError_t e;
    for (int round = 0; round < 2; ++round) {
        if ((e = project(Lz, B, B.Z, b, B.Z, false, 0, st)) != cudaSuccess) return e;
        const bool last = round == 1;
        // B_j itself is not written into T: the next step's projection V^T K~ V_{j+1} holds
        // the block T(block j, block j+1) = B_j^T (and the last block column of T_m is this
        // step's projection), so B_j only serves the residual bound
        bl_chol_kernel<<<1, 32, 0, st>>>(B.H, b, B.Rinv, B.Bacc, round == 0 ? 1 : 0, B.flag);
        dm_count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        bl_scale_kernel<<<nblk(Lz.N, 256), 256, 0, st>>>(B.Z, Lz.ldv, b, Lz.N, B.Rinv, last ? Vn : B.Z, Lz.ldv);
        dm_count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t dm_bl_orth(DmLanczos &Lz, DmBlockLanczos &B, int j, cudaStream_t st) {
    // after Z = K~ V_j: CGS2 against V[:, 0 .. (j+1) b), T(:, block j) = H1 + H2, then CholQR2
    const int ncols = (j + 1) * B.b;
    cudaError_t e;
    for (int pass = 0; pass < 2; ++pass) {
        if ((e = project(Lz, B, Lz.V, ncols, B.Z, true, j * B.b, st)) != cudaSuccess) return e;
        const size_t sm = sizeof(float) * (size_t)ncols * B.b;
        if ((e = dm_allow_smem((const void *)bl_update_kernel, sm)) != cudaSuccess) return e;
        bl_update_kernel<<<nblk(Lz.N, kBlThreads), kBlThreads, sm, st>>>(Lz.V, Lz.ldv, ncols, B.Z, Lz.ldv, B.b,
                                                                         Lz.N, B.H);
        dm_count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return dm_bl_cholqr(Lz, B, j, true, st);
}

cudaError_t dm_bl_ritz(DmLanczos &Lz, DmBlockLanczos &B, int m, int k, cudaStream_t st) {
    const int in_smem = m <= kTrSmemMax ? 1 : 0;
    const size_t sm = sizeof(double) * (2 * (size_t)m + 4 + (in_smem ? (size_t)m * m : 0));
    cudaError_t e = dm_allow_smem((const void *)bl_tridiag_kernel, sm);
    if (e != cudaSuccess) return e;
    bl_tridiag_kernel<<<1, kTrThreads, sm, st>>>(B.T, Lz.m_max, m, B.W, Lz.m_max, Lz.alpha, Lz.beta, B.hb, in_smem);
    dm_count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = dm_lanczos_ritz(Lz, m, k, 0.0, st)) != cudaSuccess) return e;
    if ((e = dm_lanczos_tvecs(Lz, m, k, st)) != cudaSuccess) return e;
    const int staged = m <= kTrSmemMax ? 1 : 0;
    const size_t smb = sizeof(double) * ((staged ? (size_t)m * m : 0) + (size_t)kBtWarps * m);
    if ((e = dm_allow_smem((const void *)bl_backtransform_kernel, smb)) != cudaSuccess) return e;
    bl_backtransform_kernel<<<(k + kBtWarps - 1) / kBtWarps, 32 * kBtWarps, smb, st>>>(
        B.W, Lz.m_max, B.hb, m, k, Lz.Y, Lz.m_max, Lz.Yf, B.Bacc, B.b, Lz.resid, staged);
    dm_count_launches(1);
    return cudaGetLastError();
}
