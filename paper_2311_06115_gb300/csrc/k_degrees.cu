// k_degrees.cu -- kernel scale, degree vectors and the exact on-the-fly matvec.
//
// Algorithm 1, steps 1-3 of the paper: W_ij = exp(-|x_i - x_j|^2 / eps) (Eq. W),
// q = W 1, W^a = Q^-a W Q^-a, dg = W^a 1, and the symmetric scaling
// s = q^-a dg^-1/2 so that S = diag(s) W diag(s) is the symmetric conjugate of
// the Markov matrix P = Dg^-1 W^a. The two O(N^2) passes run on the FP32
// pipes: coordinates are pre-scaled by sqrt(log2(e)/eps) so that every entry
// is one MUFU ex2 of minus a squared distance; partial sums over a tile of
// columns are FP32, tiles are accumulated in FP64 and the column splits meet in
// FP64 atomics.
#include "dm_internal.cuh"

namespace {

constexpr int kDegThreads = 128;   // rows per CTA (one per thread)
constexpr int kDegTile = 256;      // columns per shared-memory tile

// ---- bandwidth: squared pair distances in FP64 (reproducible) --------------
__global__ void all_pairs_kernel(const float *__restrict__ X, int64_t N, int d, double *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int64_t base = i * N - i * (i + 1) / 2;  // pairs (i, j>i) start here
    for (int64_t j = i + 1; j < N; ++j) out[base + (j - i - 1)] = dm_sqdist64(X + i * d, X + j * d, d);
}

__global__ void sampled_pairs_kernel(const float *__restrict__ X, int64_t N, int d, uint64_t key,
                                     double *__restrict__ out, int64_t m) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= m) return;
    int64_t i = (int64_t)dm_below(dm_rng(key, 2 * (uint64_t)c), (uint64_t)N);
    int64_t j = (int64_t)dm_below(dm_rng(key, 2 * (uint64_t)c + 1), (uint64_t)(N - 1));
    if (j >= i) j += 1;
    out[c] = dm_sqdist64(X + i * d, X + j * d, d);
}

// median of m non-negative doubles (their bit patterns order like the values);
// an even count averages the two middle values
__global__ void __launch_bounds__(1024) median_kernel(const double *__restrict__ v, int64_t m,
                                                      double *__restrict__ result) {
    __shared__ unsigned hist[256];
    auto key = [v](int64_t i) { return (uint64_t)__double_as_longlong(v[i]); };
    int64_t below;
    uint64_t hi = dm_cta_select(key, m, m / 2, hist, &below);
    double r = __longlong_as_double((long long)hi);
    if (m % 2 == 0) {
        uint64_t lo = dm_cta_select(key, m, m / 2 - 1, hist, &below);
        r = __dmul_rn(0.5, __dadd_rn(__longlong_as_double((long long)lo), r));
    }
    if (threadIdx.x == 0) *result = r;
}

__global__ void scale_points_kernel(const float *__restrict__ X, int64_t n, float c, float *__restrict__ Xs) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) Xs[i] = X[i] * c;
}

// ---- O(N^2) weighted row sums: out_i += sum_j exp2(-|xs_i - xs_j|^2) w_j -----
// grid.x: row blocks of kDegThreads rows; grid.y: column splits.
template <int D>
__global__ void __launch_bounds__(kDegThreads) degree_pass_kernel(const float *__restrict__ Xs, int64_t N, int d,
                                                                  const float *__restrict__ w,
                                                                  double *__restrict__ out, int64_t cols_per_split) {
    constexpr int DS = D > 0 ? D : 1;
    __shared__ float sx[kDegTile * (D > 0 ? D : 8)];
    __shared__ float sw[kDegTile];
    const int64_t i = blockIdx.x * (int64_t)kDegThreads + threadIdx.x;
    const bool valid = i < N;
    float xi[DS];
    if (D > 0) {
#pragma unroll
        for (int k = 0; k < DS; ++k) xi[k] = valid ? Xs[i * D + k] : 0.f;
    }
    const int64_t c0 = blockIdx.y * cols_per_split;
    const int64_t c1 = (c0 + cols_per_split < N) ? c0 + cols_per_split : N;
    double acc = 0.0;
    for (int64_t t0 = c0; t0 < c1; t0 += kDegTile) {
        const int tn = (int)(c1 - t0 < kDegTile ? c1 - t0 : kDegTile);
        __syncthreads();
        if (D > 0) {
            for (int e = threadIdx.x; e < tn * D; e += kDegThreads) sx[e] = Xs[t0 * D + e];
        }
        for (int e = threadIdx.x; e < tn; e += kDegThreads) sw[e] = w ? w[t0 + e] : 1.f;
        __syncthreads();
        float part = 0.f;
        if (D > 0) {
#pragma unroll 4
            for (int j = 0; j < tn; ++j) {
                float r2 = 0.f;
#pragma unroll
                for (int k = 0; k < DS; ++k) {
                    float t = xi[k] - sx[j * D + k];
                    r2 = fmaf(t, t, r2);
                }
                part = fmaf(dm_ex2(-r2), sw[j], part);
            }
        } else if (valid) {
            // generic dimension: coordinates straight from global memory (L1/L2 resident)
            for (int j = 0; j < tn; ++j) {
                const float *xj = Xs + (t0 + j) * d;
                const float *xa = Xs + i * d;
                float r2 = 0.f;
                for (int k = 0; k < d; ++k) {
                    float t = xa[k] - xj[k];
                    r2 = fmaf(t, t, r2);
                }
                part = fmaf(dm_ex2(-r2), sw[j], part);
            }
        }
        acc += (double)part;
    }
    if (valid) atomicAdd(out + i, acc);
}

__global__ void finish_degrees_kernel(int64_t N, double alpha, const double *__restrict__ q,
                                      double *__restrict__ qa, float *__restrict__ qaf) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double v = (alpha == 1.0) ? 1.0 / q[i] : (alpha == 0.0 ? 1.0 : pow(q[i], -alpha));
    qa[i] = v;
    qaf[i] = (float)v;
}

// dg_i = qa_i * sum_j W_ij qa_j (in place over dgsum); s_i = qa_i / sqrt(dg_i)
__global__ void finish_scaling_kernel(int64_t N, const double *__restrict__ qa, double *__restrict__ dg,
                                      double *__restrict__ s, float *__restrict__ sf) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double g = qa[i] * dg[i];
    dg[i] = g;
    double v = qa[i] / sqrt(g);
    s[i] = v;
    sf[i] = (float)v;
}

__global__ void mul_vec_kernel(int64_t N, const float *__restrict__ a, const float *__restrict__ b,
                               float *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) out[i] = a[i] * b[i];
}

__global__ void scale_out_kernel(int64_t N, const float *__restrict__ sf, const double *__restrict__ acc,
                                 float *__restrict__ y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) y[i] = (float)((double)sf[i] * acc[i]);
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t dm_launch_pair_sqdist(const float *X, int64_t N, int d, uint64_t seed, double *out, int64_t m,
                                  cudaStream_t st) {
    int64_t npairs = N * (N - 1) / 2;
    if (npairs == m) {
        all_pairs_kernel<<<blocks_for(N, 128), 128, 0, st>>>(X, N, d, out);
        dm_count_launches(1);
    } else {
        sampled_pairs_kernel<<<blocks_for(m, 256), 256, 0, st>>>(X, N, d, dm_stream_key(seed, DM_TAG_PAIRS, 0),
                                                                  out, m);
        dm_count_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t dm_launch_select_median(double *vals, int64_t m, double *result, cudaStream_t st) {
    median_kernel<<<1, 1024, 0, st>>>(vals, m, result);
    dm_count_launches(1);
    return cudaGetLastError();
}

cudaError_t dm_launch_scale_points(const float *X, int64_t N, int d, double eps, float *Xs, cudaStream_t st) {
    const double log2e = 1.4426950408889634;  // 1/ln 2: exp(-r^2/eps) = 2^(-r^2 log2(e)/eps)
    float c = (float)sqrt(log2e / eps);
    int64_t n = N * d;
    scale_points_kernel<<<blocks_for(n, 256), 256, 0, st>>>(X, n, c, Xs);
    dm_count_launches(1);
    return cudaGetLastError();
}

cudaError_t dm_launch_degree_pass(const float *Xs, int64_t N, int d, const float *wcol, double *out,
                                  cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * N, st);
    if (e != cudaSuccess) return e;
    int64_t rowblocks = (N + kDegThreads - 1) / kDegThreads;
    // enough column splits to put ~16 CTAs on each of the 152 SMs, each split >= 2 tiles
    int64_t want = (16 * 152 + rowblocks - 1) / rowblocks;
    int64_t maxsplit = (N + 2 * kDegTile - 1) / (2 * kDegTile);
    int64_t splits = want < 1 ? 1 : (want > maxsplit ? maxsplit : want);
    if (splits < 1) splits = 1;
    int64_t per = (N + splits - 1) / splits;
    per = (per + kDegTile - 1) / kDegTile * kDegTile;
    splits = (N + per - 1) / per;
    dim3 grid((unsigned)rowblocks, (unsigned)splits);
    switch (d) {
        case 1: degree_pass_kernel<1><<<grid, kDegThreads, 0, st>>>(Xs, N, d, wcol, out, per); dm_count_launches(1); break;
        case 2: degree_pass_kernel<2><<<grid, kDegThreads, 0, st>>>(Xs, N, d, wcol, out, per); dm_count_launches(1); break;
        case 3: degree_pass_kernel<3><<<grid, kDegThreads, 0, st>>>(Xs, N, d, wcol, out, per); dm_count_launches(1); break;
        case 4: degree_pass_kernel<4><<<grid, kDegThreads, 0, st>>>(Xs, N, d, wcol, out, per); dm_count_launches(1); break;
        case 6: degree_pass_kernel<6><<<grid, kDegThreads, 0, st>>>(Xs, N, d, wcol, out, per); dm_count_launches(1); break;
        case 8: degree_pass_kernel<8><<<grid, kDegThreads, 0, st>>>(Xs, N, d, wcol, out, per); dm_count_launches(1); break;
        default: degree_pass_kernel<0><<<grid, kDegThreads, 0, st>>>(Xs, N, d, wcol, out, per); dm_count_launches(1); break;
    }
    return cudaGetLastError();
}

cudaError_t dm_launch_finish_degrees(int64_t N, double alpha, const double *q, double *qa, float *qaf,
                                     cudaStream_t st) {
    finish_degrees_kernel<<<blocks_for(N, 256), 256, 0, st>>>(N, alpha, q, qa, qaf);
    dm_count_launches(1);
    return cudaGetLastError();
}

cudaError_t dm_launch_finish_scaling(int64_t N, const double *qa, double *dgsum, double *s, float *sf,
                                     cudaStream_t st) {
    finish_scaling_kernel<<<blocks_for(N, 256), 256, 0, st>>>(N, qa, dgsum, s, sf);
    dm_count_launches(1);
    return cudaGetLastError();
}

// y = S x exactly: y_i = s_i sum_j W_ij (s_j x_j). `tmpw` holds N floats, `acc` N doubles.
cudaError_t dm_launch_dense_matvec_ws(const float *Xs, const float *sf, int64_t N, int d, const float *x, float *y,
                                      float *tmpw, double *acc, cudaStream_t st) {
    mul_vec_kernel<<<blocks_for(N, 256), 256, 0, st>>>(N, sf, x, tmpw);
    dm_count_launches(1);
    cudaError_t e = dm_launch_degree_pass(Xs, N, d, tmpw, acc, st);
    if (e != cudaSuccess) return e;
    scale_out_kernel<<<blocks_for(N, 256), 256, 0, st>>>(N, sf, acc, y);
    dm_count_launches(1);
    return cudaGetLastError();
}
