// k_degrees.cu -- kernel scale, degree vectors and the exact on-the-fly matvec.
//
// Algorithm 1 of the paper (similarity matrix and normalisations): W_ij = exp(-|x_i - x_j|^2 / eps) (Eq. W),
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

// ---- exact order statistics of m non-negative doubles (their bit patterns order
// like the values) by a multi-block most-significant-digit radix select:
// 11-bit digits, one histogram pass over all values per digit.
constexpr int kSelBits = 11;
constexpr int kSelBins = 1 << kSelBits;

struct SelectState {
    unsigned long long prefix;  // digits found so far
    unsigned long long mask;    // bits they cover
    long long k;                // rank still to find among values matching prefix
    unsigned hist[kSelBins];
};

__global__ void __launch_bounds__(512) select_hist_kernel(const double *__restrict__ v, int64_t m, int shift,
                                                          SelectState *__restrict__ st) {
    __shared__ unsigned h[kSelBins];
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const unsigned long long prefix = st->prefix, mask = st->mask;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < m; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        bool act = false;
        unsigned bin = 0;
        if (i < m) {
            const unsigned long long u = (unsigned long long)__double_as_longlong(v[i]);
            if ((u & mask) == prefix) {
                act = true;
                bin = (unsigned)((u >> shift) & (kSelBins - 1));
            }
        }
        const unsigned am = __ballot_sync(DM_FULL, act);
        if (act) {
            const unsigned peers = __match_any_sync(am, bin);
            if (lane == __ffs(peers) - 1) atomicAdd(&h[bin], (unsigned)__popc(peers));
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x)
        if (h[b]) atomicAdd(&st->hist[b], h[b]);
}

// one block: pick the bin holding rank k, extend the prefix, clear the histogram. Thread t
// sums its `per` bins; a block scan of those sums finds the first thread t <= T - 2 whose
// inclusive count exceeds k (else the last one), and that thread walks its own bins.
__global__ void __launch_bounds__(1024) select_step_kernel(int shift, int bits, SelectState *__restrict__ st) {
    __shared__ long long wsum[32];
    __shared__ int s_t, s_bin;
    __shared__ long long s_before;
    const int per = kSelBins / blockDim.x;  // bins per thread (2 with 1024 threads)
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nt = blockDim.x;
    long long loc = 0;
    for (int q = 0; q < per; ++q) loc += st->hist[t * per + q];
    long long x = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(DM_FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    if (t == 0) s_t = nt - 1;
    __syncthreads();
    long long off = 0;
    for (int w = 0; w < warp; ++w) off += wsum[w];
    const long long incl = off + x, excl = incl - loc;
    const long long k = st->k;
    if (t < nt - 1 && incl > k) atomicMin(&s_t, t);
    __syncthreads();
    if (t == s_t) {
        long long acc = excl;
        int b = t * per;
        for (; b < kSelBins - 1; ++b) {
            if (acc + st->hist[b] > k) break;
            acc += st->hist[b];
        }
        s_bin = b;
        s_before = acc;
    }
    __syncthreads();
    for (int b = t; b < kSelBins; b += nt) st->hist[b] = 0;
    if (t == 0) {
        const unsigned long long digit_mask = ((1ull << bits) - 1ull) << shift;
        st->prefix |= ((unsigned long long)s_bin << shift) & digit_mask;
        st->mask |= digit_mask;
        st->k -= s_before;
    }
}

__global__ void select_init_kernel(SelectState *st, long long k) {
    if (threadIdx.x == 0) {
        st->prefix = 0ull;
        st->mask = 0ull;
        st->k = k;
    }
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) st->hist[b] = 0;
}

// result = 0.5 (lo + hi) for an even count, else hi (matching the oracle's arithmetic)
__global__ void median_finish_kernel(const SelectState *lo, const SelectState *hi, int even, double *result) {
    const double h = __longlong_as_double((long long)hi->prefix);
    *result = even ? __dmul_rn(0.5, __dadd_rn(__longlong_as_double((long long)lo->prefix), h)) : h;
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

// d = 3 specialisation, two rows per thread in packed FP32x2 arithmetic.
// With centred, pre-scaled coordinates u and n = |u|^2 the entry is
//   2^-|u_i - u_j|^2 = 2^-n_i * 2^(2 u_i.u_j - n_j),
// three FMAs and one MUFU ex2 per entry; the row factor 2^-n_i is applied once per
// row in FP64. The form is used when every n <= kDotFormMaxNorm (device flag), so
// the exponent stays below 2^8 in magnitude and its rounding below ~2e-6 relative
// per entry; otherwise the direct difference form runs. The shared tile holds each
// column duplicated as pairs so that 128-bit loads feed the packed operands.
constexpr int kD3Threads = 128;
constexpr int kD3Rows = 4 * kD3Threads;  // four rows per thread: two packed pairs
constexpr float kDotFormMaxNorm = 8.f;
#ifndef DM_SYM_ROW_PAIRS
#define DM_SYM_ROW_PAIRS 4
#endif
constexpr int kSymRowPairs = DM_SYM_ROW_PAIRS;  // row pairs per thread of the symmetric pass
#ifndef DM_SYM_MIN_BLOCKS
#define DM_SYM_MIN_BLOCKS 10
#endif
constexpr int kSymMinBlocks = DM_SYM_MIN_BLOCKS;  // CTAs per SM the register budget is sized for

struct Rows4 {
    float2 x0[2], x1[2], x2[2];
};

__global__ void __launch_bounds__(kD3Threads) degree_pass_d3_kernel(const float *__restrict__ Xs,
                                                                    const float *__restrict__ nrm,
                                                                    const float *__restrict__ nmax, int64_t N,
                                                                    const float *__restrict__ w,
                                                                    double *__restrict__ out,
                                                                    int64_t cols_per_split) {
    __shared__ float4 ta[kDegTile];
    __shared__ float4 tb[kDegTile];
    __shared__ float2 tw[kDegTile];
    const bool dot_form = nrm != nullptr && *nmax <= kDotFormMaxNorm;
    const float sc = dot_form ? 2.f : 1.f;
    // rows of this thread: base + threadIdx.x + {0, 1, 2, 3} * kD3Threads; pair p holds rows 2p, 2p+1
    const int64_t row0 = blockIdx.x * (int64_t)kD3Rows + threadIdx.x;
    float xr[4][3];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t rq = row0 + (int64_t)q * kD3Threads;
#pragma unroll
        for (int k = 0; k < 3; ++k) xr[q][k] = rq < N ? sc * Xs[rq * 3 + k] : 0.f;
    }
    Rows4 X;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        X.x0[p] = make_float2(xr[2 * p][0], xr[2 * p + 1][0]);
        X.x1[p] = make_float2(xr[2 * p][1], xr[2 * p + 1][1]);
        X.x2[p] = make_float2(xr[2 * p][2], xr[2 * p + 1][2]);
    }
    const int64_t c0 = blockIdx.y * cols_per_split;
    const int64_t c1 = (c0 + cols_per_split < N) ? c0 + cols_per_split : N;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t t0 = c0; t0 < c1; t0 += kDegTile) {
        const int tn = (int)(c1 - t0 < kDegTile ? c1 - t0 : kDegTile);
        __syncthreads();
        for (int e = threadIdx.x; e < tn; e += kD3Threads) {
            const int64_t j = t0 + e;
            const float x = Xs[j * 3], y = Xs[j * 3 + 1], z = Xs[j * 3 + 2];
            const float wj = w ? w[j] : 1.f;
            if (dot_form) {
                const float nj = -nrm[j];
                ta[e] = make_float4(x, x, y, y);
                tb[e] = make_float4(z, z, nj, nj);
            } else {
                ta[e] = make_float4(-x, -x, -y, -y);
                tb[e] = make_float4(-z, -z, 0.f, 0.f);
            }
            tw[e] = make_float2(wj, wj);
        }
        __syncthreads();
        float2 part0 = make_float2(0.f, 0.f), part1 = make_float2(0.f, 0.f);
        if (dot_form) {
#pragma unroll 2
            for (int j = 0; j < tn; ++j) {
                const float4 a = ta[j], b = tb[j];
                const float2 wj = tw[j];
                const float2 cx = make_float2(a.x, a.y), cy = make_float2(a.z, a.w), cz = make_float2(b.x, b.y);
                const float2 cn = make_float2(b.z, b.w);
                float2 g0 = __ffma2_rn(X.x2[0], cz, cn);
                float2 g1 = __ffma2_rn(X.x2[1], cz, cn);
                g0 = __ffma2_rn(X.x1[0], cy, g0);
                g1 = __ffma2_rn(X.x1[1], cy, g1);
                g0 = __ffma2_rn(X.x0[0], cx, g0);
                g1 = __ffma2_rn(X.x0[1], cx, g1);
                const float2 e0 = make_float2(dm_ex2(g0.x), dm_ex2(g0.y));
                const float2 e1 = make_float2(dm_ex2(g1.x), dm_ex2(g1.y));
                part0 = __ffma2_rn(e0, wj, part0);
                part1 = __ffma2_rn(e1, wj, part1);
            }
        } else {
#pragma unroll 2
            for (int j = 0; j < tn; ++j) {
                const float4 a = ta[j], b = tb[j];
                const float2 wj = tw[j];
                const float2 cx = make_float2(a.x, a.y), cy = make_float2(a.z, a.w), cz = make_float2(b.x, b.y);
                float2 d0 = __fadd2_rn(X.x0[0], cx), e0 = __fadd2_rn(X.x0[1], cx);
                float2 d1 = __fadd2_rn(X.x1[0], cy), e1 = __fadd2_rn(X.x1[1], cy);
                float2 d2 = __fadd2_rn(X.x2[0], cz), e2 = __fadd2_rn(X.x2[1], cz);
                float2 r0 = __fmul2_rn(d0, d0), r1 = __fmul2_rn(e0, e0);
                r0 = __ffma2_rn(d1, d1, r0);
                r1 = __ffma2_rn(e1, e1, r1);
                r0 = __ffma2_rn(d2, d2, r0);
                r1 = __ffma2_rn(e2, e2, r1);
                const float2 x0 = make_float2(dm_ex2(-r0.x), dm_ex2(-r0.y));
                const float2 x1 = make_float2(dm_ex2(-r1.x), dm_ex2(-r1.y));
                part0 = __ffma2_rn(x0, wj, part0);
                part1 = __ffma2_rn(x1, wj, part1);
            }
        }
        acc[0] += (double)part0.x;
        acc[1] += (double)part0.y;
        acc[2] += (double)part1.x;
        acc[3] += (double)part1.y;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t rq = row0 + (int64_t)q * kD3Threads;
        if (rq >= N) continue;
        double v = acc[q];
        if (dot_form) v *= (double)dm_ex2(-nrm[rq]);
        atomicAdd(out + rq, v);
    }
}

// Symmetric form of the d = 3 pass: W is symmetric, so only the tiles (I, J) with J >= I of
// the row blocks (kD3Rows = 512 points each) are evaluated. A tile adds each entry to its row
// sum (thread-local, as in degree_pass_d3_kernel) and, when J > I, also to its column sum:
// w_i e_ij over the block's 512 rows. Column partials are collected per thread for 32
// columns at a time and folded across the warp by a reduce-scatter (31 shuffles leave lane
// l with column l's sum), then the four warps meet in shared memory and each tile column
// gets one FP64 atomic. Half the exponentials of the full pass; the same per-entry
// arithmetic (dot form with the row factor 2^-n_i applied once per row, or the difference
// form), FP32 tile partials and FP64 accumulation.
__device__ __forceinline__ float warp_reduce_scatter32(float (&v)[32], int lane) {
#pragma unroll
    for (int sft = 16; sft >= 1; sft >>= 1) {
        const bool upper = (lane & sft) != 0;
#pragma unroll
        for (int i = 0; i < sft; ++i) {
            const float send = upper ? v[i] : v[i + sft];
            const float keep = upper ? v[i + sft] : v[i];
            v[i] = keep + __shfl_xor_sync(DM_FULL, send, sft);
        }
    }
    return v[0];
}

template <int RP>
__global__ void __launch_bounds__(kD3Rows / (2 * RP), kSymMinBlocks) degree_sym_d3_kernel(const float *__restrict__ Xs,
                                                                           const float *__restrict__ nrm,
                                                                           const float *__restrict__ nmax, int64_t N,
                                                                           const float *__restrict__ w,
                                                                           double *__restrict__ out, int nb) {
    // RP packed row pairs per thread: 2 RP rows of the tile against each column, so the
    // column's shared loads and its lane reduce-scatter are shared by 2 RP entries
    constexpr int T = kD3Rows / (2 * RP);
    __shared__ float4 ta[kDegTile];
    __shared__ float4 tb[kDegTile];
    __shared__ float2 tw[kDegTile];
    __shared__ float colsum[kDegTile];
    // tile (I, J), J >= I, from the flat index: row I of the triangle starts at I nb - I (I - 1) / 2
    const int64_t t = blockIdx.x;
    const double B2 = 2.0 * nb + 1.0;
    int I = (int)floor((B2 - sqrt(fmax(B2 * B2 - 8.0 * (double)t, 0.0))) * 0.5);
    auto start = [&](int64_t r) { return r * nb - r * (r - 1) / 2; };
    while (I > 0 && start(I) > t) --I;
    while (start(I + 1) <= t) ++I;
    const int J = I + (int)(t - start(I));
    const bool offdiag = J > I;
    const bool dot_form = nrm != nullptr && *nmax <= kDotFormMaxNorm;
    const float sc = dot_form ? 2.f : 1.f;
    const int lane = threadIdx.x & 31;
    // rows of this thread: I kD3Rows + threadIdx.x + q T, q < 2 RP; pair p holds rows 2p, 2p+1
    const int64_t row0 = (int64_t)I * kD3Rows + threadIdx.x;
    float2 X0[RP], X1[RP], X2[RP], W[RP];
#pragma unroll
    for (int p = 0; p < RP; ++p) {
        float xr[2][3], wr[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t rq = row0 + (int64_t)(2 * p + h) * T;
            const bool ok = rq < N;
#pragma unroll
            for (int k = 0; k < 3; ++k) xr[h][k] = ok ? sc * Xs[rq * 3 + k] : 0.f;
            // column weights: w_i, times the row factor 2^-n_i in the dot form
            wr[h] = ok ? (w ? w[rq] : 1.f) * (dot_form ? dm_ex2(-nrm[rq]) : 1.f) : 0.f;
        }
        X0[p] = make_float2(xr[0][0], xr[1][0]);
        X1[p] = make_float2(xr[0][1], xr[1][1]);
        X2[p] = make_float2(xr[0][2], xr[1][2]);
        W[p] = make_float2(wr[0], wr[1]);
    }
    const int64_t c0 = (int64_t)J * kD3Rows;
    const int64_t c1 = (c0 + kD3Rows < N) ? c0 + kD3Rows : N;
    // FP64 row sums in shared memory (touched once per column tile), keeping registers for the
    // packed inner loop so that more CTAs fit on an SM
    __shared__ double acc_s[2 * RP][T];
#pragma unroll
    for (int q = 0; q < 2 * RP; ++q) acc_s[q][threadIdx.x] = 0.0;
    for (int64_t t0 = c0; t0 < c1; t0 += kDegTile) {
        const int tn = (int)(c1 - t0 < kDegTile ? c1 - t0 : kDegTile);
        __syncthreads();
        for (int e = threadIdx.x; e < kDegTile; e += T) {
            colsum[e] = 0.f;
            if (e >= tn) continue;
            const int64_t j = t0 + e;
            const float x = Xs[j * 3], y = Xs[j * 3 + 1], z = Xs[j * 3 + 2];
            const float wj = w ? w[j] : 1.f;
            if (dot_form) {
                const float nj = -nrm[j];
                ta[e] = make_float4(x, x, y, y);
                tb[e] = make_float4(z, z, nj, nj);
            } else {
                ta[e] = make_float4(-x, -x, -y, -y);
                tb[e] = make_float4(-z, -z, 0.f, 0.f);
            }
            tw[e] = make_float2(wj, wj);
        }
        __syncthreads();
        float2 part[RP];
#pragma unroll
        for (int p = 0; p < RP; ++p) part[p] = make_float2(0.f, 0.f);
        for (int jc = 0; jc < tn; jc += 32) {
            float cp[32];
#pragma unroll
            for (int u = 0; u < 32; ++u) {
                const int j = jc + u;
                cp[u] = 0.f;
                if (j < tn) {
                    const float4 a = ta[j], b = tb[j];
                    const float2 wj = tw[j];
                    const float2 cx = make_float2(a.x, a.y), cy = make_float2(a.z, a.w), cz = make_float2(b.x, b.y);
                    float2 e[RP];
                    if (dot_form) {
                        const float2 cn = make_float2(b.z, b.w);
#pragma unroll
                        for (int p = 0; p < RP; ++p) {
                            float2 g = __ffma2_rn(X2[p], cz, cn);
                            g = __ffma2_rn(X1[p], cy, g);
                            g = __ffma2_rn(X0[p], cx, g);
                            e[p] = make_float2(dm_ex2(g.x), dm_ex2(g.y));
                        }
                    } else {
#pragma unroll
                        for (int p = 0; p < RP; ++p) {
                            const float2 d0 = __fadd2_rn(X0[p], cx), d1 = __fadd2_rn(X1[p], cy),
                                         d2 = __fadd2_rn(X2[p], cz);
                            float2 r = __fmul2_rn(d0, d0);
                            r = __ffma2_rn(d1, d1, r);
                            r = __ffma2_rn(d2, d2, r);
                            e[p] = make_float2(dm_ex2(-r.x), dm_ex2(-r.y));
                        }
                    }
#pragma unroll
                    for (int p = 0; p < RP; ++p) part[p] = __ffma2_rn(e[p], wj, part[p]);
                    if (offdiag) {
                        float2 c2 = __fmul2_rn(e[RP - 1], W[RP - 1]);
#pragma unroll
                        for (int p = RP - 2; p >= 0; --p) c2 = __ffma2_rn(e[p], W[p], c2);
                        cp[u] = c2.x + c2.y;
                    }
                }
            }
            if (offdiag) {
                const float v = warp_reduce_scatter32(cp, lane);
                if (jc + lane < tn) atomicAdd(&colsum[jc + lane], v);
            }
        }
#pragma unroll
        for (int p = 0; p < RP; ++p) {
            acc_s[2 * p][threadIdx.x] += (double)part[p].x;
            acc_s[2 * p + 1][threadIdx.x] += (double)part[p].y;
        }
        if (offdiag) {
            __syncthreads();
            for (int e = threadIdx.x; e < tn; e += T) atomicAdd(out + t0 + e, (double)colsum[e]);
        }
    }
#pragma unroll
    for (int q = 0; q < 2 * RP; ++q) {
        const int64_t rq = row0 + (int64_t)q * T;
        if (rq >= N) continue;
        double v = acc_s[q][threadIdx.x];
        if (dot_form) v *= (double)dm_ex2(-nrm[rq]);
        atomicAdd(out + rq, v);
    }
}

// column sums of X (FP64) for the centring
__global__ void colsum_kernel(const float *__restrict__ X, int64_t N, int d, double *__restrict__ sums) {
    double loc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int dd = d < 8 ? d : 8;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < dd; ++k) loc[k] += (double)X[i * d + k];
    for (int k = 0; k < dd; ++k) {
        const double v = dm_warp_sum_d(loc[k]);
        if ((threadIdx.x & 31) == 0) atomicAdd(sums + k, v);
    }
}

// u = (x - mean) * c, n = |u|^2 (FP32, k = 0..d-1), running max of n
__global__ void center_scale_kernel(const float *__restrict__ X, int64_t N, int d, const double *__restrict__ sums,
                                    float c, float *__restrict__ Xs, float *__restrict__ nrm,
                                    unsigned *__restrict__ nmax_bits) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float n = 0.f;
    if (i < N) {
        for (int k = 0; k < d; ++k) {
            const double mean = k < 8 ? sums[k] / (double)N : 0.0;
            const float u = (float)((double)X[i * d + k] - mean) * c;
            Xs[i * d + k] = u;
            n = fmaf(u, u, n);
        }
        nrm[i] = n;
    }
    unsigned m = __float_as_uint(n);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(DM_FULL, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(nmax_bits, m);
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
    const uint64_t key = dm_stream_key(seed, DM_TAG_PAIRS, 0);
    if (npairs == m) all_pairs_kernel<<<blocks_for(N, 128), 128, 0, st>>>(X, N, d, out);
    else sampled_pairs_kernel<<<blocks_for(m, 256), 256, 0, st>>>(X, N, d, key, out, m);
    dm_count_launches(1);
    return cudaGetLastError();
}

namespace {
__global__ void widen_kernel(const float *__restrict__ X, int64_t n, double *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)X[i];
}
}  // namespace

cudaError_t dm_launch_widen(const float *X, int64_t n, double *out, cudaStream_t st) {
    const int64_t b = (n + 255) / 256;
    widen_kernel<<<(unsigned)(b < 8 * 152 ? (b > 0 ? b : 1) : 8 * 152), 256, 0, st>>>(X, n, out);
    dm_count_launches(1);
    return cudaGetLastError();
}

size_t dm_select_state_bytes() { return sizeof(SelectState); }

// exact median of vals[0..m): two radix selects (ranks m/2-1 and m/2) into two
// SelectState records at `state` (2 * dm_select_state_bytes() of device memory)
cudaError_t dm_launch_select_median(double *vals, int64_t m, void *state, double *result, cudaStream_t st,
                                    cudaStream_t st2, cudaEvent_t fork, cudaEvent_t join) {
    SelectState *S = reinterpret_cast<SelectState *>(state);
    const int even = (m % 2 == 0) ? 1 : 0;
    const long long ranks[2] = {even ? m / 2 - 1 : m / 2, m / 2};
    const int blocks = (int)((m + 511) / 512 < 2 * 152 ? (m + 511) / 512 : 2 * 152);
    // the two selects are independent chains of small launches: the second runs on st2
    // (when given) at the same time as the first
    const bool two = st2 != nullptr && fork != nullptr && join != nullptr;
    cudaError_t e;
    if (two) {
        if ((e = cudaEventRecord(fork, st)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(st2, fork, 0)) != cudaSuccess) return e;
    }
    for (int r = 0; r < 2; ++r) {
        const cudaStream_t sr = (two && r == 1) ? st2 : st;
        select_init_kernel<<<1, 256, 0, sr>>>(S + r, ranks[r]);
        dm_count_launches(1);
        for (int top = 64; top > 0; top -= kSelBits) {
            const int bits = top >= kSelBits ? kSelBits : top;
            const int shift = top - bits;
            select_hist_kernel<<<blocks, 512, 0, sr>>>(vals, m, shift, S + r);
            dm_count_launches(1);
            select_step_kernel<<<1, 1024, 0, sr>>>(shift, bits, S + r);
            dm_count_launches(1);
        }
    }
    if (two) {
        if ((e = cudaEventRecord(join, st2)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(st, join, 0)) != cudaSuccess) return e;
    }
    median_finish_kernel<<<1, 1, 0, st>>>(S, S + 1, even, result);
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

// centred, pre-scaled points u = (x - mean) sqrt(log2(e)/eps), their squared norms and max
// (`work` holds 8 doubles + 1 unsigned of device memory)
cudaError_t dm_launch_center_scale(const float *X, int64_t N, int d, double eps, float *Xs, float *nrm, float *nmax,
                                   double *work, cudaStream_t st) {
    const double log2e = 1.4426950408889634;
    const float c = (float)sqrt(log2e / eps);
    cudaError_t e = cudaMemsetAsync(work, 0, sizeof(double) * 8, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(nmax, 0, sizeof(float), st);
    if (e != cudaSuccess) return e;
    colsum_kernel<<<(unsigned)((N + 255) / 256 < 304 ? (N + 255) / 256 : 304), 256, 0, st>>>(X, N, d, work);
    dm_count_launches(1);
    center_scale_kernel<<<blocks_for(N, 256), 256, 0, st>>>(X, N, d, work, c, Xs, nrm,
                                                            reinterpret_cast<unsigned *>(nmax));
    dm_count_launches(1);
    return cudaGetLastError();
}

cudaError_t dm_launch_degree_pass_centered(const float *Xs, const float *nrm, const float *nmax, int64_t N, int d,
                                           const float *wcol, double *out, cudaStream_t st);

cudaError_t dm_launch_degree_pass(const float *Xs, int64_t N, int d, const float *wcol, double *out,
                                  cudaStream_t st) {
    return dm_launch_degree_pass_centered(Xs, nullptr, nullptr, N, d, wcol, out, st);
}

// out_i = sum_j W_ij w_j. nrm/nmax (may be NULL) enable the centred dot-product form at d = 3:
// Xs must then be centred and pre-scaled with nrm its squared norms.
cudaError_t dm_launch_degree_pass_centered(const float *Xs, const float *nrm, const float *nmax, int64_t N, int d,
                                           const float *wcol, double *out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * N, st);
    if (e != cudaSuccess) return e;
    if (d == 3 && N >= 4 * kD3Rows) {
        // symmetric tiles: half the entries
        const int64_t nb = (N + kD3Rows - 1) / kD3Rows;
        const int64_t tiles = nb * (nb + 1) / 2;
        degree_sym_d3_kernel<kSymRowPairs><<<(unsigned)tiles, kD3Rows / (2 * kSymRowPairs), 0, st>>>(
            Xs, nrm, nmax, N, wcol, out, (int)nb);
        dm_count_launches(1);
        return cudaGetLastError();
    }
    if (d == 3) {
        const int64_t rb = (N + kD3Rows - 1) / kD3Rows;
        int64_t want = (12 * 152 + rb - 1) / rb;
        const int64_t maxs = (N + 2 * kDegTile - 1) / (2 * kDegTile);
        int64_t sp = want < 1 ? 1 : (want > maxs ? maxs : want);
        if (sp < 1) sp = 1;
        int64_t per = (N + sp - 1) / sp;
        per = (per + kDegTile - 1) / kDegTile * kDegTile;
        sp = (N + per - 1) / per;
        degree_pass_d3_kernel<<<dim3((unsigned)rb, (unsigned)sp), kD3Threads, 0, st>>>(Xs, nrm, nmax, N, wcol, out,
                                                                                       per);
        dm_count_launches(1);
        return cudaGetLastError();
    }
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

// Throughput of the MUFU ex2 instruction (the exponential of every kernel entry): each thread
// runs 8 independent chains x <- ex2(-x / 2) (one FMA-pipe multiply and one MUFU ex2 per
// link; the values stay in (0.5, 1]), so with 64 warps per SM the MUFU pipe, not latency,
// sets the rate. The result is written so no chain is eliminated.
__global__ void __launch_bounds__(256) ex2_peak_kernel(float *out, int iters) {
    float a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = 0.5f + 0.01f * (float)u + 1e-7f * (float)threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = dm_ex2(-0.5f * a[u]);
    }
    float s = 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u) s += a[u];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

cudaError_t dm_launch_ex2_peak(float *out, int blocks, int iters, cudaStream_t st) {
    ex2_peak_kernel<<<blocks, 256, 0, st>>>(out, iters);
    dm_count_launches(1);
    return cudaGetLastError();
}
