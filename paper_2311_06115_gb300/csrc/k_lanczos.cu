// k_lanczos.cu -- Lanczos with full reorthogonalisation on the device.
//
// Algorithm 2 of the paper (k-step Arnoldi factorisation) in its symmetric form,
// the Lanczos method of Section 2.3.1 that eigsh/ARPACK runs: x_1 = v/|v|; per
// step z = A x_j, h = X^T z, r = z - X h (Gram-Schmidt, done twice here), the
// projected matrix is tridiagonal T = tridiag(beta, alpha, beta) with
// alpha_j = h_j and beta_j = |r|. Ritz values of T (its eigenvalues) approximate
// those of A; a Ritz pair has residual |A phi - theta phi| = beta_m |y_m|.
//
// GB300 design: the basis X is FP32 (HBM-bound passes), every dot product is a
// warp-level FP32 partial folded into FP64 atomics (FP64 is a narrow pipe on
// this part, so it is spent only on the coefficients), and the small tridiagonal
// eigenproblem is solved in FP64 with division-free Sturm sequences
// (multisection: 32 shifts per warp per round) and inverse iteration.
#include <map>
#include <mutex>

#include "dm_internal.cuh"

namespace {

constexpr int kKMax = 32;        // max eigenpairs returned per solve

__global__ void start_vector_kernel(const int32_t *__restrict__ perm, int64_t N, uint64_t key, float *__restrict__ z,
                                    double *__restrict__ nrm2) {
    int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float v = 0.f;
    if (pos < N) {
        v = (float)(2.0 * dm_unit(dm_rng(key, (uint64_t)perm[pos])) - 1.0);
        z[pos] = v;
    }
    float ss = dm_warp_sum(v * v);
    if ((threadIdx.x & 31) == 0) atomicAdd(nrm2, (double)ss);
}

// V[:, col] = z / sqrt(nrm2)
__global__ void normalize_kernel(const float *__restrict__ z, int64_t N, const double *__restrict__ nrm2,
                                 float *__restrict__ vout) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) vout[i] = (float)((double)z[i] / sqrt(*nrm2));
}



// ---- one fused Lanczos orthogonalisation step (cooperative launch) --------------
// Classical Gram-Schmidt twice, in three passes over this block's rows of V:
//   A  h0 = V^T z                                              | grid barrier
//   B  z' = z - V h0, then h1 = V^T z' and |z'|^2 (same rows)   | grid barrier
//   C  z'' = z' - V h1, beta_j = |z''| = sqrt(|z'|^2 - |h1|^2),
//      alpha_j = h0_j + h1_j, V[:, j+1] = z'' / beta_j
// |z''|^2 = |z'|^2 - 2 h1^T V^T z' + h1^T V^T V h1 = |z'|^2 - |h1|^2 because V^T z' = h1
// and V has orthonormal columns (to FP32 rounding after the first pass); the second
// pass's correction h1 is O(FP32 eps |z'|), so the difference loses nothing.
//
// Work layout: rows in 16-byte quads (V and z are zero padded to ldv, a multiple of 64);
// a warp item is 32 consecutive quads x 8 columns, so every lane has eight 16-byte loads
// in flight. Dot products reduce by a reduce-scatter over the lanes (9 shuffles for 8
// columns) into shared FP32 partials, then one FP64 atomic per column and block. The
// update V h sums its per-chunk float4 partials in a fixed order (deterministic z').
// The projection accumulators are double-buffered by step parity: block 0 clears the
// other parity's set during step j, so no step needs a memset of its own; the barrier
// counter grows monotonically within a solve (targets (2j+1) G and (2j+2) G).
// Barriers spin with a bounded iteration count; on exhaustion they raise *err and every
// block returns (the host reports a timeout).
// block sizes: 512 threads, one block per SM, for the cooperative step (fewer arrivals at
// each grid barrier); 256 threads, two per SM, for the phased step of a shared device (small
// blocks that fit beside other solves' kernels)
constexpr int kStepThreadsCoop = 512;
constexpr int kStepThreadsPhased = 256;
// sum of v[u] over the 32 lanes, scattered: lanes with (lane & 3) == 0 end up holding
// the total for u = 4 b4 + 2 b3 + b2 (b_k = bit k of the lane); returns that value
__device__ __forceinline__ float reduce_scatter8(float (&v)[8], int lane) {
#pragma unroll
    for (int sft = 16, half = 4; sft >= 4; sft >>= 1, half >>= 1) {
        const bool upper = (lane & sft) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = upper ? v[i] : v[i + half];
            const float keep = upper ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(DM_FULL, send, sft);
        }
    }
    float r = v[0];
    r += __shfl_xor_sync(DM_FULL, r, 2);
    r += __shfl_xor_sync(DM_FULL, r, 1);
    return r;
}
__device__ __forceinline__ int scatter8_index(int lane) {
    return ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
}

__device__ __forceinline__ float4 ldq(const float *col, int64_t q) {
    return __ldcg(reinterpret_cast<const float4 *>(col) + q);
}

// acc[c] += sum over quads q0..q0+nq-1 of V(q, c) . y(q), c < ncols (shared FP32 partials);
// y is global (ys == nullptr: read yg from quad q0) or a shared tile
template <int kStepWarps>
__device__ void tile_project(const float *V, int64_t ldv, int ncols, const float *yg, const float4 *ys, int64_t q0,
                             int nq, float *acc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nch = (ncols + 7) >> 3, ng = (nq + 31) >> 5;
    for (int it = warp; it < nch * ng; it += kStepWarps) {
        const int g = it / nch, cc = it - g * nch;
        const int ql = g * 32 + lane;
        float p[8];
        if (ql < nq) {
            const float4 y = ys ? ys[ql] : ldq(yg, q0 + ql);
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                v[u] = (cc * 8 + u < ncols) ? ldq(V + (size_t)(cc * 8 + u) * ldv, q0 + ql) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 8; ++u) p[u] = fmaf(v[u].x, y.x, fmaf(v[u].y, y.y, fmaf(v[u].z, y.z, v[u].w * y.w)));
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) p[u] = 0.f;
        }
        const float r = reduce_scatter8(p, lane);
        const int c = cc * 8 + scatter8_index(lane);
        if ((lane & 3) == 0 && c < ncols) atomicAdd(acc + c, r);
    }
}

// part[cs][ql] = sum over chunks cc = cs, cs + ncs, ... (ncs = min(chunks, warps)) of
// sum_{c in cc} hs[c] V(q0 + ql, c): warp w takes chunk slot w % ncs of the quad groups
// w / ncs, w / ncs + gpr, ... (gpr = warps / ncs groups side by side)
template <int kStepWarps>
__device__ void tile_combine(const float *V, int64_t ldv, int ncols, const float *hs, int64_t q0, int nq, int qt,
                             float4 *part) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nch = (ncols + 7) >> 3, ng = (nq + 31) >> 5;
    const int ncs = nch < kStepWarps ? nch : kStepWarps, gpr = kStepWarps / ncs;
    const int cs = warp % ncs, gs = warp / ncs;
    if (gs >= gpr) return;
    for (int g = gs; g < ng; g += gpr) {
        const int ql = g * 32 + lane;
        if (ql >= nq) continue;
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int cc = cs; cc < nch; cc += ncs) {
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                v[u] = (cc * 8 + u < ncols) ? ldq(V + (size_t)(cc * 8 + u) * ldv, q0 + ql)
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float hc = hs[cc * 8 + u];  // zero past ncols
                s.x = fmaf(hc, v[u].x, s.x);
                s.y = fmaf(hc, v[u].y, s.y);
                s.z = fmaf(hc, v[u].z, s.z);
                s.w = fmaf(hc, v[u].w, s.w);
            }
        }
        part[(size_t)cs * qt + ql] = s;
    }
}

// z - (part[0][ql] + part[1][ql] + ...), slots in a fixed order
template <int kStepWarps>
__device__ __forceinline__ float4 sub_parts(float4 z, const float4 *part, int ncols, int qt, int ql) {
    const int nch = (ncols + 7) >> 3, ncs = nch < kStepWarps ? nch : kStepWarps;
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int cs = 0; cs < ncs; ++cs) {
        const float4 p = part[(size_t)cs * qt + ql];
        s.x += p.x;
        s.y += p.y;
        s.z += p.z;
        s.w += p.w;
    }
    return make_float4(z.x - s.x, z.y - s.y, z.z - s.z, z.w - s.w);
}

// body of the step for one problem: block `bid` of `nblk` blocks (its rows); shared by the
// single-problem launches and the batched one (phased passes only)
template <int NT>
__device__ __forceinline__ void lanczos_step_body(float *V, int64_t ldv, int j, float *z, double *hbuf, int hstride,
                                                  double *alpha, double *beta, int m_max, int qt, unsigned *bar,
                                                  int *err, int phase, int bid, int nblk) {
    constexpr int kStepWarps = NT / 32;
    // phase < 0: the whole step in one cooperative launch, passes separated by grid
    // barriers; phase 0..2: that pass alone (ordinary launches, the kernel boundary
    // is the barrier)
    const int nchmax = (m_max + 1 + 7) >> 3;
    extern __shared__ float4 sh4[];
    float4 *part = sh4;                                            // warps x qt
    float4 *zs = part + (size_t)kStepWarps * qt;                  // qt
    float *hs = reinterpret_cast<float *>(zs + qt);               // 8 nchmax coefficients
    float *acc = hs + 8 * nchmax;                                  // 8 nchmax partial sums
    __shared__ float red[kStepWarps];
    __shared__ double s_beta;
    const int ncols = j + 1, nch = (ncols + 7) >> 3;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double *h0 = hbuf + (size_t)(j & 1) * hstride, *h1 = h0 + (m_max + 1), *nz = h1 + (m_max + 1);
    double *other = hbuf + (size_t)((j + 1) & 1) * hstride;
    const int64_t Qn = ldv >> 2;
    const int64_t per = (Qn + nblk - 1) / nblk;
    const int64_t qb0 = bid * per, qb1 = (qb0 + per < Qn) ? qb0 + per : Qn;
    const unsigned G = (unsigned)nblk;
    const bool all = phase < 0;

    if (all || phase == 0) {  // ---- A: h0 = V^T z
        for (int c = threadIdx.x; c < 8 * nch; c += blockDim.x) acc[c] = 0.f;
        __syncthreads();
        for (int64_t q0 = qb0; q0 < qb1; q0 += qt)
            tile_project<kStepWarps>(V, ldv, ncols, z, nullptr, q0, (int)(qb1 - q0 < qt ? qb1 - q0 : qt), acc);
        __syncthreads();
        for (int c = threadIdx.x; c < ncols; c += blockDim.x) atomicAdd(h0 + c, (double)acc[c]);
    }
    if (all && !grid_barrier(bar, (2u * (unsigned)j + 1u) * G, err)) return;
    if (all || phase == 1) {  // ---- B: z' = z - V h0; h1 = V^T z'; |z'|^2
        for (int c = threadIdx.x; c < 8 * nch; c += blockDim.x) {
            hs[c] = c < ncols ? (float)__ldcg(h0 + c) : 0.f;
            acc[c] = 0.f;
        }
        float ss = 0.f;
        for (int64_t q0 = qb0; q0 < qb1; q0 += qt) {
            const int nq = (int)(qb1 - q0 < qt ? qb1 - q0 : qt);
            __syncthreads();
            tile_combine<kStepWarps>(V, ldv, ncols, hs, q0, nq, qt, part);
            __syncthreads();
            for (int ql = threadIdx.x; ql < nq; ql += blockDim.x) {
                const float4 zp = sub_parts<kStepWarps>(ldq(z, q0 + ql), part, ncols, qt, ql);
                zs[ql] = zp;
                reinterpret_cast<float4 *>(z)[q0 + ql] = zp;
                ss = fmaf(zp.x, zp.x, fmaf(zp.y, zp.y, fmaf(zp.z, zp.z, fmaf(zp.w, zp.w, ss))));
            }
            __syncthreads();
            tile_project<kStepWarps>(V, ldv, ncols, nullptr, zs, q0, nq, acc);
        }
        ss = dm_warp_sum(ss);
        if (lane == 0) red[warp] = ss;
        __syncthreads();
        for (int c = threadIdx.x; c < ncols; c += blockDim.x) atomicAdd(h1 + c, (double)acc[c]);
        if (threadIdx.x == 0) {
            float t = 0.f;
            for (int w = 0; w < kStepWarps; ++w) t += red[w];
            atomicAdd(nz, (double)t);
        }
    }
    if (all && !grid_barrier(bar, (2u * (unsigned)j + 2u) * G, err)) return;
    if (!all && phase != 2) return;
    // ---- C: z'' = z' - V h1, beta_j, V[:, j+1] = z'' / beta_j
    for (int c = threadIdx.x; c < 8 * nch; c += blockDim.x) hs[c] = c < ncols ? (float)__ldcg(h1 + c) : 0.f;
    if (warp == 0) {
        double t = 0.0;
        for (int c = lane; c < ncols; c += 32) {
            const double v = __ldcg(h1 + c);
            t = fma(v, v, t);
        }
        t = dm_warp_sum_d(t);
        if (lane == 0) s_beta = sqrt(fmax(__ldcg(nz) - t, 0.0));
    }
    __syncthreads();
    const double b = s_beta;
    const float inv = b > 0.0 ? (float)(1.0 / b) : 0.f;
    float *vn = (j + 1 <= m_max) ? V + (size_t)(j + 1) * ldv : nullptr;
    for (int64_t q0 = qb0; q0 < qb1; q0 += qt) {
        const int nq = (int)(qb1 - q0 < qt ? qb1 - q0 : qt);
        __syncthreads();
        tile_combine<kStepWarps>(V, ldv, ncols, hs, q0, nq, qt, part);
        __syncthreads();
        if (vn)
            for (int ql = threadIdx.x; ql < nq; ql += blockDim.x) {
                const float4 zpp = sub_parts<kStepWarps>(ldq(z, q0 + ql), part, ncols, qt, ql);
                reinterpret_cast<float4 *>(vn)[q0 + ql] = make_float4(zpp.x * inv, zpp.y * inv, zpp.z * inv, zpp.w * inv);
            }
    }
    // block 0 records the coefficients and clears the other parity's accumulators, which
    // step j + 1 uses (step j - 1, their last user, has finished)
    if (bid == 0) {
        if (threadIdx.x == 0) {
            alpha[j] = __ldcg(h0 + j) + __ldcg(h1 + j);
            beta[j] = b;
        }
        for (int c = threadIdx.x; c < hstride; c += blockDim.x) other[c] = 0.0;
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) lanczos_step_kernel(float *V, int64_t ldv, int j, float *z, double *hbuf,
                                                          int hstride, double *alpha, double *beta, int m_max, int qt,
                                                          unsigned *bar, int *err, int phase) {
    lanczos_step_body<NT>(V, ldv, j, z, hbuf, hstride, alpha, beta, m_max, qt, bar, err, phase, (int)blockIdx.x,
                          (int)gridDim.x);
}

// one pass (phase 0..2) of the step for many problems: map[block] = {problem, its block, its
// block count}; problem p at its own step jv[p]. In the last pass, the last of a problem's
// blocks to finish (counted in arrive[p], reset to 0 by it) moves jv[p] to the next step:
// every block of the problem has read jv[p] by then.
__global__ void __launch_bounds__(kStepThreadsPhased) lanczos_step_batch_kernel(const DmLanczosProblem *__restrict__ P,
                                                                                const int4 *__restrict__ map,
                                                                                int *jv, unsigned *arrive,
                                                                                int phase) {
    const int4 pb = map[blockIdx.x];
    const DmLanczosProblem &p = P[pb.x];
    __shared__ int sj;
    if (threadIdx.x == 0) sj = jv[pb.x];
    __syncthreads();
    const int j = sj;
    lanczos_step_body<kStepThreadsPhased>(p.V, p.ldv, j, p.z, p.h, p.hstride, p.alpha, p.beta, p.m_max, p.qt,
                                          nullptr, nullptr, phase, pb.y, pb.z);
    if (phase == 2 && threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(arrive + pb.x, 1u) == (unsigned)pb.z - 1u) {
            arrive[pb.x] = 0u;
            jv[pb.x] = j + 1;
        }
    }
}

size_t step_smem_bytes(int m_max, int qt, int warps) {
    const int nchmax = (m_max + 1 + 7) >> 3;
    return sizeof(float4) * ((size_t)warps * qt + qt) + sizeof(float) * 16 * (size_t)nchmax;
}

int step_tile_quads(int m_max, int warps, int qt_max) {
    // 256 quads (1024 rows) per tile while the shared arrays stay under ~100 KB (the
    // coefficient arrays grow with m_max)
    int qt = qt_max;
    while (qt > 32 && step_smem_bytes(m_max, qt, warps) > 100 * 1024) qt >>= 1;
    return qt;
}


// ---- Sturm count of T_m - x I by the division-free characteristic-polynomial
// recurrence p_i = (alpha_i - x) p_{i-1} - beta_{i-1}^2 p_{i-2} with exact power-of-two
// rescaling; returns the number of eigenvalues of T_m below x.
__device__ int sturm_count(const double *__restrict__ al, const double *__restrict__ b2, int m, double x) {
    double pm = 1.0, p = al[0] - x;
    int cnt = (p < 0.0) ? 1 : 0;
    bool prev_neg = p < 0.0;
    if (p == 0.0) { p = -1e-300; cnt = 1; prev_neg = true; }
    for (int i = 1; i < m; ++i) {
        double pn = fma(-b2[i - 1], pm, (al[i] - x) * p);
        if (pn == 0.0) pn = prev_neg ? 1e-300 : -1e-300;  // a zero takes the sign that counts a change
        const bool neg = pn < 0.0;
        cnt += (neg != prev_neg) ? 1 : 0;
        prev_neg = neg;
        // keep magnitudes in range: scale both terms by the same power of two, chosen
        // from the larger one so that neither overflows
        const int e = (int)((__double_as_longlong(fabs(pn) > fabs(p) ? pn : p) >> 52) & 0x7ff);
        if (e > 1023 + 500 || e < 1023 - 500) {
            const int sh = 1023 - e;
            pn = scalbn(pn, sh);
            p = scalbn(p, sh);
        }
        pm = p;
        p = pn;
    }
    return cnt;
}

// Sturm count in FP32 by the LDL^T recurrence d_i = (alpha_i - x) - beta_{i-1}^2 / d_{i-1}
// (number of negative d_i = eigenvalues below x); only used to narrow a bracket that FP64
// counts then confirm
__device__ int sturm_count_f32(const float *al, const float *b2, int m, float x) {
    float d = al[0] - x;
    int cnt = d < 0.f ? 1 : 0;
    for (int i = 1; i < m; ++i) {
        if (d == 0.f) d = -1e-30f;
        d = (al[i] - x) - b2[i - 1] / d;
        cnt += d < 0.f ? 1 : 0;
    }
    return cnt;
}

// p_m(x), p_{m-1}(x) and p_m'(x) of det(T_i - x I) by the three-term recurrence and its
// derivative, all four running terms rescaled together by powers of two (ratios are exact)
__device__ void charpoly(const double *__restrict__ al, const double *__restrict__ b2, int m, double x,
                         double *p_out, double *pm_out, double *dp_out) {
    double pm = 1.0, p = al[0] - x, dpm = 0.0, dp = -1.0;
    for (int i = 1; i < m; ++i) {
        const double t = al[i] - x;
        const double pn = fma(-b2[i - 1], pm, t * p);
        const double dpn = fma(-b2[i - 1], dpm, fma(t, dp, -p));
        pm = p;
        dpm = dp;
        p = pn;
        dp = dpn;
        const int e = (int)((__double_as_longlong(fabs(dp) > fabs(p) ? dp : p) >> 52) & 0x7ff);
        if (e > 1023 + 500 || e < 1023 - 500) {
            const int sh = 1023 - e;
            p = scalbn(p, sh);
            pm = scalbn(pm, sh);
            dp = scalbn(dp, sh);
            dpm = scalbn(dpm, sh);
        }
    }
    *p_out = p;
    *pm_out = pm;
    *dp_out = dp;
}

// One block of kRitzThreads per wanted eigenvalue (descending index i): multisection to full
// FP64 precision with one shift per thread (four warps: all four FP64 units of the SM, seven
// bits per round), then the residual bound beta_{m-1} |y_m| from
// |y_m|^2 = |p_{m-1}(theta) / p_m'(theta)|.
constexpr int kRitzThreads = 128;
__device__ __forceinline__ void ritz_body(const double *__restrict__ alpha, const double *__restrict__ beta, int m,
                                          double *__restrict__ theta, double *__restrict__ resid, int iv) {
    extern __shared__ double sd[];
    double *al = sd, *b2 = sd + m;
    float *al32 = reinterpret_cast<float *>(b2 + m), *b232 = al32 + m;
    __shared__ unsigned s_above[kRitzThreads / 32];
    __shared__ double s_lo, s_hi, s_x, s_y2;
    __shared__ int s_ok[2], s_newton;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < m; i += blockDim.x) {
        al[i] = alpha[i];
        b2[i] = (i < m - 1) ? beta[i] * beta[i] : 0.0;
        al32[i] = (float)al[i];
        b232[i] = (float)b2[i];
    }
    __syncthreads();
    // Gershgorin interval (warp 0)
    if (warp == 0) {
        double lo = 1e300, hi = -1e300;
        for (int i = lane; i < m; i += 32) {
            const double r = (i > 0 ? sqrt(b2[i - 1]) : 0.0) + (i < m - 1 ? sqrt(b2[i]) : 0.0);
            lo = fmin(lo, al[i] - r);
            hi = fmax(hi, al[i] + r);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = fmin(lo, __shfl_xor_sync(DM_FULL, lo, o));
            hi = fmax(hi, __shfl_xor_sync(DM_FULL, hi, o));
        }
        if (lane == 0) {
            const double span = fmax(hi - lo, 1e-300);
            s_lo = lo - 1e-3 * span;
            s_hi = hi + 1e-3 * span;
        }
    }
    __syncthreads();
    double lo = s_lo, hi = s_hi;
    const int target = m - 1 - iv;  // ascending index of the wanted eigenvalue
    constexpr double kDen = (double)(kRitzThreads + 1);
    // three coarse rounds with FP32 counts (the FP64 pipe is narrow on this part)
    float flo = (float)lo, fhi = (float)hi;
    for (int round = 0; round < 3; ++round) {
        const float x = flo + (fhi - flo) * (float)(tid + 1) / (float)kDen;
        const int c = sturm_count_f32(al32, b232, m, x);
        const unsigned above = __ballot_sync(DM_FULL, c > target);
        if (lane == 0) s_above[warp] = above;
        __syncthreads();
        int g = -1;
        for (int w = 0; w < kRitzThreads / 32 && g < 0; ++w)
            if (s_above[w]) g = 32 * w + __ffs(s_above[w]) - 1;
        __syncthreads();
        auto shift = [&](int t) { return flo + (fhi - flo) * (float)(t + 1) / (float)kDen; };
        if (g < 0) flo = shift(kRitzThreads - 1);
        else {
            const float xh = shift(g);
            if (g > 0) flo = shift(g - 1);
            fhi = xh;
        }
    }
    // Newton on p_m(x) = det(T - x I) from the middle of the FP32 bracket, kept inside it
    // (quadratic convergence for an eigenvalue alone in the bracket), stopped after a step
    // below 1e-9 |x| (the error left, about step^2 / gap, is then far below the tolerance
    // checked next unless the gap is tiny). The iterate is taken when two FP64 Sturm counts
    // place the wanted eigenvalue within 1e-13 ||T|| of it; the residual bound uses the
    // last Newton evaluation. Otherwise two FP64 counts check the FP32 bracket and FP64
    // multisection rounds narrow it (from the Gershgorin interval if the check fails).
    if (tid == 0) {
        s_newton = 0;
        const double blo = (double)flo, bhi = (double)fhi;
        double x = 0.5 * (blo + bhi);
        for (int it = 0; it < 12 && blo < bhi; ++it) {
            double p, pm, dp;
            charpoly(al, b2, m, x, &p, &pm, &dp);
            if (dp == 0.0) break;
            const double xn = x - p / dp;
            if (!(xn >= blo && xn <= bhi)) break;
            const double stp = fabs(xn - x);
            x = xn;
            if (stp <= 1e-9 * fabs(x)) {
                s_x = x;
                s_y2 = fabs(pm / dp);
                s_newton = 1;
                break;
            }
        }
    }
    __syncthreads();
    bool done = false;
    if (s_newton) {
        const double x = s_x, tv = 1e-13 * fmax(fabs(s_lo), fabs(s_hi));
        if (tid < 2) {
            const int c = sturm_count(al, b2, m, tid == 0 ? x - tv : x + tv);
            s_ok[tid] = tid == 0 ? (c <= target) : (c > target);
        }
        __syncthreads();
        done = s_ok[0] && s_ok[1];  // uniform
        __syncthreads();            // every thread has read s_ok before it is reused
    }
    if (!done) {
        if (tid < 2) {
            const double x = tid == 0 ? (double)flo : (double)fhi;
            const int c = sturm_count(al, b2, m, x);
            s_ok[tid] = tid == 0 ? (c <= target) : (c > target);
        }
        __syncthreads();
        if (s_ok[0] && s_ok[1] && (double)flo < (double)fhi) {
            lo = (double)flo;
            hi = (double)fhi;
        }
        for (int round = 0; round < 16; ++round) {
            if (hi - lo <= 4e-16 * fmax(fabs(lo), fabs(hi))) break;  // uniform: every thread holds the same lo, hi
            const double x = lo + (hi - lo) * (double)(tid + 1) / kDen;
            const int c = sturm_count(al, b2, m, x);
            const unsigned above = __ballot_sync(DM_FULL, c > target);  // shifts above the eigenvalue
            if (lane == 0) s_above[warp] = above;
            __syncthreads();
            int g = -1;  // first shift above
            for (int w = 0; w < kRitzThreads / 32 && g < 0; ++w)
                if (s_above[w]) g = 32 * w + __ffs(s_above[w]) - 1;
            __syncthreads();
            // every thread re-forms the bracketing shifts with the same arithmetic
            auto shift = [&](int t) { return lo + (hi - lo) * (double)(t + 1) / kDen; };
            if (g < 0) lo = shift(kRitzThreads - 1);  // all shifts below: eigenvalue in (x_last, hi]
            else {
                const double xh = shift(g);
                if (g > 0) lo = shift(g - 1);
                hi = xh;
            }
        }
    }
    if (tid == 0) {
        const double th = done ? s_x : 0.5 * (lo + hi);
        double y2 = s_y2;
        if (!done) {
            double p, pm, dp;  // p_m, p_{m-1}, p_m' at th
            charpoly(al, b2, m, th, &p, &pm, &dp);
            y2 = (dp != 0.0) ? fabs(pm / dp) : 1.0;
        }
        theta[iv] = th;
        resid[iv] = beta[m - 1] * sqrt(fmin(y2, 1.0));
    }
}

__global__ void __launch_bounds__(kRitzThreads) ritz_kernel(const double *__restrict__ alpha,
                                                            const double *__restrict__ beta, int m,
                                                            double *__restrict__ theta, double *__restrict__ resid,
                                                            double *__restrict__ work) {
    (void)work;
    ritz_body(alpha, beta, m, theta, resid, (int)blockIdx.x);
}

// Ritz values and residual bounds of many problems at the same step (grid k x problems,
// blockIdx.y indexes `act`); also copied, per problem slot, to the contiguous theta_out /
// resid_out (k per slot) for one host read
__global__ void __launch_bounds__(kRitzThreads) ritz_batch_kernel(const DmLanczosProblem *__restrict__ P,
                                                                  const int *__restrict__ act,
                                                                  const int *__restrict__ jv, int kstride,
                                                                  double *__restrict__ theta_out,
                                                                  double *__restrict__ resid_out,
                                                                  double *__restrict__ beta_out) {
    const int slot = blockIdx.y;
    const int pi = act[slot];
    const DmLanczosProblem &p = P[pi];
    const int m = jv[pi];  // steps completed
    if ((int)blockIdx.x >= p.k || m < 1) return;  // uniform per block
    ritz_body(p.alpha, p.beta, m, p.theta, p.resid, (int)blockIdx.x);
    __syncthreads();
    if (threadIdx.x == 0) {
        theta_out[(size_t)slot * kstride + blockIdx.x] = p.theta[blockIdx.x];
        resid_out[(size_t)slot * kstride + blockIdx.x] = p.resid[blockIdx.x];
        if (blockIdx.x == 0) beta_out[slot] = p.beta[m - 1];
    }
}

// Eigenvector of T_m for theta (one warp per vector, serial in lane 0): inverse
// iteration with an LU factorisation with partial pivoting of T - theta I (three
// solves), normalised; written as column i of Y (ld = ldy). The factors and the iterate
// live in shared memory when they fit (44 m bytes), else in the global workspace (6 m
// doubles per vector). Either way the time is the serial chain of dependent FP64
// operations (about 67 us at m = 32), not the memory accesses.
// The workspace is read and written through several pointers carved out of one
// buffer, so no parameter here is declared __restrict__: with it the optimised
// build reorders those accesses and returns wrong vectors.
constexpr int kTvecSmemMaxM = 1024;  // 44 KB of shared memory
template <bool kShared>
__device__ __forceinline__ void tvec_body(const double *alpha, const double *beta, int m, const double *theta,
                                          double *Y, int ldy, double *work, uint64_t key, int iv) {
    extern __shared__ double tsm[];
    double *dl = kShared ? tsm : work + (size_t)iv * 6 * m;  // sub (L multipliers)
    double *dd = dl + m, *du = dd + m, *du2 = du + m, *y = du2 + m;
    int *ip = reinterpret_cast<int *>(y + m);
    const double th = theta[iv];
    double tnorm = 0.0;
    for (int i = 0; i < m; ++i) tnorm = fmax(tnorm, fabs(alpha[i]) + (i > 0 ? fabs(beta[i - 1]) : 0.0) + (i < m - 1 ? fabs(beta[i]) : 0.0));
    const double pivmin = 1e-300 + 2.2e-16 * tnorm;
    // factor T - th I = P L U (LAPACK dgttrf-style elimination)
    for (int i = 0; i < m; ++i) {
        dd[i] = alpha[i] - th;
        if (i < m - 1) { dl[i] = beta[i]; du[i] = beta[i]; }
        du2[i] = 0.0;
    }
    for (int i = 0; i < m - 1; ++i) {
        if (fabs(dd[i]) >= fabs(dl[i])) {
            ip[i] = 0;
            if (fabs(dd[i]) < pivmin) dd[i] = (dd[i] < 0 ? -pivmin : pivmin);
            const double f = dl[i] / dd[i];
            dl[i] = f;
            dd[i + 1] -= f * du[i];
        } else {
            ip[i] = 1;
            const double f = dd[i] / dl[i];
            dd[i] = dl[i];
            dl[i] = f;
            const double t = du[i];
            du[i] = dd[i + 1];
            dd[i + 1] = t - f * dd[i + 1];
            if (i < m - 2) {
                du2[i] = du[i + 1];
                du[i + 1] = -f * du[i + 1];
            }
        }
    }
    if (fabs(dd[m - 1]) < pivmin) dd[m - 1] = (dd[m - 1] < 0 ? -pivmin : pivmin);
    // the pivots are used only as divisors from here on: invert them once (FP64 division is
    // a long sequence on this part) instead of in each of the three solves
    for (int i = 0; i < m; ++i) dd[i] = 1.0 / dd[i];
    for (int i = 0; i < m; ++i) y[i] = 2.0 * dm_unit(dm_rng(key, (uint64_t)(iv * 1024 + i))) - 1.0;
    for (int it = 0; it < 3; ++it) {
        // solve L: apply row interchanges and multipliers
        for (int i = 0; i < m - 1; ++i) {
            if (ip[i] == 0) y[i + 1] -= dl[i] * y[i];
            else {
                const double t = y[i];
                y[i] = y[i + 1];
                y[i + 1] = t - dl[i] * y[i];
            }
        }
        // solve U (upper, bandwidth 2)
        y[m - 1] *= dd[m - 1];
        if (m > 1) y[m - 2] = (y[m - 2] - du[m - 2] * y[m - 1]) * dd[m - 2];
        for (int i = m - 3; i >= 0; --i) y[i] = (y[i] - du[i] * y[i + 1] - du2[i] * y[i + 2]) * dd[i];
        double nn = 0.0;
        for (int i = 0; i < m; ++i) nn += y[i] * y[i];
        const double inv = 1.0 / sqrt(nn);
        for (int i = 0; i < m; ++i) y[i] *= inv;
    }
    for (int i = 0; i < m; ++i) Y[(size_t)iv * ldy + i] = y[i];
}

template <bool kShared>
__global__ void __launch_bounds__(32) tvec_kernel(const double *alpha, const double *beta,
                                                  int m, const double *theta, double *Y,
                                                  int ldy, double *work, uint64_t key) {
    if (threadIdx.x != 0) return;
    tvec_body<kShared>(alpha, beta, m, theta, Y, ldy, work, key, (int)blockIdx.x);
}

// Gram-Schmidt of Y's columns within clusters of (numerically) equal Ritz values,
// then an FP32 copy for the Ritz-vector product.
__device__ __forceinline__ void tvec_orth_body(int m, int k, const double *theta, double *Y, int ldy, float *Yf) {
    __shared__ double red[32];
    __shared__ double th[kKMax];  // Ritz values staged once
    __shared__ unsigned char clus[kKMax * kKMax];  // clus[i][j]: pair (i, j) is in one cluster
    for (int i = threadIdx.x; i < k; i += blockDim.x) th[i] = theta[i];
    __syncthreads();
    double tmax = 0.0;
    for (int i = 0; i < k; ++i) tmax = fmax(tmax, fabs(th[i]));
    // every pair tested once, in parallel (a serial scan of the pairs waits out the FP64
    // latency of each test in turn)
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        const int i = e / k, j = e - i * k;
        clus[i * kKMax + j] = (j < i && !(fabs(th[i] - th[j]) > 1e-10 * tmax)) ? 1 : 0;
    }
    __syncthreads();
    for (int i = 1; i < k; ++i) {
        for (int j = 0; j < i; ++j) {
            if (!clus[i * kKMax + j]) continue;
            double part = 0.0;
            for (int t = threadIdx.x; t < m; t += blockDim.x) part += Y[(size_t)i * ldy + t] * Y[(size_t)j * ldy + t];
            part = dm_warp_sum_d(part);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
            __syncthreads();
            double dot = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) dot += red[w];
            __syncthreads();
            for (int t = threadIdx.x; t < m; t += blockDim.x) Y[(size_t)i * ldy + t] -= dot * Y[(size_t)j * ldy + t];
            __syncthreads();
            part = 0.0;
            for (int t = threadIdx.x; t < m; t += blockDim.x) part += Y[(size_t)i * ldy + t] * Y[(size_t)i * ldy + t];
            part = dm_warp_sum_d(part);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
            __syncthreads();
            double nn = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) nn += red[w];
            __syncthreads();
            const double inv = 1.0 / sqrt(nn);
            for (int t = threadIdx.x; t < m; t += blockDim.x) Y[(size_t)i * ldy + t] *= inv;
            __syncthreads();
        }
    }
    for (int e = threadIdx.x; e < m * k; e += blockDim.x) {
        const int i = e / m, t = e % m;
        Yf[(size_t)t * k + i] = (float)Y[(size_t)i * ldy + t];
    }
}

__global__ void tvec_orth_kernel(int m, int k, const double *theta, double *Y, int ldy, float *Yf) {
    tvec_orth_body(m, k, theta, Y, ldy, Yf);
}

// Phi~[pos, i] = sum_t V[t][pos] Y[t][i] (position order), plus per-column |.|^2 (FP64)
__device__ __forceinline__ void ritzvec_body(const float *__restrict__ V, int64_t ldv, int m, int k,
                                             const float *__restrict__ Yf, int64_t N, float *__restrict__ Phi,
                                             double *__restrict__ colsum, int bx) {
    extern __shared__ float sY[];  // m x k
    __shared__ float csum[kKMax][8];  // per-warp sums of squares
    for (int e = threadIdx.x; e < m * k; e += blockDim.x) sY[e] = Yf[e];
    __syncthreads();
    const int64_t pos = bx * (int64_t)blockDim.x + threadIdx.x;
    float acc[kKMax];
#pragma unroll
    for (int i = 0; i < kKMax; ++i) acc[i] = 0.f;
    if (pos < N) {
        // basis entries eight at a time, all loads issued before the products
        for (int t0 = 0; t0 < m; t0 += 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = t0 + u < m ? __ldcs(V + (size_t)(t0 + u) * ldv + pos) : 0.f;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (t0 + u >= m) break;
#pragma unroll
                for (int i = 0; i < kKMax; ++i)
                    if (i < k) acc[i] = fmaf(v[u], sY[(t0 + u) * k + i], acc[i]);
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < kKMax; ++i) {
        if (i < k) {
            if (pos < N) Phi[(size_t)i * N + pos] = acc[i];
            const float ss = dm_warp_sum(acc[i] * acc[i]);
            if (lane == 0) csum[i][warp] = ss;
        }
    }
    __syncthreads();
    // one FP64 atomic per column and block (the per-warp form queued thousands on each address)
    if (threadIdx.x < k) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += (double)csum[threadIdx.x][w];
        atomicAdd(colsum + threadIdx.x, t);
    }
}

__global__ void __launch_bounds__(256) ritzvec_kernel(const float *__restrict__ V, int64_t ldv, int m, int k,
                                                      const float *__restrict__ Yf, int64_t N,
                                                      float *__restrict__ Phi, double *__restrict__ colsum) {
    ritzvec_body(V, ldv, m, k, Yf, N, Phi, colsum, (int)blockIdx.x);
}

// normalise each column and find its largest-magnitude entry (ties: lowest original index)
__device__ __forceinline__ void colmax_body(const float *__restrict__ Phi, const int32_t *__restrict__ perm,
                                            int64_t N, unsigned long long *__restrict__ best, int bx, int i) {
    __shared__ unsigned long long wk[8];
    const int64_t pos = bx * (int64_t)blockDim.x + threadIdx.x;
    unsigned long long key = 0ull;
    if (pos < N) {
        const float a = fabsf(Phi[(size_t)i * N + pos]);
        key = ((unsigned long long)__float_as_uint(a) << 32) | (unsigned long long)(0xffffffffu - (unsigned)perm[pos]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(DM_FULL, key, o);
        key = other > key ? other : key;
    }
    if ((threadIdx.x & 31) == 0) wk[threadIdx.x >> 5] = key;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = wk[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = wk[w] > b ? wk[w] : b;
        atomicMax(best + i, b);  // one atomic per block and column
    }
}

__global__ void __launch_bounds__(256) colmax_kernel(const float *__restrict__ Phi, const int32_t *__restrict__ perm,
                                                     int64_t N, int k, const double *__restrict__ colsum,
                                                     unsigned long long *__restrict__ best) {
    colmax_body(Phi, perm, N, best, (int)blockIdx.x, (int)blockIdx.y);
}

// sign of each column's largest-magnitude entry: the thread holding that original index reports it
__device__ __forceinline__ void sign_pick_body(const float *__restrict__ Phi, const int32_t *__restrict__ perm,
                                               int64_t N, const unsigned long long *__restrict__ best,
                                               int *__restrict__ neg, int bx, int i) {
    const int64_t pos = bx * (int64_t)blockDim.x + threadIdx.x;
    if (pos >= N) return;
    const int arg = (int)(0xffffffffu - (unsigned)(best[i] & 0xffffffffull));
    if (perm[pos] == arg) neg[i] = Phi[(size_t)i * N + pos] < 0.f ? 1 : 0;
}

__global__ void sign_pick_kernel(const float *__restrict__ Phi, const int32_t *__restrict__ perm, int64_t N,
                                 const unsigned long long *__restrict__ best, int *__restrict__ neg) {
    sign_pick_body(Phi, perm, N, best, neg, (int)blockIdx.x, (int)blockIdx.y);
}

// unit norm, largest-magnitude entry positive, scattered to the original order
__device__ __forceinline__ void finalize_vec_body(const float *__restrict__ Phi, const int32_t *__restrict__ perm,
                                                  int64_t N, const double *__restrict__ colsum,
                                                  const int *__restrict__ neg, float *__restrict__ out, int bx,
                                                  int i) {
    __shared__ double s_sc;
    // the column's scale once per block (FP64 square root and division are long sequences here)
    if (threadIdx.x == 0) s_sc = (neg[i] ? -1.0 : 1.0) / sqrt(colsum[i]);
    __syncthreads();
    const int64_t pos = bx * (int64_t)blockDim.x + threadIdx.x;
    if (pos >= N) return;
    out[(size_t)i * N + perm[pos]] = (float)((double)Phi[(size_t)i * N + pos] * s_sc);
}

__global__ void finalize_vec_kernel(const float *__restrict__ Phi, const int32_t *__restrict__ perm, int64_t N,
                                    const double *__restrict__ colsum, const int *__restrict__ neg,
                                    float *__restrict__ out) {
    finalize_vec_body(Phi, perm, N, colsum, neg, out, (int)blockIdx.x, (int)blockIdx.y);
}

// ---- the same steps for many finished problems at once: F[f] describes problem f; the
// vector launches run over map[block] = {f, its block of 256 positions}, blockIdx.y the column
template <bool kShared>
__global__ void __launch_bounds__(32) tvec_batch_kernel(const DmFinish *__restrict__ F, uint64_t key) {
    const DmFinish &f = F[blockIdx.y];
    if (threadIdx.x != 0 || (int)blockIdx.x >= f.k) return;
    tvec_body<kShared>(f.alpha, f.beta, f.m, f.theta, f.Y, f.ldy, f.twork, key, (int)blockIdx.x);
}

__global__ void tvec_orth_batch_kernel(const DmFinish *__restrict__ F) {
    const DmFinish &f = F[blockIdx.x];
    tvec_orth_body(f.m, f.k, f.theta, f.Y, f.ldy, f.Yf);
    // the column sums and arg-max keys start from zero in the launches that follow
    for (int i = threadIdx.x; i < f.k; i += blockDim.x) {
        f.colsum[i] = 0.0;
        f.best[i] = 0ull;
    }
}

__global__ void __launch_bounds__(256) ritzvec_batch_kernel(const DmFinish *__restrict__ F,
                                                            const int2 *__restrict__ map) {
    const int2 fb = map[blockIdx.x];
    const DmFinish &f = F[fb.x];
    ritzvec_body(f.V, f.ldv, f.m, f.k, f.Yf, f.N, f.phi, f.colsum, fb.y);
}

__global__ void __launch_bounds__(256) colmax_batch_kernel(const DmFinish *__restrict__ F,
                                                           const int2 *__restrict__ map) {
    const int2 fb = map[blockIdx.x];
    const DmFinish &f = F[fb.x];
    if ((int)blockIdx.y >= f.k) return;
    colmax_body(f.phi, f.perm, f.N, f.best, fb.y, (int)blockIdx.y);
}

__global__ void sign_pick_batch_kernel(const DmFinish *__restrict__ F, const int2 *__restrict__ map) {
    const int2 fb = map[blockIdx.x];
    const DmFinish &f = F[fb.x];
    if ((int)blockIdx.y >= f.k) return;
    sign_pick_body(f.phi, f.perm, f.N, f.best, f.neg, fb.y, (int)blockIdx.y);
}

__global__ void finalize_vec_batch_kernel(const DmFinish *__restrict__ F, const int2 *__restrict__ map) {
    const int2 fb = map[blockIdx.x];
    const DmFinish &f = F[fb.x];
    if ((int)blockIdx.y >= f.k) return;
    finalize_vec_body(f.phi, f.perm, f.N, f.colsum, f.neg, f.evecs, fb.y, (int)blockIdx.y);
}

__global__ void coords_kernel(const float *__restrict__ evecs, const double *__restrict__ theta,
                              const double *__restrict__ dg, int64_t N, int t, float *__restrict__ psi) {
    const int i = blockIdx.y;
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= N) return;
    const double lt = pow(theta[i], (double)t);
    psi[(size_t)i * N + r] = (float)(lt * (double)evecs[(size_t)i * N + r] / sqrt(dg[r]));
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int dm_lanczos_kmax() { return kKMax; }

// ---- start vectors of many problems: zero their accumulators, draw, normalise (three launches)
__global__ void start_zero_batch_kernel(const DmStart *__restrict__ S) {
    const DmStart &s = S[blockIdx.x];
    for (int i = threadIdx.x; i < s.hlen; i += blockDim.x) s.h[i] = 0.0;
    if (threadIdx.x == 0) {
        *s.nrm2 = 0.0;
        *s.jv = 0;
    }
}

__global__ void start_vector_batch_kernel(const DmStart *__restrict__ S, const int2 *__restrict__ map) {
    const int2 sb = map[blockIdx.x];
    const DmStart &s = S[sb.x];
    const int64_t pos = sb.y * (int64_t)blockDim.x + threadIdx.x;
    float v = 0.f;
    if (pos < s.N) {
        v = (float)(2.0 * dm_unit(dm_rng(s.key, (uint64_t)s.perm[pos])) - 1.0);
        s.z[pos] = v;
    }
    const float ss = dm_warp_sum(v * v);
    if ((threadIdx.x & 31) == 0) atomicAdd(s.nrm2, (double)ss);
}

__global__ void normalize_batch_kernel(const DmStart *__restrict__ S, const int2 *__restrict__ map) {
    const int2 sb = map[blockIdx.x];
    const DmStart &s = S[sb.x];
    const int64_t i = sb.y * (int64_t)blockDim.x + threadIdx.x;
    if (i < s.N) s.V[i] = (float)((double)s.z[i] / sqrt(*s.nrm2));
}

uint64_t dm_start_key(uint64_t seed) { return dm_stream_key(seed, DM_TAG_V0, 0); }

cudaError_t dm_lanczos_start_batch(const DmStart *S, int ns, const int2 *map, int nmap, cudaStream_t st) {
    start_zero_batch_kernel<<<ns, 256, 0, st>>>(S);
    start_vector_batch_kernel<<<nmap, 256, 0, st>>>(S, map);
    normalize_batch_kernel<<<nmap, 256, 0, st>>>(S, map);
    dm_count_launches(3);
    return cudaGetLastError();
}

cudaError_t dm_lanczos_start(DmLanczos &Lz, const int32_t *perm, uint64_t seed, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(Lz.nrm2, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
    start_vector_kernel<<<nblk(Lz.N, 256), 256, 0, st>>>(perm, Lz.N, dm_stream_key(seed, DM_TAG_V0, 0), Lz.z, Lz.nrm2);
    dm_count_launches(1);
    normalize_kernel<<<nblk(Lz.N, 256), 256, 0, st>>>(Lz.z, Lz.N, Lz.nrm2, Lz.V);
    dm_count_launches(1);
    return cudaGetLastError();
}

namespace {
std::mutex g_coop_mu;
std::map<std::pair<int, void *>, cudaEvent_t> g_coop_events;  // per (device, stream); kept for the process
cudaEvent_t g_coop_last = nullptr;
}  // namespace

// After Lz.z = A v_j: two Gram-Schmidt passes against V[:, 0..j], alpha_j, beta_j and
// V[:, j+1], as one cooperative launch (grid = co-resident blocks on every SM).
cudaError_t dm_lanczos_orth(DmLanczos &Lz, int j, bool phased, cudaStream_t st) {
    const int hstride = 2 * (Lz.m_max + 1) + 2;
    cudaError_t e;
    if (j == 0) {
        if ((e = cudaMemsetAsync(Lz.h, 0, sizeof(double) * 2 * (size_t)hstride, st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(Lz.bar, 0, sizeof(unsigned), st)) != cudaSuccess) return e;
    }
    // phased (shared device): 256-thread blocks, two per SM, 512-row tiles; cooperative:
    // 512-thread blocks, one per SM, 1024-row tiles
    const int nt = phased ? kStepThreadsPhased : kStepThreadsCoop;
    const void *kern = phased ? (const void *)lanczos_step_kernel<kStepThreadsPhased>
                              : (const void *)lanczos_step_kernel<kStepThreadsCoop>;
    const int qt = step_tile_quads(Lz.m_max, nt / 32, phased ? 128 : 256);
    const size_t shm = step_smem_bytes(Lz.m_max, qt, nt / 32);
    if ((e = dm_allow_smem(kern, shm)) != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    int grid = 0;
    {
        // co-resident grid for this block size and shared-memory size
        static std::mutex mu;
        static std::map<std::pair<int, size_t>, int> grids;
        std::lock_guard<std::mutex> lk(mu);
        int &g = grids[std::make_pair(dev * 2 + (phased ? 1 : 0), shm)];
        if (g == 0) {
            int sms = 0, per_sm = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, shm);
            if (e != cudaSuccess) return e;
            if (per_sm < 1) return cudaErrorLaunchOutOfResources;
            const int want = phased ? 2 : 1;
            g = sms * (per_sm < want ? per_sm : want);
        }
        grid = g;
    }
    int jj = j, mm = Lz.m_max, hs = hstride, q = qt;
    int64_t ldv = Lz.ldv;
    if (phased) {
        for (int ph = 0; ph < 3; ++ph) {
            lanczos_step_kernel<kStepThreadsPhased><<<grid, kStepThreadsPhased, shm, st>>>(
                Lz.V, ldv, jj, Lz.z, Lz.h, hs, Lz.alpha, Lz.beta, mm, q, Lz.bar, Lz.err, ph);
            dm_count_launches(1);
        }
        return cudaGetLastError();
    }
    int phase_all = -1;
    void *args[] = {&Lz.V, &ldv, &jj, &Lz.z, &Lz.h, &hs, &Lz.alpha, &Lz.beta, &mm, &q, &Lz.bar, &Lz.err, &phase_all};
    // Each step kernel fills every SM; two of them from different streams (concurrent
    // solves) could each hold part of the device while waiting at a grid barrier for
    // blocks that cannot become resident. So all step launches of the process form one
    // chain: a launch waits for the previous one, whichever stream it was on.
    std::lock_guard<std::mutex> lk(g_coop_mu);
    cudaEvent_t &mine = g_coop_events[std::make_pair(dev, (void *)st)];
    if (!mine) {
        e = cudaEventCreateWithFlags(&mine, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            mine = nullptr;
            return e;
        }
    }
    if (g_coop_last && g_coop_last != mine) {
        e = cudaStreamWaitEvent(st, g_coop_last, 0);
        if (e != cudaSuccess) return e;
    }
    e = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(kStepThreadsCoop), args, shm, st);
    dm_count_launches(1);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(mine, st);
    if (e == cudaSuccess) g_coop_last = mine;
    return e;
}

cudaError_t dm_lanczos_ritz(DmLanczos &Lz, int m, int k, double conv_tol, cudaStream_t st) {
    (void)conv_tol;
    ritz_kernel<<<k, kRitzThreads, (sizeof(double) + sizeof(float)) * 2 * (size_t)m, st>>>(Lz.alpha, Lz.beta, m,
                                                                                            Lz.theta, Lz.resid, nullptr);
    dm_count_launches(1);
    return cudaGetLastError();
}

cudaError_t dm_lanczos_tvecs(DmLanczos &Lz, int m, int k, cudaStream_t st) {
    const uint64_t key = dm_stream_key(0x5eedULL, DM_TAG_V0, 1);
    if (m <= kTvecSmemMaxM)
        tvec_kernel<true><<<k, 32, (sizeof(double) * 5 + sizeof(int)) * (size_t)m, st>>>(
            Lz.alpha, Lz.beta, m, Lz.theta, Lz.Y, Lz.m_max, Lz.twork, key);
    else
        tvec_kernel<false><<<k, 32, 0, st>>>(Lz.alpha, Lz.beta, m, Lz.theta, Lz.Y, Lz.m_max, Lz.twork, key);
    dm_count_launches(1);
    tvec_orth_kernel<<<1, 256, 0, st>>>(m, k, Lz.theta, Lz.Y, Lz.m_max, Lz.Yf);
    dm_count_launches(1);
    return cudaGetLastError();
}

cudaError_t dm_lanczos_vectors(DmLanczos &Lz, int m, int k, const int32_t *perm, float *evecs_orig,
                               cudaStream_t st) {
    cudaError_t e = dm_lanczos_tvecs(Lz, m, k, st);
    if (e != cudaSuccess) return e;
    return dm_lanczos_phi(Lz, m, k, perm, evecs_orig, st);
}

cudaError_t dm_lanczos_phi(DmLanczos &Lz, int m, int k, const int32_t *perm, float *evecs_orig, cudaStream_t st) {
    float *phi_work = Lz.phi;
    unsigned long long *best = Lz.best;
    cudaError_t e = cudaMemsetAsync(Lz.colsum, 0, sizeof(double) * k, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(best, 0, sizeof(unsigned long long) * k, st);
    if (e != cudaSuccess) return e;
    const size_t ysh = sizeof(float) * (size_t)m * k;
    e = dm_allow_smem((const void *)ritzvec_kernel, ysh);
    if (e != cudaSuccess) return e;
    ritzvec_kernel<<<nblk(Lz.N, 256), 256, ysh, st>>>(Lz.V, Lz.ldv, m, k, Lz.Yf, Lz.N, phi_work, Lz.colsum);
    dm_count_launches(1);
    const dim3 g2(nblk(Lz.N, 256), (unsigned)k);
    colmax_kernel<<<g2, 256, 0, st>>>(phi_work, perm, Lz.N, k, Lz.colsum, best);
    dm_count_launches(1);
    sign_pick_kernel<<<g2, 256, 0, st>>>(phi_work, perm, Lz.N, best, Lz.neg);
    dm_count_launches(1);
    finalize_vec_kernel<<<g2, 256, 0, st>>>(phi_work, perm, Lz.N, Lz.colsum, Lz.neg, evecs_orig);
    dm_count_launches(1);
    return cudaGetLastError();
}

int dm_finish_blocks(int64_t N) { return nblk(N, 256); }

cudaError_t dm_lanczos_finish_batch(const DmFinish *F, int nf, const int2 *map, int nmap, int m_hi, int k_hi,
                                    cudaStream_t st) {
    const uint64_t key = dm_stream_key(0x5eedULL, DM_TAG_V0, 1);  // the single-problem path's draws
    cudaError_t e;
    if (m_hi <= kTvecSmemMaxM) {
        const size_t sh = (sizeof(double) * 5 + sizeof(int)) * (size_t)m_hi;
        if ((e = dm_allow_smem((const void *)tvec_batch_kernel<true>, sh)) != cudaSuccess) return e;
        tvec_batch_kernel<true><<<dim3((unsigned)k_hi, (unsigned)nf), 32, sh, st>>>(F, key);
    } else {
        tvec_batch_kernel<false><<<dim3((unsigned)k_hi, (unsigned)nf), 32, 0, st>>>(F, key);
    }
    dm_count_launches(1);
    tvec_orth_batch_kernel<<<nf, 256, 0, st>>>(F);
    dm_count_launches(1);
    const size_t ysh = sizeof(float) * (size_t)m_hi * k_hi;
    if ((e = dm_allow_smem((const void *)ritzvec_batch_kernel, ysh)) != cudaSuccess) return e;
    ritzvec_batch_kernel<<<nmap, 256, ysh, st>>>(F, map);
    dm_count_launches(1);
    const dim3 g2((unsigned)nmap, (unsigned)k_hi);
    colmax_batch_kernel<<<g2, 256, 0, st>>>(F, map);
    sign_pick_batch_kernel<<<g2, 256, 0, st>>>(F, map);
    finalize_vec_batch_kernel<<<g2, 256, 0, st>>>(F, map);
    dm_count_launches(3);
    return cudaGetLastError();
}

// Thick restart (Section 2.3's implicit restart with exact shifts, in its explicit form):
// the kr Ritz vectors V[:, 0:m] Y[:, 0:kr] (normalised) replace the first kr basis columns,
// the newest block V[:, src:src+b] moves to columns kr..kr+b-1, and the projected matrix
// becomes diag(theta_1..theta_kr); the next block step's projection fills the coupling
// column (B_j y_i, last block) itself.
__global__ void restart_basis_kernel(float *V, int64_t ldv, int64_t N, const float *__restrict__ Phi,
                                     const double *__restrict__ colsum, int kr, int src, int b) {
    const int c = blockIdx.y;
    const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c < kr) {
        if (pos < N) V[(size_t)c * ldv + pos] = Phi[(size_t)c * N + pos] * (float)(1.0 / sqrt(colsum[c]));
    } else if (pos < ldv) {
        V[(size_t)c * ldv + pos] = V[(size_t)(src + c - kr) * ldv + pos];
    }
}

__global__ void restart_T_kernel(double *T, int ldT, int n, const double *__restrict__ theta, int kr) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * ldT) return;
    const int c = (int)(e / ldT), r = (int)(e - (int64_t)c * ldT);
    T[e] = (r == c && r < kr) ? theta[r] : 0.0;
}

cudaError_t dm_lanczos_restart(DmLanczos &Lz, int m, int kr, int src, int b, double *T, int ldT, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(Lz.colsum, 0, sizeof(double) * kr, st);
    if (e != cudaSuccess) return e;
    const size_t ysh = sizeof(float) * (size_t)m * kr;
    if ((e = dm_allow_smem((const void *)ritzvec_kernel, ysh)) != cudaSuccess) return e;
    ritzvec_kernel<<<nblk(Lz.N, 256), 256, ysh, st>>>(Lz.V, Lz.ldv, m, kr, Lz.Yf, Lz.N, Lz.phi, Lz.colsum);
    dm_count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    restart_basis_kernel<<<dim3(nblk(Lz.ldv, 256), (unsigned)(kr + b)), 256, 0, st>>>(Lz.V, Lz.ldv, Lz.N, Lz.phi,
                                                                                     Lz.colsum, kr, src, b);
    dm_count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t tot = (int64_t)Lz.m_max * ldT;
    restart_T_kernel<<<nblk(tot, 256), 256, 0, st>>>(T, ldT, Lz.m_max, Lz.theta, kr);
    dm_count_launches(1);
    return cudaGetLastError();
}

cudaError_t dm_launch_coords(const float *evecs, const double *theta, const double *dg, int64_t N, int k, int t,
                             float *psi, cudaStream_t st) {
    coords_kernel<<<dim3(nblk(N, 256), (unsigned)k), 256, 0, st>>>(evecs, theta, dg, N, t, psi);
    dm_count_launches(1);
    return cudaGetLastError();
}

// Failure-detection self-test of the bounded grid barrier above: `blocks` blocks meet at a
// barrier whose target counts `missing` more arrivals than there are blocks. With missing
// = 0 every block passes (blocks <= 8, always co-resident); with missing > 0 nothing ever
// completes the count, every block gives up after `spin_limit` polls, raises *err and
// returns, and ctr[1] counts the blocks that passed.
__global__ void barrier_selftest_kernel(unsigned *ctr, unsigned target, int *err, long long spin_limit) {
    if (!grid_barrier(ctr, target, err, spin_limit)) return;
    if (threadIdx.x == 0) atomicAdd(ctr + 1, 1u);
}

cudaError_t dm_launch_barrier_selftest(unsigned *ctr, int *err, int blocks, int missing, long long spin_limit,
                                       cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    barrier_selftest_kernel<<<blocks, 128, 0, st>>>(ctr, (unsigned)(blocks + missing), err, spin_limit);
    dm_count_launches(1);
    return cudaGetLastError();
}

int dm_step_phased_threads() { return kStepThreadsPhased; }
int dm_step_tile_quads(int m_max) { return step_tile_quads(m_max, kStepThreadsPhased / 32, 128); }

size_t dm_step_batch_smem(int m_max) {
    return step_smem_bytes(m_max, dm_step_tile_quads(m_max), kStepThreadsPhased / 32);
}

cudaError_t dm_lanczos_step_batch(const DmLanczosProblem *P, const int4 *map, int nblocks, int *jv,
                                  unsigned *arrive, size_t shm, cudaStream_t st) {
    cudaError_t e = dm_allow_smem((const void *)lanczos_step_batch_kernel, shm);
    if (e != cudaSuccess) return e;
    for (int ph = 0; ph < 3; ++ph) {
        lanczos_step_batch_kernel<<<nblocks, kStepThreadsPhased, shm, st>>>(P, map, jv, arrive, ph);
        dm_count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t dm_lanczos_ritz_batch(const DmLanczosProblem *P, const int *act, int nact, const int *jv, int m_hi,
                                  int k_hi, double *theta_out, double *resid_out, double *beta_out, cudaStream_t st) {
    const size_t shm = (sizeof(double) + sizeof(float)) * 2 * (size_t)m_hi;
    cudaError_t e = dm_allow_smem((const void *)ritz_batch_kernel, shm);
    if (e != cudaSuccess) return e;
    ritz_batch_kernel<<<dim3((unsigned)k_hi, (unsigned)nact), kRitzThreads, shm, st>>>(P, act, jv, k_hi, theta_out,
                                                                                       resid_out, beta_out);
    dm_count_launches(1);
    return cudaGetLastError();
}

int dm_lanczos_hstride(int m_max) { return 2 * (m_max + 1) + 2; }
