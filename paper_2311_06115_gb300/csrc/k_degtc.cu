// k_degtc.cu -- degree passes for high-dimensional points on the tensor cores.
//
// A degree pass is out_i = sum_j W_ij w_j with W_ij = exp(-|x_i - x_j|^2 / eps) (Eq. W and
// Algorithm 1: similarity matrix and normalisations). For large d the work is the Gram matrix G = X X^T: with
// n_i = |x_i|^2, |x_i - x_j|^2 = n_i + n_j - 2 G_ij. Here G is a tcgen05 GEMM with FP32
// accumulation in TMEM (128 x 256 tiles), and the epilogue turns each accumulator row into
// 2^(2 k G_ij - a_i - a_j) w_j (a_i = k n_i, k = log2(e) sigma^2 / eps) summed over the
// tile's columns -- the N x N matrix never exists.
//
// Operands (prepared once per handle):
//   quantised data (every coordinate within 1e-4 / 255 of a multiple of 1/255, as FP32
//     copies of 8-bit pixel data): v = rint(255 x) minus the integer-rounded column mean,
//     integers in [-255, 255], exact in BF16: a BF16 GEMM (kind::f16), sigma = 1/255, K = d;
//   otherwise: centred u = x - mean split as hi = tf32_rn(u), lo = u - hi (exact), and
//     A = [hi | hi | lo], B = [hi | lo | hi] along K: a TF32 GEMM (kind::tf32) of
//     A B^T = hi hi^T + hi lo^T + lo hi^T, relative error about 2^-20 (the dropped lo lo^T
//     term and the TF32 reading of lo), sigma = 1, K = 3 d.
// n_i is the same product's diagonal, so the diagonal entries are exp(0) = 1 up to the
// FP32 accumulation order.
//
// One CTA per (128-row, 256-column) tile, in a grouped tile order (see the kernel); warp 0
// issues TMA loads into a 2-stage ring, warp 1 issues the MMAs, all four warps run the
// epilogue (thread = row). Two CTAs fit on an SM (shared memory, and 2 x 256 TMEM columns),
// so one's epilogue overlaps the other's MMAs. Waits are bounded; a timeout raises *err and
// the tile is skipped.
#include <cuda_bf16.h>

#include "dm_internal.cuh"
#include "dm_tc.cuh"

namespace {

using namespace dmtc;

constexpr int kDtThreads = 128;
constexpr int kDtStages = 2;
constexpr int kDtBM = 128;
constexpr int kDtBN = 256;
constexpr uint32_t kDtABytes = kDtBM * 128;   // 128 rows x 128 bytes (64 BF16 or 32 FP32)
constexpr uint32_t kDtBBytes = kDtBN * 128;   // 256 rows x 128 bytes
constexpr uint32_t kDtStage = kDtABytes + kDtBBytes;
constexpr int kDtGroup = 16;  // row tiles per group of the tile order

template <bool kTf32>
__global__ void __launch_bounds__(kDtThreads) degtc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                           const __grid_constant__ CUtensorMap tmB, int64_t N,
                                                           int kpad, float kappa, const float *__restrict__ an,
                                                           const float *__restrict__ w, double *__restrict__ out,
                                                           int *err) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = su32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *tiles = smem_raw + (base - raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(tiles + kDtStages * kDtStage);
    uint64_t *empty = full + kDtStages;
    uint64_t *done = empty + kDtStages;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    float *s_a = reinterpret_cast<float *>(tmem_slot + 4);  // kDtBN column terms a_j
    float *s_w = s_a + kDtBN;                               // kDtBN weights (0 past N)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // tiles in groups of kDtGroup row tiles: consecutive CTAs walk the column tiles of one
    // group, so the CTAs resident at a time share a few row tiles and a band of column tiles
    // in L2 (in launch order along whole rows, every row tile would stream all of X again)
    const int64_t ntm = (N + kDtBM - 1) / kDtBM, ntn = (N + kDtBN - 1) / kDtBN;
    const int64_t pid = blockIdx.x, per_group = (int64_t)kDtGroup * ntn;
    const int64_t first_m = (pid / per_group) * kDtGroup;
    const int64_t gsize = ntm - first_m < kDtGroup ? ntm - first_m : kDtGroup;
    const int64_t r = pid - (pid / per_group) * per_group;
    const int64_t i0 = (first_m + r % gsize) * kDtBM, j0 = (r / gsize) * kDtBN;
    constexpr int kElems = kTf32 ? 32 : 64;  // K elements per 128-byte row
    const int ksteps = kpad / kElems;

    for (int t = threadIdx.x; t < kDtBN; t += blockDim.x) {
        const int64_t j = j0 + t;
        s_a[t] = j < N ? an[j] : 0.f;
        s_w[t] = j < N ? (w ? w[j] : 1.f) : 0.f;
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kDtStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tmem_slot, kDtBN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        for (int k = 0; k < ksteps; ++k) {
            const int s = k % kDtStages;
            if (k >= kDtStages && !mbar_wait(&empty[s], (unsigned)((k / kDtStages) - 1) & 1u)) {
                atomicExch(err, 1);
                break;
            }
            uint8_t *sa = tiles + s * kDtStage, *sb = sa + kDtABytes;
            mbar_expect_tx(&full[s], kDtStage);
            tma_load_2d(sa, &tmA, kElems * k, (int)i0, &full[s]);
            tma_load_2d(sb, &tmB, kElems * k, (int)j0, &full[s]);
        }
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = kTf32 ? idesc_tf32(kDtBN) : idesc_bf16(kDtBN);
        bool ok = true;
        for (int k = 0; k < ksteps; ++k) {
            const int s = k % kDtStages;
            if (!mbar_wait(&full[s], (unsigned)(k / kDtStages) & 1u)) {
                atomicExch(err, 1);
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t sa = base + (uint32_t)s * kDtStage, sb = sa + kDtABytes;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint64_t da = desc_sw128(sa + 32u * kk), db = desc_sw128(sb + 32u * kk);
                const uint32_t acc = (k > 0 || kk > 0) ? 1u : 0u;
                if (kTf32) tc_mma_tf32(tmem, da, db, idesc, acc);
                else tc_mma_f16(tmem, da, db, idesc, acc);
            }
            tc_commit(&empty[s]);
        }
        if (ok) tc_commit(done);
    }
    __syncwarp();
    const bool ready = __all_sync(0xffffffffu, mbar_wait(done, 0u) ? 1 : 0) != 0;
    if (!ready && lane == 0) atomicExch(err, 1);
    tc_fence_after();
    if (ready) {
        const int64_t i = i0 + 32 * warp + lane;
        const float ai = i < N ? an[i] : 0.f;
        const float k2 = 2.f * kappa;
        float acc0 = 0.f, acc1 = 0.f;
#pragma unroll 1
        for (int cc = 0; cc < kDtBN; cc += 16) {
            uint32_t v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)cc, v);
#pragma unroll
            for (int t = 0; t < 16; t += 2) {
                const float g0 = __uint_as_float(v[t]), g1 = __uint_as_float(v[t + 1]);
                const float e0 = dm_ex2(fminf(fmaf(k2, g0, -(ai + s_a[cc + t])), 0.f));
                const float e1 = dm_ex2(fminf(fmaf(k2, g1, -(ai + s_a[cc + t + 1])), 0.f));
                acc0 = fmaf(e0, s_w[cc + t], acc0);
                acc1 = fmaf(e1, s_w[cc + t + 1], acc1);
            }
        }
        if (i < N) atomicAdd(out + i, (double)(acc0 + acc1));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kDtBN);
    }
}

// ---- operand preparation

// column means (FP64) and the quantisation check: q_bad counts columns with a coordinate
// whose 255 x is not within 1e-4 of an integer in [0, 255]
__global__ void degtc_stats_kernel(const float *__restrict__ X, int64_t N, int d, double *__restrict__ sums,
                                   unsigned *__restrict__ q_bad) {
    const int k = blockIdx.x;
    double s = 0.0;
    unsigned bad = 0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const float x = X[i * d + k];
        s += (double)x;
        const float v = x * 255.f;
        if (!(v >= -1e-4f && v <= 255.0001f && fabsf(v - rintf(v)) <= 1e-4f)) bad = 1;
    }
    s = dm_warp_sum_d(s);
    bad = __any_sync(0xffffffffu, bad != 0) ? 1u : 0u;
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(sums + k, s);
        if (bad) atomicAdd(q_bad, 1u);
    }
}

// A (and B) rows, zero padded to kpad (`sums` holds the column means by now). Quantised:
// A = [v] (BF16), v = rint(255 x) - rint(255 mean). Otherwise (FP32 storage): A = [hi | hi | lo], B = [hi | lo | hi] of the
// centred u = x - mean, hi = u rounded to TF32 (10 mantissa bits), lo = u - hi.
// nrm_i = the diagonal of A B^T in FP32 (the epilogue's a_i = kappa nrm_i).
__device__ __forceinline__ float tf32_rn(float u) {
    // round to nearest (ties away) at 10 mantissa bits: add half of the dropped range, truncate
    uint32_t b = __float_as_uint(u);
    b = (b + 0x1000u) & 0xFFFFE000u;
    return __uint_as_float(b);
}

__global__ void degtc_prep_kernel(const float *__restrict__ X, int64_t N, int d, const double *__restrict__ sums,
                                  int quant, int dpad, void *Av, void *Bv, float *__restrict__ nrm) {
    const int64_t i = blockIdx.x;
    float nn = 0.f;
    if (quant) {
        __nv_bfloat16 *ar = reinterpret_cast<__nv_bfloat16 *>(Av) + i * dpad;
        for (int k = threadIdx.x; k < dpad; k += blockDim.x) {
            float v = 0.f;
            if (k < d) v = rintf(X[i * d + k] * 255.f) - (float)rint(255.0 * sums[k]);
            ar[k] = __float2bfloat16_rn(v);
            nn = fmaf(v, v, nn);
        }
    } else {
        float *ar = reinterpret_cast<float *>(Av) + i * 3 * (int64_t)dpad;
        float *br = reinterpret_cast<float *>(Bv) + i * 3 * (int64_t)dpad;
        for (int k = threadIdx.x; k < dpad; k += blockDim.x) {
            float hi = 0.f, lo = 0.f;
            if (k < d) {
                const float u = (float)((double)X[i * d + k] - sums[k]);
                hi = tf32_rn(u);
                lo = u - hi;
            }
            ar[k] = hi;
            ar[dpad + k] = hi;
            ar[2 * dpad + k] = lo;
            br[k] = hi;
            br[dpad + k] = lo;
            br[2 * dpad + k] = hi;
            nn = fmaf(hi, hi, fmaf(2.f * hi, lo, nn));
        }
    }
    __shared__ float red[32];
    nn = dm_warp_sum(nn);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nn;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        nrm[i] = t;
    }
}

// column sums -> column means, once (d divisions instead of one per element)
__global__ void degtc_means_kernel(double *sums, int64_t N, int d) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < d) sums[k] = sums[k] / (double)N;
}

__global__ void degtc_scale_kernel(float *nrm, int64_t N, double kappa) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    nrm[i] = (float)((double)nrm[i] * kappa);
}

}  // namespace

size_t dm_degtc_work_bytes(int64_t N, int d) {
    const int64_t dpad = (d + 63) / 64 * 64;
    return 2 * (size_t)N * 3 * dpad * 4 + (((size_t)N * 4 + 255) & ~(size_t)255) + (size_t)d * 8 + 256;
}

bool dm_degtc_available() { return tc_encode_fn() != nullptr; }

cudaError_t dm_degtc_prepare(const float *X, int64_t N, int d, double eps, void *work, DmDegTc *S,
                             cudaStream_t st) {
    const int dpad = (d + 63) / 64 * 64;
    uint8_t *p = reinterpret_cast<uint8_t *>(work);
    S->N = N;
    S->d = d;
    S->dpad = dpad;
    S->A = p;
    S->B = p + (size_t)N * 3 * dpad * 4;
    S->an = reinterpret_cast<float *>(p + 2 * (size_t)N * 3 * dpad * 4);
    S->sums = reinterpret_cast<double *>(reinterpret_cast<uint8_t *>(S->an) + (((size_t)N * 4 + 255) & ~(size_t)255));
    S->q_bad = reinterpret_cast<unsigned *>(S->sums + d);
    cudaError_t e = cudaMemsetAsync(S->sums, 0, sizeof(double) * d + sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    degtc_stats_kernel<<<d, 256, 0, st>>>(X, N, d, S->sums, S->q_bad);
    dm_count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the quantisation flag decides the operand type: read it back (once per handle)
    unsigned bad = 0;
    if ((e = cudaMemcpyAsync(&bad, S->q_bad, sizeof(unsigned), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    S->quant = bad == 0;
    S->kpad = S->quant ? dpad : 3 * dpad;
    degtc_means_kernel<<<(unsigned)((d + 255) / 256), 256, 0, st>>>(S->sums, N, d);
    dm_count_launches(1);
    degtc_prep_kernel<<<(unsigned)N, 128, 0, st>>>(X, N, d, S->sums, S->quant ? 1 : 0, dpad, S->A, S->B, S->an);
    dm_count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const double log2e = 1.4426950408889634;
    const double kappa = log2e / eps * (S->quant ? 1.0 / (255.0 * 255.0) : 1.0);
    degtc_scale_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(S->an, N, kappa);
    dm_count_launches(1);
    S->kappa = (float)kappa;
    return cudaGetLastError();
}

template <bool kTf32>
cudaError_t degtc_launch(const DmDegTc &S, const float *w, double *out, int *err, cudaStream_t st) {
    CUtensorMap tmA, tmB;
    const CUtensorMapDataType dt = kTf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const size_t es = kTf32 ? 4 : 2;
    const uint32_t bc = kTf32 ? 32 : 64;
    const void *B = kTf32 ? S.B : S.A;
    if (!tc_make_map(&tmA, dt, es, S.A, (uint64_t)S.kpad, (uint64_t)S.N, (uint64_t)S.kpad, bc, kDtBM) ||
        !tc_make_map(&tmB, dt, es, B, (uint64_t)S.kpad, (uint64_t)S.N, (uint64_t)S.kpad, bc, kDtBN))
        return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * S.N, st);
    if (e != cudaSuccess) return e;
    const size_t smem = 1024 + (size_t)kDtStages * kDtStage + 256 + 2 * kDtBN * sizeof(float);
    if ((e = dm_allow_smem((const void *)degtc_kernel<kTf32>, smem)) != cudaSuccess) return e;
    const int64_t tiles = ((S.N + kDtBN - 1) / kDtBN) * ((S.N + kDtBM - 1) / kDtBM);
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    degtc_kernel<kTf32><<<(unsigned)tiles, kDtThreads, smem, st>>>(tmA, tmB, S.N, S.kpad, S.kappa, S.an, w, out, err);
    dm_count_launches(1);
    return cudaGetLastError();
}

// out_i = sum_j W_ij w_j (w == nullptr: all ones); out is zeroed here
cudaError_t dm_degtc_pass(const DmDegTc &S, const float *w, double *out, int *err, cudaStream_t st) {
    return S.quant ? degtc_launch<false>(S, w, out, err, st) : degtc_launch<true>(S, w, out, err, st);
}
