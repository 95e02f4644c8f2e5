// k_tc.cu -- the near field of the block H-matvec on the tensor cores (tcgen05, TF32).
//
// For a block of nb right-hand sides the near field is one small GEMM per leaf,
// C_a = K(I_a, I_a) X(I_a, :) (Eq. 2.18, the block-diagonal D). Here it runs as
// tcgen05.mma kind::tf32 (FP32 operands read as TF32, FP32 accumulation in tensor
// memory): one CTA per (leaf, 128-row tile of the leaf block, panel of NT columns).
//
//   warp 0, one lane   TMA producer: 128 x 32 FP32 tiles of K (a 128-byte-swizzled
//                      row per block row) and NT x 32 tiles of X^T, into a 4-stage ring
//   warp 1, one lane   MMA issuer: 4 MMAs (K = 8) per stage, accumulating in TMEM;
//                      tcgen05.commit frees the stage, the last commit signals the epilogue
//   warps 0-3          epilogue: tcgen05.ld of the 128 x NT accumulator (a row per thread)
//                      and coalesced stores into the padded leaf layout
//
// The tail tile of a leaf (fewer than 128 rows) is fetched as 8-row boxes so that only the
// leaf's own rows cross HBM; accumulator rows past the leaf are never stored. Columns past
// the block (ldk) and right-hand sides past nb are zero-filled by TMA.
//
// Split mode (three-term TF32, accuracy close to FP32): warps 2-3 split every staged tile
// into a TF32-exact high part (the low 13 mantissa bits cleared, written in place) and the
// low remainder (x - hi, exact in FP32, into a second buffer), then release the stage to the
// MMA issuer through a third mbarrier; the issuer accumulates hi*hi + hi*lo + lo*hi (the
// lo*lo term, ~2^-20 relative, is dropped). The split tiles halve the stages that fit.
//
// Every mbarrier wait is bounded (about a second of clock cycles); a wait that gives up
// raises *err, skips the stores and still frees the tensor memory, and the host reports
// DM_ETIMEOUT.
#include "dm_internal.cuh"
#include "dm_tc.cuh"

namespace {

using namespace dmtc;

constexpr int kTcThreads = 128;
constexpr uint32_t kTcABytes = 128 * 128;  // 128 rows x 32 FP32
constexpr int kSplitThreads = 64;          // warps 2-3 split the tiles in split mode

template <int NT, bool SPLIT>
__host__ __device__ constexpr int tc_stages() {
    return !SPLIT ? 4 : (NT >= 256 ? 2 : (NT >= 128 ? 3 : 4));
}
template <int NT, bool SPLIT>
__host__ __device__ constexpr uint32_t tc_stage_bytes() {
    return (kTcABytes + NT * 128) * (SPLIT ? 2u : 1u);
}

template <int NT, bool SPLIT>
__global__ void __launch_bounds__(kTcThreads) tc_near_kernel(const __grid_constant__ CUtensorMap tmA,
                                                             const __grid_constant__ CUtensorMap tmA8,
                                                             const __grid_constant__ CUtensorMap tmB,
                                                             const __grid_constant__ DmHmat H, int nb,
                                                             float *__restrict__ Yb, int64_t ldx, int mtiles,
                                                             int *err) {
    static_assert(NT >= 16 && NT <= 256 && (NT & (NT - 1)) == 0, "NT: power of two in [16, 256]");
    constexpr int kTcStages = tc_stages<NT, SPLIT>();
    constexpr uint32_t kBBytes = NT * 128;
    constexpr uint32_t kHiBytes = kTcABytes + kBBytes;  // A then B (high parts); low parts follow
    constexpr uint32_t kStageBytes = tc_stage_bytes<NT, SPLIT>();
    constexpr uint32_t kTmemCols = NT < 32 ? 32 : NT;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = su32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *tiles = smem_raw + (base - raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(tiles + kTcStages * kStageBytes);
    uint64_t *empty = full + kTcStages;
    uint64_t *conv = empty + kTcStages;  // split mode: the stage's tiles are split
    uint64_t *done = conv + kTcStages;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int a = blockIdx.x / mtiles, mt = blockIdx.x - a * mtiles;
    const int c0 = blockIdx.y * NT;
    int64_t st, sz;
    dm_node_range(H.N, (1 << H.L) - 1 + a, &st, &sz);
    const int m = (int)sz, r0 = mt * 128;
    if (r0 >= m) return;  // uniform: this leaf is one row shorter than the longest
    const int nr = min(128, m - r0);
    const int ksteps = (((m + 3) & ~3) + 31) / 32;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
            mbar_init(&conv[s], kSplitThreads);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer
        const int arow = a * H.leaf_max + r0;
        const int nbox8 = (nr + 7) / 8;
        const bool whole = nr == 128;
        const uint32_t abytes = whole ? kTcABytes : (uint32_t)nbox8 * 1024u;
        for (int k = 0; k < ksteps; ++k) {
            const int s = k % kTcStages;
            if (k >= kTcStages && !mbar_wait(&empty[s], (unsigned)((k / kTcStages) - 1) & 1u)) {
                atomicExch(err, 1);
                break;
            }
            uint8_t *sa = tiles + s * kStageBytes, *sb = sa + kTcABytes;
            mbar_expect_tx(&full[s], abytes + kBBytes);
            if (whole) tma_load_2d(sa, &tmA, 32 * k, arow, &full[s]);
            else
                for (int q = 0; q < nbox8; ++q) tma_load_2d(sa + 1024 * q, &tmA8, 32 * k, arow + 8 * q, &full[s]);
            tma_load_2d(sb, &tmB, a * H.ldk + 32 * k, c0, &full[s]);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_tf32(NT);
        bool ok = true;
        for (int k = 0; k < ksteps; ++k) {
            const int s = k % kTcStages;
            if (!mbar_wait(SPLIT ? &conv[s] : &full[s], (unsigned)(k / kTcStages) & 1u)) {
                atomicExch(err, 1);
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t sa = base + (uint32_t)s * kStageBytes, sb = sa + kTcABytes;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                tc_mma_tf32(tmem, desc_sw128(sa + 32u * kk), desc_sw128(sb + 32u * kk), idesc,
                            (k > 0 || kk > 0) ? 1u : 0u);
                if (SPLIT) {
                    const uint32_t la = sa + kHiBytes, lb = la + kTcABytes;
                    tc_mma_tf32(tmem, desc_sw128(sa + 32u * kk), desc_sw128(lb + 32u * kk), idesc, 1u);
                    tc_mma_tf32(tmem, desc_sw128(la + 32u * kk), desc_sw128(sb + 32u * kk), idesc, 1u);
                }
            }
            tc_commit(&empty[s]);  // the stage is free once these MMAs have read it
        }
        if (ok) tc_commit(done);
    } else if (SPLIT && warp >= 2) {
        // tile splitters: x = hi + lo with hi TF32-exact (written in place), lo = x - hi
        const int t = threadIdx.x - 64;
        for (int k = 0; k < ksteps; ++k) {
            const int s = k % kTcStages;
            if (!mbar_wait(&full[s], (unsigned)(k / kTcStages) & 1u)) {
                atomicExch(err, 1);
                break;
            }
            float4 *hi = reinterpret_cast<float4 *>(tiles + (size_t)s * kStageBytes);
            float4 *lo = reinterpret_cast<float4 *>(tiles + (size_t)s * kStageBytes + kHiBytes);
            for (int e = t; e < (int)(kHiBytes / 16); e += kSplitThreads) {
                const float4 x = hi[e];
                float4 h, l;
                h.x = __uint_as_float(__float_as_uint(x.x) & 0xFFFFE000u);
                h.y = __uint_as_float(__float_as_uint(x.y) & 0xFFFFE000u);
                h.z = __uint_as_float(__float_as_uint(x.z) & 0xFFFFE000u);
                h.w = __uint_as_float(__float_as_uint(x.w) & 0xFFFFE000u);
                l.x = x.x - h.x;
                l.y = x.y - h.y;
                l.z = x.z - h.z;
                l.w = x.w - h.w;
                hi[e] = h;
                lo[e] = l;
            }
            // make the generic-proxy writes visible to the tensor core (async proxy)
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&conv[s]);
        }
    }
    __syncwarp();
    // epilogue: thread = accumulator row (TMEM lane) 32 warp + lane
    // warp-uniform decision: tcgen05.ld below is a .sync.aligned warp instruction
    const bool ready = __all_sync(0xffffffffu, mbar_wait(done, 0u) ? 1 : 0) != 0;
    if (!ready && lane == 0) atomicExch(err, 1);
    tc_fence_after();
    if (ready) {
        const int r = 32 * warp + lane;
        float *yrow = Yb + (size_t)a * H.ldk + r0 + r;
#pragma unroll 1
        for (int cc = 0; cc < NT; cc += 16) {
            uint32_t v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)cc, v);
            if (r < nr) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int c = c0 + cc + j;
                    if (c < nb) yrow[(size_t)c * ldx] = __uint_as_float(v[j]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

template <int NT, bool SPLIT>
cudaError_t launch_tc(const DmHmat &H, const float *Xb, int64_t ldx, int nb, float *Yb, int *err, cudaStream_t st) {
    CUtensorMap tmA, tmA8, tmB;
    const uint64_t arows = (uint64_t)(1 << H.L) * H.leaf_max;
    const CUtensorMapDataType f32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    if (!tc_make_map(&tmA, f32, 4, H.Knear, (uint64_t)H.ldk, arows, (uint64_t)H.ldk, 32, 128) ||
        !tc_make_map(&tmA8, f32, 4, H.Knear, (uint64_t)H.ldk, arows, (uint64_t)H.ldk, 32, 8) ||
        !tc_make_map(&tmB, f32, 4, Xb, (uint64_t)ldx, (uint64_t)nb, (uint64_t)ldx, 32, NT))
        return cudaErrorInvalidValue;
    const int mtiles = (H.leaf_max + 127) / 128;
    constexpr int stages = tc_stages<NT, SPLIT>();
    const size_t smem = 1024 + (size_t)stages * tc_stage_bytes<NT, SPLIT>() + (3 * stages + 1) * 8 + 16;
    cudaError_t e = dm_allow_smem((const void *)tc_near_kernel<NT, SPLIT>, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((1 << H.L) * mtiles), (unsigned)((nb + NT - 1) / NT));
    tc_near_kernel<NT, SPLIT><<<grid, kTcThreads, smem, st>>>(tmA, tmA8, tmB, H, nb, Yb, ldx, mtiles, err);
    dm_count_launches(1);
    return cudaGetLastError();
}

template <bool SPLIT>
cudaError_t launch_tc_nb(const DmHmat &H, const float *Xb, int64_t ldx, int nb, float *Yb, int *err,
                         cudaStream_t st) {
    if (nb <= 16) return launch_tc<16, SPLIT>(H, Xb, ldx, nb, Yb, err, st);
    if (nb <= 32) return launch_tc<32, SPLIT>(H, Xb, ldx, nb, Yb, err, st);
    if (nb <= 64) return launch_tc<64, SPLIT>(H, Xb, ldx, nb, Yb, err, st);
    if (nb <= 128) return launch_tc<128, SPLIT>(H, Xb, ldx, nb, Yb, err, st);
    return launch_tc<256, SPLIT>(H, Xb, ldx, nb, Yb, err, st);
}

}  // namespace

bool dm_tc_available() { return tc_encode_fn() != nullptr; }

cudaError_t dm_launch_near_tc(const DmHmat &H, const float *Xb, int64_t ldx, int nb, float *Yb, int *err,
                              bool split, cudaStream_t st) {
    if (!H.Knear || (ldx & 3) != 0 || (H.ldk & 3) != 0) return cudaErrorInvalidValue;
    return split ? launch_tc_nb<true>(H, Xb, ldx, nb, Yb, err, st) : launch_tc_nb<false>(H, Xb, ldx, nb, Yb, err, st);
}
