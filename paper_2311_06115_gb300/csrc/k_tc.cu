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
// Every mbarrier wait is bounded (about a second of clock cycles); a wait that gives up
// raises *err, skips the stores and still frees the tensor memory, and the host reports
// DM_ETIMEOUT.
#include <cuda.h>

#include "dm_internal.cuh"

namespace {

constexpr int kTcThreads = 128;
constexpr int kTcStages = 4;
constexpr uint32_t kTcABytes = 128 * 128;  // 128 rows x 32 FP32
constexpr long long kTcWaitCycles = 1ll << 31;

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}
// wait until the phase with the given parity has completed; false after ~kTcWaitCycles
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
    const long long t0 = clock64();
    while (true) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(su32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > kTcWaitCycles) return false;
    }
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tm, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(su32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor for a K-major operand in the 128-byte swizzled layout:
// rows of 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), tile base 1024-byte
// aligned; the leading byte offset is not used by this layout.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;             // leading byte offset (16 B; unused here)
    d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
    d |= (uint64_t)1 << 46;             // descriptor version
    d |= (uint64_t)2 << 61;             // 128-byte swizzle
    return d;
}
// Instruction descriptor: D FP32, A and B TF32, both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void tc_mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int NT>
__global__ void __launch_bounds__(kTcThreads) tc_near_kernel(const __grid_constant__ CUtensorMap tmA,
                                                             const __grid_constant__ CUtensorMap tmA8,
                                                             const __grid_constant__ CUtensorMap tmB,
                                                             const __grid_constant__ DmHmat H, int nb,
                                                             float *__restrict__ Yb, int64_t ldx, int mtiles,
                                                             int *err) {
    static_assert(NT >= 16 && NT <= 256 && (NT & (NT - 1)) == 0, "NT: power of two in [16, 256]");
    constexpr uint32_t kBBytes = NT * 128;
    constexpr uint32_t kStageBytes = kTcABytes + kBBytes;
    constexpr uint32_t kTmemCols = NT < 32 ? 32 : NT;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = su32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *tiles = smem_raw + (base - raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(tiles + kTcStages * kStageBytes);
    uint64_t *empty = full + kTcStages;
    uint64_t *done = empty + kTcStages;
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
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
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
            if (!mbar_wait(&full[s], (unsigned)(k / kTcStages) & 1u)) {
                atomicExch(err, 1);
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t sa = base + (uint32_t)s * kStageBytes, sb = sa + kTcABytes;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                tc_mma_tf32(tmem, desc_sw128(sa + 32u * kk), desc_sw128(sb + 32u * kk), idesc,
                            (k > 0 || kk > 0) ? 1u : 0u);
            tc_commit(&empty[s]);  // the stage is free once these MMAs have read it
        }
        if (ok) tc_commit(done);
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// 2-D FP32 tensor map: `rows` rows of `cols` elements, row stride `ld` elements, box
// box_rows x 32 elements, 128-byte swizzle, zero fill outside
bool make_map(CUtensorMap *tm, const float *ptr, uint64_t cols, uint64_t rows, uint64_t ld, uint32_t box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {ld * sizeof(float)};
    const cuuint32_t box[2] = {32, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int NT>
cudaError_t launch_tc(const DmHmat &H, const float *Xb, int64_t ldx, int nb, float *Yb, int *err, cudaStream_t st) {
    CUtensorMap tmA, tmA8, tmB;
    const uint64_t arows = (uint64_t)(1 << H.L) * H.leaf_max;
    if (!make_map(&tmA, H.Knear, (uint64_t)H.ldk, arows, (uint64_t)H.ldk, 128) ||
        !make_map(&tmA8, H.Knear, (uint64_t)H.ldk, arows, (uint64_t)H.ldk, 8) ||
        !make_map(&tmB, Xb, (uint64_t)ldx, (uint64_t)nb, (uint64_t)ldx, NT))
        return cudaErrorInvalidValue;
    const int mtiles = (H.leaf_max + 127) / 128;
    const size_t smem = 1024 + (size_t)kTcStages * (kTcABytes + NT * 128) + (2 * kTcStages + 1) * 8 + 16;
    cudaError_t e = dm_allow_smem((const void *)tc_near_kernel<NT>, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((1 << H.L) * mtiles), (unsigned)((nb + NT - 1) / NT));
    tc_near_kernel<NT><<<grid, kTcThreads, smem, st>>>(tmA, tmA8, tmB, H, nb, Yb, ldx, mtiles, err);
    dm_count_launches(1);
    return cudaGetLastError();
}

}  // namespace

bool dm_tc_available() { return encode_fn() != nullptr; }

cudaError_t dm_launch_near_tc(const DmHmat &H, const float *Xb, int64_t ldx, int nb, float *Yb, int *err,
                              cudaStream_t st) {
    if (!H.Knear || (ldx & 3) != 0 || (H.ldk & 3) != 0) return cudaErrorInvalidValue;
    if (nb <= 16) return launch_tc<16>(H, Xb, ldx, nb, Yb, err, st);
    if (nb <= 32) return launch_tc<32>(H, Xb, ldx, nb, Yb, err, st);
    if (nb <= 64) return launch_tc<64>(H, Xb, ldx, nb, Yb, err, st);
    if (nb <= 128) return launch_tc<128>(H, Xb, ldx, nb, Yb, err, st);
    return launch_tc<256>(H, Xb, ldx, nb, Yb, err, st);
}
