// dm_capi.cu -- the C ABI of include/dmaps.h: handle lifetime, memory, host
// orchestration of the device phases, host/device buffer marshalling.
//
// Phases (all device work on the handle's stream):
//   dm_create   : bandwidth (optional), pre-scaled points, degrees q, dg, scaling s
//                 (Algorithm 1: similarity matrix and normalisations)
//   dm_compress : partition tree -> skeletons (interpolative decompositions) ->
//                 packed near and far blocks (Eq. 2.18)
//   dm_matvec   : y = K~ x (the LinearOperator of Section 3.3)
//   dm_eigs     : Lanczos with full reorthogonalisation (Algorithm 2, symmetric form)
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <algorithm>
#include <memory>
#include <vector>

#include <map>
#include <mutex>
#include "dm_internal.cuh"

cudaError_t dm_launch_dense_matvec_ws(const float *Xs, const float *sf, int64_t N, int d, const float *x, float *y,
                                      float *tmpw, double *acc, cudaStream_t st);

static std::atomic<long long> g_launches{0};
void dm_count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

// Pinned host staging for the convergence checks' device-to-host reads, one buffer per
// host thread, allocated once and reused (an eigensolve runs on one thread at a time):
// copies to pageable memory would each wait for the stream on their own.
double *check_staging(size_t count) {
    struct Buf {
        double *p = nullptr;
        size_t n = 0;
        ~Buf() {
            if (p) cudaFreeHost(p);
        }
    };
    thread_local Buf b;
    if (b.n < count) {
        if (b.p) cudaFreeHost(b.p);
        b.p = nullptr;
        b.n = 0;
        void *q = nullptr;
        if (cudaHostAlloc(&q, sizeof(double) * count, cudaHostAllocPortable) != cudaSuccess) return nullptr;
        b.p = static_cast<double *>(q);
        b.n = count;
    }
    return b.p;
}

}  // namespace

cudaError_t dm_allow_smem(const void *kern, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> raised;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    size_t &cap = raised[std::make_pair(dev, kern)];
    if (bytes <= cap) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cap = bytes;
    return e;
}

// message + status for entry points defined in other translation units
int dm_fail_msg(int code, const char *msg) { return fail(code, "%s", msg); }

namespace {

#define DM_CUDA(expr)                                                                                  \
    do {                                                                                               \
        cudaError_t _e = (expr);                                                                       \
        if (_e != cudaSuccess)                                                                         \
            return fail(DM_ECUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__, __LINE__); \
    } while (0)

#define DM_CHECK(expr)          \
    do {                        \
        int _s = (expr);        \
        if (_s != DM_OK) return _s; \
    } while (0)

enum Group { G_BASE = 0, G_STRUCT = 1, G_WORK = 2, G_LANCZOS = 3, G_IO = 4, G_BLOCK = 5, G_BLANCZOS = 6, G_NB = 7 };

// right-hand sides per block H-matvec call (wider blocks run as several panels): the FP32
// near field tiles 64 columns, the tensor-core one up to 256 (the largest MMA N)
constexpr int kBlockPanelFp32 = 64;
constexpr int kBlockPanelTc = 256;

struct Alloc {
    void *p;
    size_t bytes;
    int group;
};

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

}  // namespace

// The default pool of this process's context on `dev` keeps freed memory instead of
// returning it at every synchronisation (a setting of the pool, reset with the process)
inline void keep_pool_memory(int dev) {
    static std::mutex mu;
    static std::vector<int> done;
    std::lock_guard<std::mutex> lk(mu);
    for (int d : done)
        if (d == dev) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done.push_back(dev);
}

struct dm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    dm_config cfg;
    int64_t N = 0;
    int d = 0;
    double eps = 0, alpha = 1;
    std::vector<Alloc> allocs;
    // base
    float *X = nullptr, *Xs = nullptr, *sf = nullptr, *qaf = nullptr, *tmpw = nullptr;
    double *q = nullptr, *dg = nullptr, *s = nullptr, *qa = nullptr, *acc = nullptr;
    // structure
    bool compressed = false;
    double tol = 0;
    int L = 0, leaf_max = 0, ldk = 0, max_rank = 0, rank_hi = 0, cmax = 0, ldp = 0, near_mode = DM_NEAR_CACHED;
    int32_t *perm = nullptr, *ranks = nullptr, *skel = nullptr;
    float *P = nullptr, *B = nullptr, *Knear = nullptr, *Xp = nullptr, *sp = nullptr;
    float *what = nullptr, *uhat = nullptr, *ynear = nullptr, *PT = nullptr;
    unsigned *cnt = nullptr;
    int ldt = 4;
    int64_t *pt_off = nullptr;  // per leaf: offset and row stride of its point-major basis
    int *pt_ld = nullptr;
    int4 *tlay = nullptr;
    int2 *town = nullptr;
    float *timg = nullptr;
    int *timg_off = nullptr;
    int tree_ok = 0, tree_ls = 0, tree_smem = 0;
    int *herr = nullptr;
    std::vector<int32_t> rk_host;  // ranks per node (host copy, for layouts built later)
    // narrow-block (2..4 columns) cluster pass: nbt.nb = 0 until built; nb_fits = 0 when the
    // nb-wide layout of the last request did not fit the cluster's shared memory
    DmNbTree nbt{};
    int nb_tried = 0, nb_fits = 0;
    // lanczos
    DmLanczos lz{};
    bool lz_ready = false;
    int last_k = 0;
    float *evecs = nullptr;  // N x kmax, original order, last dm_eigs
    // block Lanczos state (bl.b = 0: not allocated)
    DmBlockLanczos bl{};
    // block H-matvec workspace (nb_max = 0: not allocated) and its near-field stream
    DmBlockWork blk{};
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // the tree build runs on its own high-priority stream, concurrently with the degree
    // passes still in flight on `stream` (it needs the points and eps, not the degrees)
    cudaStream_t tstream = nullptr;
    cudaEvent_t ev_pre = nullptr;   // recorded on `stream` before the degree passes
    cudaEvent_t ev_tree = nullptr;  // end of the tree build on `tstream`
    cudaEvent_t ev_sel = nullptr;   // end of the second median select on `tstream`
    cudaEvent_t cr_a = nullptr, cr_b = nullptr;  // create phase, resolved when stats are read
    cudaEvent_t ev_chk = nullptr;                 // end of a convergence check's reads
    cudaEvent_t ev_step = nullptr;                // end of the Lanczos step a check reads
    cudaStream_t cstream = nullptr;               // convergence checks beside the next step
    bool cr_pending = false;
    // phases timed by event pairs on a stream, resolved when stats are read (no host wait)
    struct Lap {
        cudaEvent_t a, b;
        float *dst;
    };
    std::vector<Lap> laps;
    cudaEvent_t lap_begin(cudaStream_t s) {
        cudaEvent_t a = nullptr;
        if (cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, s);
        return a;
    }
    void lap_end(cudaStream_t s, cudaEvent_t a, float *dst) {
        cudaEvent_t b = nullptr;
        if (!a || cudaEventCreate(&b) != cudaSuccess) return;
        cudaEventRecord(b, s);
        laps.push_back({a, b, dst});
    }
    void resolve_laps() {
        for (auto &l : laps) {
            float ms = 0.f;
            if (cudaEventSynchronize(l.b) == cudaSuccess && cudaEventElapsedTime(&ms, l.a, l.b) == cudaSuccess)
                *l.dst = ms;
            cudaEventDestroy(l.a);
            cudaEventDestroy(l.b);
        }
        laps.clear();
    }
    // io staging
    float *io_x = nullptr, *io_y = nullptr;
    int64_t io_elems = 0;
    dm_stats stats{};

    ~dm_ctx() {
        for (auto &a : allocs) release(a);
        allocs.clear();
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (side) cudaStreamDestroy(side);
        if (ev_pre) cudaEventDestroy(ev_pre);
        if (ev_tree) cudaEventDestroy(ev_tree);
        if (ev_sel) cudaEventDestroy(ev_sel);
        for (auto &l : laps) {
            cudaEventDestroy(l.a);
            cudaEventDestroy(l.b);
        }
        if (cr_a) cudaEventDestroy(cr_a);
        if (cr_b) cudaEventDestroy(cr_b);
        if (ev_chk) cudaEventDestroy(ev_chk);
        if (ev_step) cudaEventDestroy(ev_step);
        if (cstream) cudaStreamDestroy(cstream);
        if (tstream) cudaStreamDestroy(tstream);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
    void release(const Alloc &a) {
        if (!a.p) return;
        if (cfg.free) cfg.free(a.p, a.bytes, cfg.alloc_user);
        else cudaFreeAsync(a.p, stream);  // after every use enqueued on (or joined into) `stream`
    }
    // Without a caller allocator: stream-ordered allocations from the device's default pool
    // (no device-wide synchronisation; the pool keeps freed memory for the next request),
    // ordered on `on` (the stream that first uses the buffer; default `stream`).
    template <class T>
    int alloc(T **out, size_t count, int group, cudaStream_t on = nullptr) {
        size_t bytes = sizeof(T) * (count > 0 ? count : 1);
        bytes = (bytes + 255) & ~size_t(255);
        void *p = nullptr;
        if (cfg.alloc) {
            p = cfg.alloc(bytes, cfg.alloc_user);
            if (!p) return fail(DM_ENOMEM, "device allocation of %zu bytes failed (caller allocator)", bytes);
        } else {
            keep_pool_memory(device);
            cudaError_t e = cudaMallocAsync(&p, bytes, on ? on : stream);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(DM_ENOMEM, "cudaMallocAsync of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
            }
        }
        allocs.push_back({p, bytes, group});
        *out = reinterpret_cast<T *>(p);
        return DM_OK;
    }
    void free_group(int group) {
        std::vector<Alloc> keep;
        for (auto &a : allocs) {
            if (a.group == group) release(a);
            else keep.push_back(a);
        }
        allocs.swap(keep);
    }
    DmHmat hmat() const {
        DmHmat H;
        H.N = N;
        H.d = d;
        H.L = L;
        H.leaf_max = leaf_max;
        H.ldk = ldk;
        H.max_rank = max_rank;
        H.rank_hi = rank_hi > 0 ? rank_hi : max_rank;
        H.cmax = cmax;
        H.ldp = ldp;
        H.perm = perm;
        H.ranks = ranks;
        H.skel = skel;
        H.P = P;
        H.PT = PT;
        H.ldt = ldt;
        H.pt_off = pt_off;
        H.pt_ld = pt_ld;
        H.B = B;
        H.Knear = Knear;
        H.Xs = Xp;
        H.sp = sp;
        H.what = what;
        H.uhat = uhat;
        H.ynear = ynear;
        H.cnt = cnt;
        H.tlay = tlay;
        H.tree_ok = tree_ok;
        H.tree_ls = tree_ls;
        H.tree_smem = tree_smem;
        H.timg = timg;
        H.town = town;
        H.timg_off = timg_off;
        H.err = herr;
        return H;
    }
};

namespace {

struct PhaseTimer {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t st;
    explicit PhaseTimer(cudaStream_t s) : st(s) {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, st);
    }
    float stop() {
        cudaEventRecord(b, st);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        return ms;
    }
    ~PhaseTimer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// the handle's side stream (tree build, second median select) and its events
int ensure_tree_stream(dm_ctx *h) {
    if (h->tstream) return DM_OK;
    int lo = 0, hi = 0;
    DM_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    // highest priority: the tree's small latency-bound launches take SM slots ahead of the
    // degree pass's many blocks (only created when the solve has the device to itself)
    DM_CUDA(cudaStreamCreateWithPriority(&h->tstream, cudaStreamNonBlocking, hi));
    DM_CUDA(cudaEventCreateWithFlags(&h->ev_tree, cudaEventDisableTiming));
    DM_CUDA(cudaEventCreateWithFlags(&h->ev_sel, cudaEventDisableTiming));
    return DM_OK;
}

// the create phase is timed by two events resolved on first read, so dm_create returns with
// the degree passes still running (dm_compress overlaps its tree build with them)
void resolve_create_time(dm_ctx *h) {
    if (!h->cr_pending) return;
    float ms = 0.f;
    if (cudaEventSynchronize(h->cr_b) == cudaSuccess && cudaEventElapsedTime(&ms, h->cr_a, h->cr_b) == cudaSuccess)
        h->stats.ms_create = ms;
    h->cr_pending = false;
}

int set_device(dm_ctx *h) {
    int cur = -1;
    DM_CUDA(cudaGetDevice(&cur));
    if (cur != h->device) DM_CUDA(cudaSetDevice(h->device));
    return DM_OK;
}

// ensure io staging buffers of `elems` floats each
int ensure_io(dm_ctx *h, int64_t elems) {
    if (h->io_elems >= elems) return DM_OK;
    h->free_group(G_IO);
    h->io_x = h->io_y = nullptr;
    DM_CHECK(h->alloc(&h->io_x, (size_t)elems, G_IO));
    DM_CHECK(h->alloc(&h->io_y, (size_t)elems, G_IO));
    h->io_elems = elems;
    return DM_OK;
}

int copy_out(dm_ctx *h, void *dst, const void *src, size_t bytes) {
    DM_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, h->stream));
    return DM_OK;
}

// pack blocks, permuted points and matvec workspaces for the current tree/skeletons
// Shared-memory layout of the cluster pass over the upper tree. The tree is cut at level
// ls = min(3, L - 1) into 2^ls subtrees; CTA c of the cluster owns the subtree under node
// 2^ls - 1 + c (its internal nodes and its leaves' skeleton vectors). The 2^ls - 1 nodes above
// ls are spread one per CTA and level: node i of level lv < ls goes to CTA (2i+1) 2^(ls-lv-1).
// Each CTA's shared memory starts with the node metadata (layout and ranks of every node).
// The children of an internal node share a slot [w_l | w_r | u_l | u_r] (lay.z below ls, a
// scratch copy at lay.w above it); nodes at level ls keep their own [w | u] at lay.w, nodes
// above ls at lay.z; each internal node's P (column-major, column stride rank|1) and B (row
// stride s_r|1) follow.
// img_off gets each CTA's offset in the image buffer (floats, multiples of 4). Returns false
// when a CTA's share does not fit the budget (the chained two-launch path is used then).
bool tree_layout(const std::vector<int32_t> &rk, int L, int budget_floats, int ls_want, std::vector<int4> &lay,
                 std::vector<int2> &own, int &ls, int &smem_bytes, std::vector<int> &img_off) {
    if (L < 1) return false;
    ls = L - 1 < ls_want ? L - 1 : ls_want;
    const int nc = 1 << ls, nnodes = (1 << (L + 1)) - 1, ninternal = (1 << L) - 1;
    lay.assign(nnodes, make_int4(-1, -1, -1, -1));
    // every CTA first holds the node metadata: the layout (int4 per node), the ranks, and the
    // offsets of each node's own w and u (int2 per node)
    const int64_t meta = 4 * (int64_t)nnodes + ((nnodes + 3) & ~3) + 2 * (int64_t)nnodes;
    if (meta > budget_floats / 2) return false;
    std::vector<int64_t> used(nc, meta);
    auto owner = [&](int n) {
        const int lv = dm_level_of(n);
        if (lv >= ls) return ((n + 1) >> (lv - ls)) - nc;
        const int i = n - ((1 << lv) - 1);
        return (2 * i + 1) * (nc >> (lv + 1));
    };
    for (int n = 0; n < ninternal; ++n) {
        const int c = owner(n), lv = dm_level_of(n);
        const int64_t pair = 2 * (int64_t)(rk[2 * n + 1] + rk[2 * n + 2]);
        if (lv >= ls) {
            lay[n].z = (int)used[c];  // the children's [w_l | w_r | u_l | u_r]
            used[c] += pair;
            if (lv == ls && n > 0) {
                lay[n].w = (int)used[c];  // own [w | u]
                used[c] += 2 * rk[n];
            }
        } else {
            lay[n].w = (int)used[c];  // scratch copy of the children's pair
            used[c] += pair;
            if (n > 0) {
                lay[n].z = (int)used[c];  // own [w | u]
                used[c] += 2 * rk[n];
            }
        }
    }
    for (int n = 0; n < ninternal; ++n) {
        const int c = owner(n);
        const int sl = rk[2 * n + 1], sr = rk[2 * n + 2];
        lay[n].y = (int)used[c];
        used[c] += (int64_t)sl * (sr | 1);
        if (n == 0) continue;
        lay[n].x = (int)used[c];
        used[c] += (int64_t)(sl + sr) * (rk[n] | 1);
    }
    // own [w | u] of every non-root node: levels <= ls have their own slot, deeper nodes sit in
    // their parent's pair slot [w_l | w_r | u_l | u_r]
    own.assign(nnodes, make_int2(-1, -1));
    for (int n = 1; n < nnodes; ++n) {
        const int lv = dm_level_of(n);
        if (lv <= ls) {
            const int w = lv == ls ? lay[n].w : lay[n].z;
            own[n] = make_int2(w, w + rk[n]);
        } else {
            const int p = (n - 1) >> 1, sl = rk[2 * p + 1], sr = rk[2 * p + 2];
            const bool left = (n & 1) != 0;
            own[n] = make_int2(lay[p].z + (left ? 0 : sl), lay[p].z + sl + sr + (left ? 0 : sl));
        }
    }
    int64_t mx = 0;
    img_off.assign(nc + 1, 0);
    for (int c = 0; c < nc; ++c) {
        used[c] = (used[c] + 3) & ~int64_t(3);
        if (used[c] > budget_floats) return false;
        mx = used[c] > mx ? used[c] : mx;
        img_off[c + 1] = img_off[c] + (int)used[c];
    }
    smem_bytes = (int)(mx * 4);
    return true;
}

int finish_structure(dm_ctx *h) {
    const int nnodes = (1 << (h->L + 1)) - 1;
    const int nleaves = 1 << h->L;
    const bool cached = h->near_mode == DM_NEAR_CACHED;
    if (cached) DM_CHECK(h->alloc(&h->Knear, (size_t)nleaves * h->leaf_max * h->ldk, G_STRUCT));
    DM_CHECK(h->alloc(&h->B, (size_t)(nleaves > 1 ? nleaves - 1 : 1) * h->max_rank * h->max_rank, G_STRUCT));
    DM_CHECK(h->alloc(&h->what, (size_t)nnodes * h->max_rank, G_STRUCT));
    DM_CHECK(h->alloc(&h->uhat, (size_t)nnodes * h->max_rank, G_STRUCT));
    DM_CHECK(h->alloc(&h->ynear, (size_t)h->N, G_STRUCT));
    DM_CHECK(h->alloc(&h->cnt, (size_t)nnodes, G_STRUCT));
    DM_CUDA(cudaMemsetAsync(h->cnt, 0, sizeof(unsigned) * nnodes, h->stream));
    DM_CUDA(cudaMemsetAsync(h->what, 0, sizeof(float) * (size_t)nnodes * h->max_rank, h->stream));
    DM_CUDA(cudaMemsetAsync(h->uhat, 0, sizeof(float) * (size_t)nnodes * h->max_rank, h->stream));
    // near and sibling blocks need nothing from the host: enqueue them before the ranks'
    // round trip, which they then hide
    {
        DmHmat H0 = h->hmat();
        DM_CUDA(dm_pack(H0, h->Knear, h->B, cached, h->stream));
    }
    // statistics
    std::vector<int32_t> rk(nnodes);
    DM_CUDA(cudaMemcpyAsync(rk.data(), h->ranks, sizeof(int32_t) * nnodes, cudaMemcpyDeviceToHost, h->stream));
    DM_CUDA(cudaStreamSynchronize(h->stream));
    h->free_group(G_WORK);  // the skeletonization workspace: everything before is complete
    int rank_hi = 1;
    for (int node = 1; node < nnodes; ++node) rank_hi = rk[node] > rank_hi ? rk[node] : rank_hi;
    h->rank_hi = rank_hi;
    h->rk_host = rk;
    h->ldt = (int)round_up(rank_hi, 4);
    // point-major leaf bases, each leaf's rows at its own rank's stride (rounded up to 4):
    // the S2N reads then touch only the basis, not the padding to the largest leaf rank
    {
        std::vector<int64_t> off(nleaves);
        std::vector<int> ld(nleaves);
        int64_t tot = 0;
        for (int lf = 0; lf < nleaves; ++lf) {
            const int r = rk[nleaves - 1 + lf];
            ld[lf] = r > 4 ? (int)round_up(r, 4) : 4;
            off[lf] = tot;
            tot += (int64_t)h->leaf_max * ld[lf];
        }
        DM_CHECK(h->alloc(&h->PT, (size_t)tot, G_STRUCT));
        DM_CHECK(h->alloc(&h->pt_off, (size_t)nleaves, G_STRUCT));
        DM_CHECK(h->alloc(&h->pt_ld, (size_t)nleaves, G_STRUCT));
        // pageable sources: each copy returns once its source is staged
        DM_CUDA(cudaMemcpyAsync(h->pt_off, off.data(), sizeof(int64_t) * nleaves, cudaMemcpyHostToDevice, h->stream));
        DM_CUDA(cudaMemcpyAsync(h->pt_ld, ld.data(), sizeof(int) * nleaves, cudaMemcpyHostToDevice, h->stream));
    }
    DM_CHECK(h->alloc(&h->herr, 1, G_STRUCT));
    DM_CUDA(cudaMemsetAsync(h->herr, 0, sizeof(int), h->stream));
    {
        std::vector<int4> lay;
        std::vector<int2> own;
        std::vector<int> img_off;
        int ls = 0, smem = 0;
        h->tree_ok = 0;
        // a cluster of 8 CTAs (cut at level 3) when the upper tree fits their shared memory,
        // else 16 (cut at level 4; a non-portable cluster size, used when the device can
        // schedule it)
        bool fits = tree_layout(rk, h->L, kTreeSmemBudget / 4, 3, lay, own, ls, smem, img_off);
        if (!fits && h->L - 1 >= 4 && dm_tree_cluster_supported(16))
            fits = tree_layout(rk, h->L, kTreeSmemBudget / 4, 4, lay, own, ls, smem, img_off);
        if (fits) {
            DM_CHECK(h->alloc(&h->tlay, lay.size(), G_STRUCT));
            DM_CHECK(h->alloc(&h->town, own.size(), G_STRUCT));
            DM_CUDA(cudaMemcpyAsync(h->town, own.data(), sizeof(int2) * own.size(), cudaMemcpyHostToDevice,
                                    h->stream));
            DM_CHECK(h->alloc(&h->timg_off, img_off.size(), G_STRUCT));
            DM_CHECK(h->alloc(&h->timg, (size_t)img_off.back(), G_STRUCT));
            DM_CUDA(cudaMemcpyAsync(h->tlay, lay.data(), sizeof(int4) * lay.size(), cudaMemcpyHostToDevice,
                                    h->stream));
            // pageable sources: each copy returns once its source is staged, so the host
            // temporaries may go out of scope without a synchronisation
            DM_CUDA(cudaMemcpyAsync(h->timg_off, img_off.data(), sizeof(int) * img_off.size(),
                                    cudaMemcpyHostToDevice, h->stream));
            h->tree_ok = 1;
            h->tree_ls = ls;
            h->tree_smem = smem;
        }
    }
    DmHmat H = h->hmat();
    DM_CUDA(dm_transpose_leaf_bases(H, h->PT, h->stream));
    DM_CUDA(dm_tree_image(H, h->stream));
    int rmin = 1 << 30, rmax = 0;
    double rsum = 0;
    int64_t basis = 0, far = 0, near = 0;
    for (int node = 1; node < nnodes; ++node) {
        rmin = rk[node] < rmin ? rk[node] : rmin;
        rmax = rk[node] > rmax ? rk[node] : rmax;
        rsum += rk[node];
        int64_t st, sz;
        dm_node_range(h->N, node, &st, &sz);
        const int lvl = dm_level_of(node);
        const int64_t c = (lvl == h->L) ? sz : (int64_t)rk[2 * node + 1] + rk[2 * node + 2];
        basis += (int64_t)rk[node] * c * 4;
    }
    for (int node = 0; node < nleaves - 1; ++node) far += (int64_t)rk[2 * node + 1] * rk[2 * node + 2] * 4;
    for (int lf = 0; lf < nleaves; ++lf) {
        int64_t st, sz;
        dm_node_range(h->N, nleaves - 1 + lf, &st, &sz);
        near += sz * sz * 4;
    }
    int64_t sksum = 0;
    for (int node = 1; node < nnodes; ++node) sksum += rk[node];
    dm_stats &S = h->stats;
    S.L = h->L;
    S.tol = h->tol;
    S.leaf_max = h->leaf_max;
    S.max_rank = h->max_rank;
    S.rank_min = nnodes > 1 ? rmin : 0;
    S.rank_max = rmax;
    S.rank_mean = nnodes > 1 ? rsum / (nnodes - 1) : 0.0;
    S.near_bytes = cached ? near : 0;
    S.basis_bytes = basis;
    S.far_bytes = far;
    // algorithmic bytes of one nrhs=1 matvec: stored operands once, x and y once, skeleton
    // weights written and read once each
    S.matvec_bytes = (cached ? near : (int64_t)h->N * (h->d + 1) * 4) + basis + far + 2 * h->N * 4 + 2 * sksum * 4 * 2;
    S.near_mode = h->near_mode;
    S.hmatvec_path = (h->L == 0 || h->tree_ok) ? (h->tree_ok && h->tree_ls >= 4 ? 2 : 0) : 1;
    h->compressed = true;
    return DM_OK;
}

int alloc_structure(dm_ctx *h, int L, int max_rank) {
    h->free_group(G_STRUCT);
    h->free_group(G_NB);
    h->nbt = DmNbTree{};
    h->nb_tried = h->nb_fits = 0;
    h->free_group(G_BLOCK);
    h->blk.nb_max = 0;
    h->free_group(G_BLANCZOS);
    h->bl.b = 0;
    h->free_group(G_LANCZOS);
    h->lz_ready = false;
    h->compressed = false;
    h->Knear = nullptr;
    h->tlay = nullptr;
    h->town = nullptr;
    h->timg = nullptr;
    h->timg_off = nullptr;
    h->herr = nullptr;
    h->tree_ok = 0;
    h->L = L;
    h->leaf_max = (int)((h->N + ((int64_t)1 << L) - 1) >> L);
    h->ldk = (int)round_up(h->leaf_max, 4);
    h->max_rank = max_rank;
    h->cmax = h->leaf_max > 2 * max_rank ? h->leaf_max : 2 * max_rank;
    h->ldp = (int)round_up(h->cmax, 4);
    const int nnodes = (1 << (L + 1)) - 1;
    DM_CHECK(h->alloc(&h->ranks, (size_t)nnodes, G_STRUCT));
    DM_CHECK(h->alloc(&h->skel, (size_t)nnodes * max_rank, G_STRUCT));
    DM_CHECK(h->alloc(&h->P, (size_t)nnodes * max_rank * h->ldp, G_STRUCT));
    DM_CHECK(h->alloc(&h->Xp, (size_t)h->N * h->d, G_STRUCT));
    DM_CHECK(h->alloc(&h->sp, (size_t)h->N, G_STRUCT));
    DM_CUDA(cudaMemsetAsync(h->P, 0, sizeof(float) * (size_t)nnodes * max_rank * h->ldp, h->stream));
    return DM_OK;
}

int resolve_near_mode(dm_ctx *h) {
    int mode = h->cfg.near_mode;
    const size_t otf_smem = sizeof(float) * ((size_t)round_up(h->leaf_max, 4) + (size_t)h->leaf_max * h->d);
    if (mode == DM_NEAR_ONTHEFLY && otf_smem > 200 * 1024) mode = DM_NEAR_CACHED;
    if (mode == DM_NEAR_AUTO) mode = DM_NEAR_CACHED;
    h->near_mode = mode;
    return DM_OK;
}

// block H-matvec workspace for up to nb columns (sized for the current structure)
int ensure_block(dm_ctx *h, int nb) {
    if (h->blk.nb_max >= nb) return DM_OK;
    h->free_group(G_BLOCK);
    h->blk.nb_max = 0;
    const DmHmat H = h->hmat();
    const int64_t ldx = dm_block_ldx(H);
    const size_t nnodes = ((size_t)2 << h->L) - 1;
    DmBlockWork &W = h->blk;
    W.ldx = ldx;
    DM_CHECK(h->alloc(&W.Xb, (size_t)nb * ldx, G_BLOCK));
    DM_CHECK(h->alloc(&W.Yb, (size_t)nb * ldx, G_BLOCK));
    DM_CHECK(h->alloc(&W.Wb, nnodes * h->max_rank * nb, G_BLOCK));
    DM_CHECK(h->alloc(&W.Ub, nnodes * h->max_rank * nb, G_BLOCK));
    if (!h->side) {
        DM_CUDA(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
        DM_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        DM_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    }
    W.side = h->side;
    W.fork = h->ev_fork;
    W.join = h->ev_join;
    W.nb_max = nb;
    return DM_OK;
}

// The nb-column cluster pass (2 <= nb <= 4, cached near field): its layout, image and vector
// buffers, built on first use. *fits = 0 when the nb-wide upper tree does not fit the
// cluster's shared memory (the per-level block path is used then).
int ensure_nb(dm_ctx *h, int nb, bool *fits) {
    *fits = false;
    if (h->L < 1 || h->near_mode != DM_NEAR_CACHED || nb < 2 || nb > 4) return DM_OK;
    if (h->nbt.nb == nb) {
        *fits = true;
        return DM_OK;
    }
    if (h->nb_tried == nb && !h->nb_fits) return DM_OK;
    h->free_group(G_NB);
    h->nbt = DmNbTree{};
    h->nb_tried = nb;
    h->nb_fits = 0;
    DmNbLayout lay;
    if (!dm_nb_tree_layout(h->rk_host, h->L, nb, kTreeSmemBudget / 4, lay)) return DM_OK;
    const size_t nnodes = ((size_t)2 << h->L) - 1;
    DmNbTree T{};
    int4 *dlay = nullptr;
    int2 *down = nullptr;
    int *downer = nullptr, *doff = nullptr;
    DM_CHECK(h->alloc(&dlay, lay.lay.size(), G_NB));
    DM_CHECK(h->alloc(&down, lay.own.size(), G_NB));
    DM_CHECK(h->alloc(&downer, lay.owner.size(), G_NB));
    DM_CHECK(h->alloc(&doff, lay.img_off.size(), G_NB));
    DM_CHECK(h->alloc(&T.img, (size_t)lay.img_off.back(), G_NB));
    DM_CHECK(h->alloc(&T.what, nnodes * h->max_rank * nb, G_NB));
    DM_CHECK(h->alloc(&T.uhat, nnodes * h->max_rank * nb, G_NB));
    DM_CUDA(cudaMemcpyAsync(dlay, lay.lay.data(), sizeof(int4) * lay.lay.size(), cudaMemcpyHostToDevice, h->stream));
    DM_CUDA(cudaMemcpyAsync(down, lay.own.data(), sizeof(int2) * lay.own.size(), cudaMemcpyHostToDevice, h->stream));
    DM_CUDA(cudaMemcpyAsync(downer, lay.owner.data(), sizeof(int) * lay.owner.size(), cudaMemcpyHostToDevice,
                            h->stream));
    DM_CUDA(cudaMemcpyAsync(doff, lay.img_off.data(), sizeof(int) * lay.img_off.size(), cudaMemcpyHostToDevice,
                            h->stream));
    T.nb = nb;
    T.ls = lay.ls;
    T.smem = lay.smem;
    T.lay = dlay;
    T.own = down;
    T.owner = downer;
    T.img_off = doff;
    DM_CUDA(dm_nb_tree_image(h->hmat(), T, h->stream));
    // the host vectors above are pageable sources: each copy has staged them on return;
    // wait anyway so the layout is resident before the handle reports it
    DM_CUDA(cudaStreamSynchronize(h->stream));
    h->nbt = T;
    h->nb_fits = 1;
    *fits = true;
    return DM_OK;
}

// block Lanczos buffers for block size b (the basis itself is the Lanczos V)
int ensure_block_lanczos(dm_ctx *h, int b) {
    if (h->bl.b == b) return DM_OK;
    h->free_group(G_BLANCZOS);
    h->bl.b = 0;
    DmBlockLanczos &B = h->bl;
    const int mm = h->lz.m_max;
    int sms = 0;
    DM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    B.nparts = 2 * sms;
    if ((int64_t)B.nparts > h->N) B.nparts = (int)h->N;
    B.ldpart = mm + 1;
    DM_CHECK(h->alloc(&B.Z, (size_t)b * h->lz.ldv, G_BLANCZOS));
    DM_CHECK(h->alloc(&B.part, (size_t)B.nparts * B.ldpart * b, G_BLANCZOS));
    DM_CHECK(h->alloc(&B.H, (size_t)dm_bstep_hcopies() * B.ldpart * b, G_BLANCZOS));
    DM_CHECK(h->alloc(&B.Rinv, (size_t)b * b, G_BLANCZOS));
    DM_CHECK(h->alloc(&B.Bacc, (size_t)b * b, G_BLANCZOS));
    DM_CHECK(h->alloc(&B.T, (size_t)mm * mm, G_BLANCZOS));
    DM_CHECK(h->alloc(&B.W, (size_t)mm * mm, G_BLANCZOS));
    DM_CHECK(h->alloc(&B.hb, (size_t)mm, G_BLANCZOS));
    DM_CHECK(h->alloc(&B.flag, 1, G_BLANCZOS));
    DM_CHECK(h->alloc(&B.H1, (size_t)dm_bstep_hcopies() * B.ldpart * b, G_BLANCZOS));
    DM_CHECK(h->alloc(&B.Gacc, (size_t)3 * b * b, G_BLANCZOS));
    DM_CUDA(cudaMemsetAsync(B.Z, 0, sizeof(float) * (size_t)b * h->lz.ldv, h->stream));
    B.b = b;
    return DM_OK;
}

int ensure_lanczos(dm_ctx *h) {
    if (h->lz_ready) return DM_OK;
    const int kmax = dm_lanczos_kmax();
    DmLanczos &L = h->lz;
    L.N = h->N;
    L.ldv = round_up(h->N, 64);
    L.m_max = h->cfg.m_max;
    // every buffer of the eigensolver carved from one allocation (one allocator call per
    // handle: many small handles -- batched clouds, serving -- pay for calls, not bytes)
    size_t total = 0;
    auto take = [&](size_t bytes) {
        const size_t off = total;
        total += (bytes + 255) & ~size_t(255);
        return off;
    };
    const size_t oV = take(sizeof(float) * (size_t)(L.m_max + 1) * L.ldv);
    const size_t oz = take(sizeof(float) * (size_t)L.ldv);
    const size_t oal = take(sizeof(double) * ((size_t)L.m_max + 1));
    const size_t obe = take(sizeof(double) * ((size_t)L.m_max + 1));
    const size_t oh = take(sizeof(double) * (size_t)2 * (2 * (L.m_max + 1) + 2));
    const size_t onr = take(sizeof(double));
    const size_t oth = take(sizeof(double) * (size_t)kmax);
    const size_t ors = take(sizeof(double) * (size_t)kmax);
    const size_t oY = take(sizeof(double) * (size_t)kmax * L.m_max);
    const size_t oYf = take(sizeof(float) * (size_t)kmax * L.m_max);
    const size_t otw = take(sizeof(double) * (size_t)kmax * 6 * L.m_max);
    const size_t ocs = take(sizeof(double) * (size_t)kmax);
    const size_t oph = take(sizeof(float) * (size_t)kmax * h->N);
    const size_t obs = take(sizeof(unsigned long long) * (size_t)kmax);
    const size_t ong = take(sizeof(int) * (size_t)kmax);
    const size_t obar = take(sizeof(unsigned));
    const size_t oerr = take(sizeof(int));
    const size_t oev = take(sizeof(float) * (size_t)kmax * h->N);
    unsigned char *base = nullptr;
    DM_CHECK(h->alloc(&base, total, G_LANCZOS));
    L.V = reinterpret_cast<float *>(base + oV);
    L.z = reinterpret_cast<float *>(base + oz);
    L.alpha = reinterpret_cast<double *>(base + oal);
    L.beta = reinterpret_cast<double *>(base + obe);
    L.h = reinterpret_cast<double *>(base + oh);
    L.nrm2 = reinterpret_cast<double *>(base + onr);
    L.theta = reinterpret_cast<double *>(base + oth);
    L.resid = reinterpret_cast<double *>(base + ors);
    L.Y = reinterpret_cast<double *>(base + oY);
    L.Yf = reinterpret_cast<float *>(base + oYf);
    L.twork = reinterpret_cast<double *>(base + otw);
    L.colsum = reinterpret_cast<double *>(base + ocs);
    L.phi = reinterpret_cast<float *>(base + oph);
    L.best = reinterpret_cast<unsigned long long *>(base + obs);
    L.neg = reinterpret_cast<int *>(base + ong);
    L.bar = reinterpret_cast<unsigned *>(base + obar);
    L.err = reinterpret_cast<int *>(base + oerr);
    h->evecs = reinterpret_cast<float *>(base + oev);
    DM_CUDA(cudaMemsetAsync(L.err, 0, sizeof(int), h->stream));
    // zero the whole basis once: padding rows beyond N must read as zero
    // only the padding rows N..ldv-1 of each basis column are read before being written
    // (the step kernel works on 16-byte row quads up to ldv): zero those, not the whole basis
    if (L.ldv > h->N)
        DM_CUDA(cudaMemset2DAsync(L.V + h->N, sizeof(float) * (size_t)L.ldv, 0,
                                  sizeof(float) * (size_t)(L.ldv - h->N), (size_t)(L.m_max + 1), h->stream));
    DM_CUDA(cudaMemsetAsync(L.z, 0, sizeof(float) * (size_t)L.ldv, h->stream));
    h->lz_ready = true;
    return DM_OK;
}

// Block Lanczos with b <= 4 vectors per step (FP32 near field, cached blocks) when the b-wide
// upper tree fits the cluster pass: per step the three chained launches of the narrow-block
// H-matvec and one cooperative step kernel (CGS2 + CholQR2, FP64 coefficients); Rayleigh-Ritz
// on the projected matrix at the checks, as eigs_block. *done = false: not applicable.
int eigs_narrow(dm_ctx *h, int k, double *evals, float *evecs, bool *done) {
    *done = false;
    const int b = h->cfg.block_size;
    if (b < 2 || b > dm_bstep_max_b() || h->cfg.block_precision != DM_PREC_FP32 || h->cfg.shared_device) return DM_OK;
    bool fits = false;
    DM_CHECK(ensure_nb(h, b, &fits));
    if (!fits) return DM_OK;
    DmLanczos &Lz = h->lz;
    int m_cap = Lz.m_max;
    if (m_cap > h->N) m_cap = (int)h->N;
    const int jmax = m_cap / b - 1;
    if (jmax < 1 || (jmax * b) < k) return fail(DM_EINVAL, "m_max too small for block_size %d and k %d", b, k);
    DM_CHECK(ensure_block_lanczos(h, b));
    int sms = 0;
    DM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    *done = true;
    PhaseTimer t(h->stream);
    DmBlockLanczos &B = h->bl;
    const DmHmat H = h->hmat();
    const int64_t hstride = (int64_t)B.ldpart * b;
    DM_CUDA(cudaMemsetAsync(B.H, 0, sizeof(double) * (size_t)dm_bstep_hcopies() * hstride, h->stream));
    DM_CUDA(cudaMemsetAsync(B.H1, 0, sizeof(double) * (size_t)dm_bstep_hcopies() * hstride, h->stream));
    DM_CUDA(cudaMemsetAsync(B.Gacc, 0, sizeof(double) * 3 * b * b, h->stream));
    DM_CUDA(cudaMemsetAsync(Lz.bar, 0, sizeof(unsigned), h->stream));
    DM_CUDA(dm_bl_random_block(Lz, B, h->perm, h->cfg.seed, h->stream));
    unsigned bar_base = 0;
    int par = 0;
    double *G1 = B.Gacc, *G2 = B.Gacc + b * b;
    // V_0 = CholQR2 of the random block (no basis to orthogonalise against)
    DM_CUDA(dm_bstep(b, Lz.V, Lz.ldv, 0, 0, B.Z, B.H, B.H1, hstride, G1, G2, par, nullptr, Lz.m_max, B.Bacc, B.flag,
                     Lz.bar, bar_base, Lz.err, sms, h->stream));
    bar_base += 3u * (unsigned)sms;
    par ^= 1;
    std::vector<double> th(k), rs(k);
    int m = 0, flag = 0, total = 0, restarts = 0;
    bool converged = false, ritz_current = false;
    const bool prof = h->cfg.profile != 0;
    std::vector<cudaEvent_t> ev_mv;
    const int every = h->cfg.check_every / b > 2 ? h->cfg.check_every / b : 2;
    int since = 0;
    // thick restart once the basis is full: keep kr Ritz vectors (k plus half as many again, at
    // least one block more) and the newest block; the step after it needs kr + 2b columns
    const int cap = m_cap + 1;  // basis columns available (V holds m_max + 1)
    int kr = k + (k / 2 > b ? k / 2 : b);
    if (kr > dm_lanczos_kmax()) kr = dm_lanczos_kmax();
    const bool can_restart = kr >= k && kr + 3 * b <= cap;
    constexpr int kMaxRestarts = 64;
    int col = 0;  // first column of the current block V_j
    while (col + 2 * b <= cap) {
        if (prof) {
            cudaEvent_t e0, e1;
            DM_CUDA(cudaEventCreate(&e0));
            DM_CUDA(cudaEventCreate(&e1));
            ev_mv.push_back(e0);
            ev_mv.push_back(e1);
            DM_CUDA(cudaEventRecord(e0, h->stream));
        }
        DM_CUDA(dm_hmatvec_nb(H, h->nbt, b, Lz.V + (size_t)col * Lz.ldv, Lz.ldv, B.Z, Lz.ldv, true, h->stream));
        if (prof) DM_CUDA(cudaEventRecord(ev_mv.back(), h->stream));
        DM_CUDA(dm_bstep(b, Lz.V, Lz.ldv, col + b, col + b, B.Z, B.H, B.H1, hstride, G1, G2, par, B.T, Lz.m_max,
                         B.Bacc, B.flag, Lz.bar, bar_base, Lz.err, sms, h->stream));
        bar_base += 3u * (unsigned)sms;
        par ^= 1;
        col += b;
        m = col;
        total += b;
        ritz_current = false;
        ++since;
        const bool full = col + 2 * b > cap;  // the next step has no room: check (and restart) now
        if ((m >= 2 * k && since >= every) || (full && m >= k)) {
            since = 0;
            const int want = full && can_restart && restarts < kMaxRestarts ? kr : k;
            DM_CUDA(dm_bl_ritz(Lz, B, m, want, h->stream));
            DM_CUDA(cudaMemcpyAsync(th.data(), Lz.theta, sizeof(double) * k, cudaMemcpyDeviceToHost, h->stream));
            DM_CUDA(cudaMemcpyAsync(rs.data(), Lz.resid, sizeof(double) * k, cudaMemcpyDeviceToHost, h->stream));
            DM_CUDA(cudaMemcpyAsync(&flag, B.flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
            DM_CUDA(cudaStreamSynchronize(h->stream));
            ritz_current = want == k;
            const double scale = std::fabs(th[0]) > 0 ? std::fabs(th[0]) : 1.0;
            bool ok = true;
            for (int i = 0; i < k; ++i)
                if (!(rs[i] <= h->cfg.conv_tol * scale)) ok = false;
            if (ok || flag) {
                converged = ok;
                if (!ritz_current) {
                    DM_CUDA(dm_bl_ritz(Lz, B, m, k, h->stream));
                    ritz_current = true;
                }
                break;
            }
            if (want == kr) {
                DM_CUDA(dm_lanczos_restart(Lz, m, kr, m, b, B.T, Lz.m_max, h->stream));
                col = kr;
                m = kr;
                ++restarts;
                ritz_current = false;
            }
        }
    }
    if (!ritz_current) {
        DM_CUDA(dm_bl_ritz(Lz, B, m, k, h->stream));
        DM_CUDA(cudaMemcpyAsync(th.data(), Lz.theta, sizeof(double) * k, cudaMemcpyDeviceToHost, h->stream));
    }
    DM_CUDA(dm_lanczos_phi(Lz, m, k, h->perm, h->evecs, h->stream));
    DM_CUDA(cudaStreamSynchronize(h->stream));
    {
        int err = 0;
        DM_CUDA(cudaMemcpyAsync(&err, Lz.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        DM_CUDA(cudaStreamSynchronize(h->stream));
        if (err) {
            DM_CUDA(cudaMemsetAsync(Lz.err, 0, sizeof(int), h->stream));
            DM_CUDA(cudaStreamSynchronize(h->stream));
            return fail(DM_ETIMEOUT, "a grid barrier of the block Lanczos step gave up waiting");
        }
    }
    if (is_device_ptr(evals))
        DM_CUDA(cudaMemcpyAsync(evals, th.data(), sizeof(double) * k, cudaMemcpyHostToDevice, h->stream));
    else
        for (int i = 0; i < k; ++i) evals[i] = th[i];
    if (evecs) DM_CHECK(copy_out(h, evecs, h->evecs, sizeof(float) * (size_t)k * h->N));
    DM_CUDA(cudaStreamSynchronize(h->stream));
    h->stats.matvec_calls = 0;
    h->stats.ms_matvec = 0.f;
    for (size_t e = 0; e + 1 < ev_mv.size(); e += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev_mv[e], ev_mv[e + 1]) == cudaSuccess) {
            h->stats.ms_matvec += ms;
            h->stats.matvec_calls += 1;
        }
        cudaEventDestroy(ev_mv[e]);
        cudaEventDestroy(ev_mv[e + 1]);
    }
    h->last_k = k;
    h->stats.lanczos_iters = total;
    h->stats.converged = converged ? 1 : 0;
    h->stats.ms_eigs = t.stop();
    return converged ? DM_OK
                     : fail(DM_ENOCONV, "block Lanczos did not converge in %d basis vectors (%d restarts)", total,
                            restarts);
}

// dm_eigs with block Lanczos (cfg.block_size = b >= 2): per step one block H-matvec of b
// columns, block CGS2 and CholQR2; Rayleigh-Ritz on the projected matrix every check.
int eigs_block(dm_ctx *h, int k, double *evals, float *evecs) {
    const int b = h->cfg.block_size;
    {
        bool done = false;
        const int st = eigs_narrow(h, k, evals, evecs, &done);
        if (done || st != DM_OK) return st;
    }
    if (b > dm_block_lanczos_max_b()) return fail(DM_EINVAL, "block_size must be <= %d", dm_block_lanczos_max_b());
    DmLanczos &Lz = h->lz;
    int m_cap = Lz.m_max;
    if (m_cap > h->N) m_cap = (int)h->N;
    // blocks 0..jmax of V (and of T's columns, whose last block holds B^T) fit in m_cap columns
    const int jmax = m_cap / b - 1;
    if (jmax < 1 || (jmax * b) < k) return fail(DM_EINVAL, "m_max too small for block_size %d and k %d", b, k);
    DM_CHECK(ensure_block_lanczos(h, b));
    DM_CHECK(ensure_block(h, b));
    const bool tc = h->cfg.block_precision != DM_PREC_FP32 && h->near_mode == DM_NEAR_CACHED;
    if (tc && !dm_tc_available()) return fail(DM_ECUDA, "the driver does not provide cuTensorMapEncodeTiled");
    const int near_prec = tc ? h->cfg.block_precision : DM_PREC_FP32;
    PhaseTimer t(h->stream);
    DmBlockLanczos &B = h->bl;
    const DmHmat H = h->hmat();
    DM_CUDA(dm_bl_start(Lz, B, h->perm, h->cfg.seed, h->stream));
    std::vector<double> th(k), rs(k);
    int m = 0, flag = 0;
    bool converged = false, ritz_current = false;
    const bool prof = h->cfg.profile != 0;
    std::vector<cudaEvent_t> ev_mv;
    // each Rayleigh-Ritz check costs an FP64 tridiagonalisation: at most every other block
    const int every = h->cfg.check_every / b > 2 ? h->cfg.check_every / b : 2;
    int since = 0;
    for (int j = 0; j < jmax; ++j) {
        if (prof) {
            cudaEvent_t e0, e1;
            DM_CUDA(cudaEventCreate(&e0));
            DM_CUDA(cudaEventCreate(&e1));
            ev_mv.push_back(e0);
            ev_mv.push_back(e1);
            DM_CUDA(cudaEventRecord(e0, h->stream));
        }
        DM_CUDA(dm_hmatvec_block(H, h->near_mode, near_prec, h->blk, b, Lz.V + (size_t)j * b * Lz.ldv, Lz.ldv,
                                 nullptr, false, B.Z, Lz.ldv, DM_BLK_POSITION, h->stream));
        if (prof) DM_CUDA(cudaEventRecord(ev_mv.back(), h->stream));
        DM_CUDA(dm_bl_orth(Lz, B, j, h->stream));
        m = (j + 1) * b;
        ritz_current = false;
        ++since;
        const bool last = j + 1 == jmax;
        if (m >= 2 * k && (since >= every || last)) {
            since = 0;
            DM_CUDA(dm_bl_ritz(Lz, B, m, k, h->stream));
            DM_CUDA(cudaMemcpyAsync(th.data(), Lz.theta, sizeof(double) * k, cudaMemcpyDeviceToHost, h->stream));
            DM_CUDA(cudaMemcpyAsync(rs.data(), Lz.resid, sizeof(double) * k, cudaMemcpyDeviceToHost, h->stream));
            DM_CUDA(cudaMemcpyAsync(&flag, B.flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
            DM_CUDA(cudaStreamSynchronize(h->stream));
            ritz_current = true;
            const double scale = std::fabs(th[0]) > 0 ? std::fabs(th[0]) : 1.0;
            bool ok = true;
            for (int i = 0; i < k; ++i)
                if (!(rs[i] <= h->cfg.conv_tol * scale)) ok = false;
            if (ok || flag) {
                converged = ok;
                break;
            }
        }
    }
    if (!ritz_current) {
        DM_CUDA(dm_bl_ritz(Lz, B, m, k, h->stream));
        DM_CUDA(cudaMemcpyAsync(th.data(), Lz.theta, sizeof(double) * k, cudaMemcpyDeviceToHost, h->stream));
    }
    DM_CUDA(dm_lanczos_phi(Lz, m, k, h->perm, h->evecs, h->stream));
    DM_CUDA(cudaStreamSynchronize(h->stream));
    if (tc) {
        int err = 0;
        DM_CUDA(cudaMemcpyAsync(&err, h->herr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        DM_CUDA(cudaStreamSynchronize(h->stream));
        if (err) {
            DM_CUDA(cudaMemsetAsync(h->herr, 0, sizeof(int), h->stream));
            DM_CUDA(cudaStreamSynchronize(h->stream));
            return fail(DM_ETIMEOUT, "a bounded wait of the tensor-core near field gave up");
        }
    }
    if (is_device_ptr(evals))
        DM_CUDA(cudaMemcpyAsync(evals, th.data(), sizeof(double) * k, cudaMemcpyHostToDevice, h->stream));
    else
        for (int i = 0; i < k; ++i) evals[i] = th[i];
    if (evecs) DM_CHECK(copy_out(h, evecs, h->evecs, sizeof(float) * (size_t)k * h->N));
    DM_CUDA(cudaStreamSynchronize(h->stream));
    h->stats.matvec_calls = 0;
    h->stats.ms_matvec = 0.f;
    for (size_t e = 0; e + 1 < ev_mv.size(); e += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev_mv[e], ev_mv[e + 1]) == cudaSuccess) {
            h->stats.ms_matvec += ms;
            h->stats.matvec_calls += 1;
        }
        cudaEventDestroy(ev_mv[e]);
        cudaEventDestroy(ev_mv[e + 1]);
    }
    h->last_k = k;
    h->stats.lanczos_iters = m;
    h->stats.converged = converged ? 1 : 0;
    h->stats.ms_eigs = t.stop();
    return converged ? DM_OK : fail(DM_ENOCONV, "block Lanczos did not converge in %d basis vectors", m);
}

}  // namespace

extern "C" {

void dm_config_default(dm_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->seed = 0;
    cfg->near_mode = DM_NEAR_AUTO;
    cfg->m_max = 300;
    cfg->conv_tol = 1e-7;
    cfg->check_every = 1;
    cfg->device = -1;
    cfg->stream = nullptr;
}

const char *dm_status_str(int status) {
    switch (status) {
        case DM_OK: return "DM_OK";
        case DM_EINVAL: return "DM_EINVAL";
        case DM_ENOMEM: return "DM_ENOMEM";
        case DM_ESTATE: return "DM_ESTATE";
        case DM_ENOCONV: return "DM_ENOCONV";
        case DM_ETIMEOUT: return "DM_ETIMEOUT";
        case DM_ECUDA: return "DM_ECUDA";
        case DM_EBUSY: return "DM_EBUSY";
        default: return "DM_UNKNOWN";
    }
}

const char *dm_last_error(void) { return g_err.c_str(); }

int64_t dm_kernel_launches(void) { return (int64_t)g_launches.load(); }

int dm_sfu_peak(int64_t *ex2_count, float *ms) {
    if (!ex2_count || !ms) return fail(DM_EINVAL, "dm_sfu_peak: NULL output");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(DM_ECUDA, "dm_sfu_peak: no device");
    }
    const int blocks = 8 * sms, iters = 4096;
    float *out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * (size_t)blocks * 256) != cudaSuccess) {
        cudaGetLastError();
        return fail(DM_ENOMEM, "dm_sfu_peak: cudaMalloc failed");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = dm_launch_ex2_peak(out, blocks, iters, 0);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) e = dm_launch_ex2_peak(out, blocks, iters, 0);
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(DM_ECUDA, "dm_sfu_peak: %s", cudaGetErrorString(e));
    }
    *ex2_count = (int64_t)blocks * 256 * 8 * iters;
    *ms = t;
    return DM_OK;
}

int dm_selftest_wait_timeout(int32_t blocks, int32_t missing, int64_t spin_limit, int32_t *passed) {
    if (blocks < 1 || blocks > 8 || missing < 0 || spin_limit < 1 || spin_limit > ((int64_t)1 << 24))
        return fail(DM_EINVAL, "dm_selftest_wait_timeout: needs 1 <= blocks <= 8, missing >= 0, "
                               "1 <= spin_limit <= 2^24");
    void *mem = nullptr;
    if (cudaMalloc(&mem, 16) != cudaSuccess) {
        cudaGetLastError();
        return fail(DM_ENOMEM, "dm_selftest_wait_timeout: cudaMalloc of 16 bytes failed");
    }
    unsigned *ctr = static_cast<unsigned *>(mem);
    int *err = reinterpret_cast<int *>(ctr + 2);
    unsigned host[2] = {0, 0};
    int herr = 0;
    cudaError_t e = dm_launch_barrier_selftest(ctr, err, blocks, missing, (long long)spin_limit, 0);
    if (e == cudaSuccess) e = cudaMemcpy(host, ctr, sizeof(host), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(mem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(DM_ECUDA, "dm_selftest_wait_timeout: %s", cudaGetErrorString(e));
    }
    if (passed) *passed = (int32_t)host[1];
    if (herr) return fail(DM_ETIMEOUT, "dm_selftest_wait_timeout: the grid barrier gave up waiting (as intended "
                                       "when arrivals are missing)");
    return DM_OK;
}

int dm_create(const float *points, int64_t N, int32_t d, double eps, double alpha, const dm_config *cfg,
              dm_handle *out) {
    if (!out) return fail(DM_EINVAL, "out handle is NULL");
    *out = nullptr;
    if (!points) return fail(DM_EINVAL, "points is NULL");
    if (N < 2) return fail(DM_EINVAL, "N must be >= 2 (got %lld)", (long long)N);
    if (N > (int64_t)0x7fffffff) return fail(DM_EINVAL, "N must fit in int32");
    if (d < 1) return fail(DM_EINVAL, "d must be >= 1 (got %d)", d);
    if (!(alpha >= 0.0) || !std::isfinite(alpha)) return fail(DM_EINVAL, "alpha must be finite and >= 0");
    if (!std::isfinite(eps)) return fail(DM_EINVAL, "eps must be finite");
    if (cfg && (cfg->block_precision < DM_PREC_FP32 || cfg->block_precision > DM_PREC_TF32X3))
        return fail(DM_EINVAL, "block_precision must be DM_PREC_FP32, DM_PREC_TF32 or DM_PREC_TF32X3");
    dm_ctx *h = new dm_ctx();
    dm_config_default(&h->cfg);
    if (cfg) h->cfg = *cfg;
    if (h->cfg.m_max < 2) h->cfg.m_max = 2;
    if (h->cfg.check_every < 1) h->cfg.check_every = 1;
    if (!(h->cfg.conv_tol > 0)) h->cfg.conv_tol = 1e-7;
    int rc;
    {
        int cur = 0;
        if (cudaGetDevice(&cur) != cudaSuccess) {
            delete h;
            return fail(DM_ECUDA, "no CUDA device available");
        }
        h->device = h->cfg.device >= 0 ? h->cfg.device : cur;
        if (cudaSetDevice(h->device) != cudaSuccess) {
            delete h;
            return fail(DM_ECUDA, "cudaSetDevice(%d) failed", h->device);
        }
    }
    if (h->cfg.stream) h->stream = reinterpret_cast<cudaStream_t>(h->cfg.stream);
    else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            return fail(DM_ECUDA, "cudaStreamCreate failed");
        }
        h->own_stream = true;
    }
    h->N = N;
    h->d = d;
    h->alpha = alpha;
    h->stats.N = N;
    h->stats.d = d;
    h->stats.alpha = alpha;
    rc = [&]() -> int {
        DM_CUDA(cudaEventCreate(&h->cr_a));
        DM_CUDA(cudaEventCreate(&h->cr_b));
        DM_CUDA(cudaEventCreateWithFlags(&h->ev_pre, cudaEventDisableTiming));
        // a side stream for the overlapped phases when the solve has the device to itself;
        // on a shared device (serving slots) the other solves fill it, and one stream per
        // request avoids creating streams per request
        if (!h->cfg.shared_device) DM_CHECK(ensure_tree_stream(h));
        DM_CUDA(cudaEventRecord(h->cr_a, h->stream));
        DM_CHECK(h->alloc(&h->X, (size_t)N * d, G_BASE));
        DM_CUDA(cudaMemcpyAsync(h->X, points, sizeof(float) * (size_t)N * d, cudaMemcpyDefault, h->stream));
        // the caller may reuse `points` once dm_create returns: wait for this copy (only)
        DM_CUDA(cudaEventRecord(h->ev_pre, h->stream));
        DM_CUDA(cudaEventSynchronize(h->ev_pre));
        if (eps <= 0.0) {
            const int64_t npairs = N * (N - 1) / 2;
            const int64_t m = npairs <= ((int64_t)1 << 20) ? npairs : ((int64_t)1 << 20);
            double *pairs = nullptr, *res = nullptr;
            unsigned char *sel = nullptr;
            DM_CHECK(h->alloc(&pairs, (size_t)m, G_WORK));
            DM_CHECK(h->alloc(&res, 1, G_WORK));
            DM_CHECK(h->alloc(&sel, 2 * dm_select_state_bytes(), G_WORK));
            DM_CUDA(dm_launch_pair_sqdist(h->X, N, d, h->cfg.seed, pairs, m, h->stream));
            DM_CUDA(dm_launch_select_median(pairs, m, sel, res, h->stream, h->tstream, h->ev_tree, h->ev_sel));
            // (tstream, ev_tree, ev_sel are null on a shared device: one stream)
            DM_CUDA(cudaMemcpyAsync(&eps, res, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            DM_CUDA(cudaStreamSynchronize(h->stream));
            h->free_group(G_WORK);
            if (!(eps > 0.0)) return fail(DM_EINVAL, "median squared distance is %g (duplicate points?)", eps);
        }
        h->eps = eps;
        h->stats.eps = eps;
        DM_CHECK(h->alloc(&h->Xs, (size_t)N * d, G_BASE));
        DM_CHECK(h->alloc(&h->q, (size_t)N, G_BASE));
        DM_CHECK(h->alloc(&h->dg, (size_t)N, G_BASE));
        DM_CHECK(h->alloc(&h->s, (size_t)N, G_BASE));
        DM_CHECK(h->alloc(&h->qa, (size_t)N, G_BASE));
        DM_CHECK(h->alloc(&h->acc, (size_t)N, G_BASE));
        DM_CHECK(h->alloc(&h->sf, (size_t)N, G_BASE));
        DM_CHECK(h->alloc(&h->qaf, (size_t)N, G_BASE));
        DM_CHECK(h->alloc(&h->tmpw, (size_t)N, G_BASE));
        // the degree passes' temporaries live as long as the handle: dm_create returns while
        // those passes may still run
        float *nrm = nullptr, *nmax = nullptr;
        double *cwork = nullptr;
        DM_CHECK(h->alloc(&nrm, (size_t)N, G_BASE));
        DM_CHECK(h->alloc(&nmax, 1, G_BASE));
        DM_CHECK(h->alloc(&cwork, 8, G_BASE));
        DM_CUDA(dm_launch_center_scale(h->X, N, d, eps, h->Xs, nrm, nmax, cwork, h->stream));
        DM_CUDA(cudaEventRecord(h->ev_pre, h->stream));
        if (d >= kDegTcMinD && dm_degtc_available()) {
            // high dimension: the Gram matrix on the tensor cores, exp and row sums fused
            unsigned char *work = nullptr;
            int *derr = nullptr;
            DM_CHECK(h->alloc(&work, dm_degtc_work_bytes(N, d), G_WORK));
            DM_CHECK(h->alloc(&derr, 1, G_WORK));
            DM_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), h->stream));
            DmDegTc S{};
            cudaEvent_t lap = h->lap_begin(h->stream);
            DM_CUDA(dm_degtc_prepare(h->X, N, d, eps, work, &S, h->stream));
            DM_CUDA(dm_degtc_pass(S, nullptr, h->q, derr, h->stream));
            DM_CUDA(dm_launch_finish_degrees(N, alpha, h->q, h->qa, h->qaf, h->stream));
            DM_CUDA(dm_degtc_pass(S, h->qaf, h->dg, derr, h->stream));
            h->lap_end(h->stream, lap, &h->stats.ms_degrees);
            DM_CUDA(dm_launch_finish_scaling(N, h->qa, h->dg, h->s, h->sf, h->stream));
            int herr = 0;
            DM_CUDA(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
            DM_CUDA(cudaStreamSynchronize(h->stream));
            if (herr) return fail(DM_ETIMEOUT, "a bounded wait of the tensor-core degree pass gave up");
            h->stats.degree_path = S.quant ? 2 : 1;
            h->free_group(G_WORK);  // the stream has been synchronised
        } else {
            cudaEvent_t lap = h->lap_begin(h->stream);
            DM_CUDA(dm_launch_degree_pass_centered(h->Xs, nrm, nmax, N, d, nullptr, h->q, h->stream));
            DM_CUDA(dm_launch_finish_degrees(N, alpha, h->q, h->qa, h->qaf, h->stream));
            DM_CUDA(dm_launch_degree_pass_centered(h->Xs, nrm, nmax, N, d, h->qaf, h->dg, h->stream));
            h->lap_end(h->stream, lap, &h->stats.ms_degrees);
            DM_CUDA(dm_launch_finish_scaling(N, h->qa, h->dg, h->s, h->sf, h->stream));
            h->stats.degree_path = 0;
        }
        DM_CUDA(cudaEventRecord(h->cr_b, h->stream));
        h->cr_pending = true;
        DM_CUDA(cudaGetLastError());
        return DM_OK;
    }();
    if (rc != DM_OK) {
        delete h;
        return rc;
    }
    *out = h;
    return DM_OK;
}

int dm_destroy(dm_handle h) {
    if (!h) return fail(DM_EINVAL, "handle is NULL");
    set_device(h);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->tstream) cudaStreamSynchronize(h->tstream);
    delete h;
    return DM_OK;
}

int dm_compress(dm_handle h, double tol, int32_t leaf_size, int32_t max_rank) {
    if (!h) return fail(DM_EINVAL, "handle is NULL");
    if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(DM_EINVAL, "tol must be finite and >= 0");
    if (leaf_size < 1) return fail(DM_EINVAL, "leaf_size must be >= 1");
    if (max_rank < 1) return fail(DM_EINVAL, "max_rank must be >= 1");
    DM_CHECK(set_device(h));
    const int L = dm_depth_for(h->N, leaf_size);
    if (L > 20) return fail(DM_EINVAL, "tree of depth %d (leaf_size %d) exceeds 2^20 leaves", L, leaf_size);
    if (((int64_t)1 << L) > h->N) return fail(DM_EINVAL, "leaf_size %d too small for N=%lld", leaf_size, (long long)h->N);
    if (max_rank > 256) return fail(DM_EINVAL, "max_rank must be <= 256");
    if (((h->N + ((int64_t)1 << L) - 1) >> L) > dm_skel_max_candidates())
        return fail(DM_EINVAL, "leaves of more than %d points are not supported", dm_skel_max_candidates());
    DM_CHECK(alloc_structure(h, L, max_rank));
    h->tol = tol;
    resolve_near_mode(h);
    const int nleaves = 1 << L;
    // ---- tree, on its own high-priority stream: it waits only for the points and eps (the
    // event before the degree passes), so it runs while those passes may still be in flight
    float ms_tree = 0;
    if (!h->cfg.shared_device) DM_CHECK(ensure_tree_stream(h));
    {
        const bool side = h->tstream != nullptr;
        const cudaStream_t ts = side ? h->tstream : h->stream;
        if (side && h->ev_pre) DM_CUDA(cudaStreamWaitEvent(ts, h->ev_pre, 0));
        PhaseTimer t(ts);
        int32_t *pa = nullptr, *pb = nullptr;
        DM_CHECK(h->alloc(&pa, (size_t)h->N, G_STRUCT, ts));
        DM_CHECK(h->alloc(&pb, (size_t)h->N, G_STRUCT, ts));
        // identity permutation: every node starts in increasing original index
        std::vector<int32_t> ident((size_t)h->N);
        for (int64_t i = 0; i < h->N; ++i) ident[(size_t)i] = (int32_t)i;
        DM_CUDA(cudaMemcpyAsync(pa, ident.data(), sizeof(int32_t) * (size_t)h->N, cudaMemcpyHostToDevice, ts));
        DmTreeWork w{};
        const size_t nitems = dm_tree_items_bound(h->N, L) + 1;
        w.max_items = (int)nitems;
        DM_CHECK(h->alloc(&w.wbuf, (size_t)h->N, G_WORK, ts));
        DM_CHECK(h->alloc(&w.keys, (size_t)h->N, G_WORK, ts));
        unsigned char *items = nullptr, *c1 = nullptr, *c2 = nullptr;
        DM_CHECK(h->alloc(&items, nitems * dm_tree_item_bytes(), G_WORK, ts));
        DM_CHECK(h->alloc(&c1, nitems * dm_tree_cand_bytes(), G_WORK, ts));
        DM_CHECK(h->alloc(&c2, nitems * dm_tree_cand_bytes(), G_WORK, ts));
        w.items = items;
        w.cand1 = c1;
        w.cand2 = c2;
        // the large levels (nodes above dm_tree_big_node() points) split over many CTAs
        w.max_big = (int)(h->N / dm_tree_big_node()) + 1;
        unsigned char *sel = nullptr;
        DM_CHECK(h->alloc(&sel, (size_t)w.max_big * dm_tree_sel_bytes(), G_WORK, ts));
        DM_CHECK(h->alloc(&w.hist, (size_t)w.max_big * 256, G_WORK, ts));
        unsigned char *icnt = nullptr;
        DM_CHECK(h->alloc(&icnt, nitems * 8, G_WORK, ts));
        if (side && h->cfg.alloc) {
            // a caller allocator's buffers are valid in `stream`'s order only: the tree then
            // waits for everything enqueued there (no overlap with the degree passes)
            DM_CUDA(cudaEventRecord(h->ev_sel, h->stream));
            DM_CUDA(cudaStreamWaitEvent(ts, h->ev_sel, 0));
        }
        w.sel = sel;
        w.icnt = icnt;
        // at high dimension the distance sums read an FP64 copy of the points (freed with the
        // workspace)
        double *X64 = nullptr;
        if (h->d >= kWideMinD) {
            DM_CHECK(h->alloc(&X64, (size_t)h->N * h->d, G_WORK, ts));
            DM_CUDA(dm_launch_widen(h->X, h->N * h->d, X64, ts));
        }
        int32_t *perm = nullptr;
        DM_CUDA(dm_tree_build(h->X, X64, h->N, h->d, h->eps, L, pa, pb, &perm, &w, ts));
        h->perm = perm;
        ms_tree = t.stop();  // the host waits for the tree only; the degree passes may still run
        h->free_group(G_WORK);
        if (side) {
            DM_CUDA(cudaEventRecord(h->ev_tree, ts));
            DM_CUDA(cudaStreamWaitEvent(h->stream, h->ev_tree, 0));
        }
    }
    // ---- skeletons (no host wait: the workspace is freed after the next synchronisation, in
    // finish_structure, and the phase is timed by deferred events)
    {
        cudaEvent_t t0 = h->lap_begin(h->stream);
        DM_CUDA(dm_permute_points(h->Xs, h->sf, h->perm, h->N, h->d, h->Xp, h->sp, h->stream));
        DmSkelWork w{};
        w.rmax = 2 * max_rank + 10;
        w.ldr = (int)round_up(w.rmax, 4);
        const size_t smem = dm_skel_smem_bytes(h->cmax, w.rmax, max_rank);
        if (smem > 220 * 1024 || h->cmax > dm_skel_max_candidates())
            return fail(DM_EINVAL, "leaf size (%d) / rank (%d) too large for the skeletonization kernel",
                        h->leaf_max, max_rank);
        DM_CHECK(h->alloc(&w.A, (size_t)nleaves * h->cmax * w.ldr, G_WORK));
        DM_CHECK(h->alloc(&w.R, (size_t)nleaves * max_rank * h->cmax, G_WORK));
        DM_CHECK(h->alloc(&w.Q, (size_t)nleaves * max_rank * w.ldr, G_WORK));
        DM_CUDA(dm_skeletonize(h->Xp, h->sp, h->N, h->d, L, h->perm, tol, max_rank, h->cmax, h->ldp, h->cfg.seed,
                               h->ranks, h->skel, h->P, &w, h->stream));
        h->lap_end(h->stream, t0, &h->stats.ms_skeleton);
    }
    {
        cudaEvent_t t0 = h->lap_begin(h->stream);
        DM_CHECK(finish_structure(h));
        h->lap_end(h->stream, t0, &h->stats.ms_pack);
    }
    h->stats.ms_tree = ms_tree;
    DM_CUDA(cudaGetLastError());
    return DM_OK;
}

int dm_matvec(dm_handle h, const float *x, float *y, int32_t nrhs) {
    if (!h) return fail(DM_EINVAL, "handle is NULL");
    if (!x || !y) return fail(DM_EINVAL, "x or y is NULL");
    if (nrhs < 1) return fail(DM_EINVAL, "nrhs must be >= 1");
    DM_CHECK(set_device(h));
    const int64_t n = h->N * nrhs;
    const bool xd = is_device_ptr(x), yd = is_device_ptr(y);
    const float *dx = x;
    float *dy = y;
    if (!xd || !yd) DM_CHECK(ensure_io(h, n));
    if (!xd) {
        DM_CUDA(cudaMemcpyAsync(h->io_x, x, sizeof(float) * n, cudaMemcpyHostToDevice, h->stream));
        dx = h->io_x;
    }
    if (!yd) dy = h->io_y;
    bool narrow = false;
    if (h->compressed && nrhs >= 2 && nrhs <= 4 && h->cfg.block_precision == DM_PREC_FP32)
        DM_CHECK(ensure_nb(h, nrhs, &narrow));
    if (narrow) {
        // 2..4 columns through the single-vector form's three chained launches
        DM_CUDA(dm_hmatvec_nb(h->hmat(), h->nbt, nrhs, dx, h->N, dy, h->N, false, h->stream));
    } else if (h->compressed && nrhs >= 2) {
        // block H-matvec: every stored operand is read once per panel of columns
        const bool tc = h->cfg.block_precision != DM_PREC_FP32 && h->near_mode == DM_NEAR_CACHED;
        if (tc && !dm_tc_available()) return fail(DM_ECUDA, "the driver does not provide cuTensorMapEncodeTiled");
        const int near_prec = tc ? h->cfg.block_precision : DM_PREC_FP32;
        const int panel = tc ? kBlockPanelTc : kBlockPanelFp32;
        const int nbp = nrhs < panel ? nrhs : panel;
        DM_CHECK(ensure_block(h, nbp));
        const DmHmat H = h->hmat();
        for (int c0 = 0; c0 < nrhs; c0 += panel) {
            const int nb = nrhs - c0 < panel ? nrhs - c0 : panel;
            DM_CUDA(dm_hmatvec_block(H, h->near_mode, near_prec, h->blk, nb, dx + (size_t)c0 * h->N, h->N, h->perm,
                                     false, dy + (size_t)c0 * h->N, h->N, DM_BLK_ORIGINAL, h->stream));
        }
        if (tc) {
            int err = 0;
            DM_CUDA(cudaMemcpyAsync(&err, h->herr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
            DM_CUDA(cudaStreamSynchronize(h->stream));
            if (err) {
                DM_CUDA(cudaMemsetAsync(h->herr, 0, sizeof(int), h->stream));
                DM_CUDA(cudaStreamSynchronize(h->stream));
                return fail(DM_ETIMEOUT, "a bounded wait of the tensor-core near field gave up");
            }
        }
    } else {
        for (int c = 0; c < nrhs; ++c) {
            const float *xc = dx + (size_t)c * h->N;
            float *yc = dy + (size_t)c * h->N;
            if (h->compressed) DM_CUDA(dm_hmatvec(h->hmat(), h->near_mode, xc, yc, false, h->stream));
            else DM_CUDA(dm_launch_dense_matvec_ws(h->Xs, h->sf, h->N, h->d, xc, yc, h->tmpw, h->acc, h->stream));
        }
    }
    if (!yd) DM_CUDA(cudaMemcpyAsync(y, dy, sizeof(float) * n, cudaMemcpyDeviceToHost, h->stream));
    DM_CUDA(cudaStreamSynchronize(h->stream));
    return DM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Single-vector Lanczos of many compressed handles advanced together: every step of every
// active problem runs in the same five launches (two H-matvec launches, three Gram-Schmidt
// passes), each problem at its own step index, so problems join and leave between steps.
// Convergence checks (Ritz values of T_m) run on each problem's own schedule; the checks due
// after a step share one launch, and their results are read one step later, while the next
// step runs, so the host never drains the stream. A problem that converged therefore takes
// one more step before it leaves (harmless: its Ritz vectors use the first m columns); one
// at m_max leaves the step list at once and is finished when its check is read. Finished
// problems are handed out one call later still, once the step after their Ritz-vector
// launches is queued, so that waiting for their vectors does not idle the GPU either.
// ---------------------------------------------------------------------------------------
namespace {
enum SlotState { kFree = 0, kStepping = 1, kLeaving = 2 };
}

struct DmBatchSolver {
    int device = 0;
    cudaStream_t st = nullptr;
    // per slot (host); a slot is reused after its problem is finished
    std::vector<dm_ctx *> h;
    std::vector<int> k, cap, jh, first, every, state, sblk;
    std::vector<size_t> shm;
    std::vector<void *> tag;
    std::vector<DmBatchShape> shape;
    std::vector<DmChainProblem> cp;
    std::vector<DmLanczosProblem> lp;
    std::vector<int> act;       // stepping slots, in join order
    std::vector<int> starting;  // slots whose start vector is drawn before the next step
    int in_use = 0;
    int64_t gstep = 0;  // steps launched by this solver
    bool dirty = true;
    // launch geometry of the stepping problems
    int n_up = 0, n_sw = 0, n_nr = 0, n_st = 0, n_start = 0, n_smap = 0;
    size_t smem_up = 0, smem_sw = 0, smem_nr = 0, smem_step = 0;
    // descriptors and launch maps in one device blob, uploaded from one of two pinned
    // staging buffers (each reused only after its last upload has completed)
    unsigned char *blob = nullptr, *stage[2] = {nullptr, nullptr};
    size_t c_blob = 0, c_stage[2] = {0, 0};
    cudaEvent_t ev_stage[2] = {nullptr, nullptr};
    int cur = 0;
    const DmChainProblem *dcp = nullptr;
    const DmLanczosProblem *dlp = nullptr;
    const int2 *dup = nullptr, *dsw = nullptr, *dnr = nullptr;
    const int4 *dst = nullptr;
    const DmStart *dss = nullptr;
    const int2 *dsm = nullptr;
    // per-slot device state: step counter jv and the arrival counter of its last pass
    int *djv = nullptr;
    unsigned *darr = nullptr;
    size_t c_slots = 0;
    // the check in flight: slots and their m; results land in pinned hres
    std::vector<int> pend, pend_m;
    int pend_khi = 1;
    int *hdue = nullptr, *ddue = nullptr;
    double *hres = nullptr, *dres = nullptr;
    cudaEvent_t ev_chk = nullptr;
    // Ritz-vector launches of the problems a check finished: descriptors and block map in
    // one device buffer, staged in pinned memory (reused once its last upload completed)
    unsigned char *fstage = nullptr, *fblob = nullptr;
    size_t c_fstage = 0, c_fblob = 0;
    cudaEvent_t ev_fstage = nullptr;
    // problems finished at the last call, handed out at the next (ready: ev_done[par])
    std::vector<DmBatchDone> fin;
    cudaEvent_t ev_done[2] = {nullptr, nullptr};
    int par = 0;

    ~DmBatchSolver() {
        if (st) cudaStreamSynchronize(st);
        void *ds[] = {blob, djv, darr, ddue, dres, fblob};
        for (void *q : ds)
            if (q) cudaFree(q);
        void *hs[] = {stage[0], stage[1], hdue, hres, fstage};
        for (void *q : hs)
            if (q) cudaFreeHost(q);
        for (cudaEvent_t e : {ev_stage[0], ev_stage[1], ev_chk, ev_done[0], ev_done[1], ev_fstage})
            if (e) cudaEventDestroy(e);
    }
};

namespace {

// per-slot arrays for `want` slots: the step counters (kept), the check lists and results
int batch_slots(DmBatchSolver &B, size_t want) {
    if (want <= B.c_slots) return DM_OK;
    size_t n = B.c_slots ? B.c_slots : 64;
    while (n < want) n *= 2;
    const size_t per = (size_t)(2 * dm_lanczos_kmax() + 1);  // theta, resid (k each) and beta
    DM_CUDA(cudaStreamSynchronize(B.st));
    int *jv = nullptr, *due = nullptr, *hdue = nullptr;
    unsigned *arr = nullptr;
    double *res = nullptr, *hres = nullptr;
    if (cudaMalloc(reinterpret_cast<void **>(&jv), sizeof(int) * n) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void **>(&arr), sizeof(unsigned) * n) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void **>(&due), sizeof(int) * n) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void **>(&res), sizeof(double) * n * per) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void **>(&hdue), sizeof(int) * n) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void **>(&hres), sizeof(double) * n * per) != cudaSuccess) {
        cudaGetLastError();
        void *ds[] = {jv, arr, due, res};
        for (void *q : ds)
            if (q) cudaFree(q);
        if (hdue) cudaFreeHost(hdue);
        if (hres) cudaFreeHost(hres);
        return fail(DM_ENOMEM, "batched eigensolver: allocation of %zu slots failed", n);
    }
    DM_CUDA(cudaMemsetAsync(arr, 0, sizeof(unsigned) * n, B.st));
    if (B.djv) {
        DM_CUDA(cudaMemcpyAsync(jv, B.djv, sizeof(int) * B.c_slots, cudaMemcpyDeviceToDevice, B.st));
        DM_CUDA(cudaMemcpyAsync(arr, B.darr, sizeof(unsigned) * B.c_slots, cudaMemcpyDeviceToDevice, B.st));
        DM_CUDA(cudaStreamSynchronize(B.st));
    }
    void *ds[] = {B.djv, B.darr, B.ddue, B.dres};
    for (void *q : ds)
        if (q) cudaFree(q);
    if (B.hdue) cudaFreeHost(B.hdue);
    if (B.hres) cudaFreeHost(B.hres);
    B.djv = jv;
    B.darr = arr;
    B.ddue = due;
    B.dres = res;
    B.hdue = hdue;
    B.hres = hres;
    B.c_slots = n;
    return DM_OK;
}

inline size_t a16(size_t x) { return (x + 15) & ~size_t(15); }

// descriptors of every slot and the launch maps of the stepping problems (the climbs, the
// near items and the Gram-Schmidt blocks of each), plus the start vectors of those joining
int batch_rebuild(DmBatchSolver &B) {
    B.n_up = B.n_sw = B.n_nr = B.n_st = 0;
    B.smem_up = B.smem_sw = B.smem_nr = B.smem_step = 0;
    for (int p : B.act) {
        B.n_up += B.shape[p].climbs;
        B.n_sw += B.shape[p].sweeps;
        B.smem_sw = B.shape[p].smem_sweep > B.smem_sw ? B.shape[p].smem_sweep : B.smem_sw;
        B.n_nr += B.shape[p].items;
        B.n_st += B.sblk[p];
        B.smem_up = B.shape[p].smem_up > B.smem_up ? B.shape[p].smem_up : B.smem_up;
        B.smem_nr = B.shape[p].smem_near > B.smem_nr ? B.shape[p].smem_near : B.smem_nr;
        B.smem_step = B.shm[p] > B.smem_step ? B.shm[p] : B.smem_step;
    }
    B.n_start = (int)B.starting.size();
    B.n_smap = 0;
    for (int p : B.starting) B.n_smap += dm_finish_blocks(B.h[p]->lz.N);
    const size_t ns = B.cp.size();
    const size_t o_cp = 0, o_lp = a16(o_cp + sizeof(DmChainProblem) * ns);
    const size_t o_up = a16(o_lp + sizeof(DmLanczosProblem) * ns);
    const size_t o_sw = a16(o_up + sizeof(int2) * (size_t)B.n_up);
    const size_t o_nr = a16(o_sw + sizeof(int2) * (size_t)B.n_sw);
    const size_t o_st = a16(o_nr + sizeof(int2) * (size_t)B.n_nr);
    const size_t o_ss = a16(o_st + sizeof(int4) * (size_t)B.n_st);
    const size_t o_sm = a16(o_ss + sizeof(DmStart) * (size_t)B.n_start);
    const size_t bytes = a16(o_sm + sizeof(int2) * (size_t)B.n_smap);
    const int c = B.cur;
    if (B.ev_stage[c]) DM_CUDA(cudaEventSynchronize(B.ev_stage[c]));
    else DM_CUDA(cudaEventCreateWithFlags(&B.ev_stage[c], cudaEventDisableTiming));
    if (bytes > B.c_stage[c]) {
        if (B.stage[c]) cudaFreeHost(B.stage[c]);
        B.stage[c] = nullptr;
        B.c_stage[c] = 0;
        if (cudaMallocHost(reinterpret_cast<void **>(&B.stage[c]), 2 * bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(DM_ENOMEM, "batched eigensolver: pinned staging of %zu bytes failed", 2 * bytes);
        }
        B.c_stage[c] = 2 * bytes;
    }
    if (bytes > B.c_blob) {
        // kernels still queued may read the old blob
        DM_CUDA(cudaStreamSynchronize(B.st));
        if (B.blob) cudaFree(B.blob);
        B.blob = nullptr;
        B.c_blob = 0;
        if (cudaMalloc(reinterpret_cast<void **>(&B.blob), 2 * bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(DM_ENOMEM, "batched eigensolver: cudaMalloc of %zu bytes failed", 2 * bytes);
        }
        B.c_blob = 2 * bytes;
    }
    unsigned char *hs = B.stage[c];
    std::memcpy(hs + o_cp, B.cp.data(), sizeof(DmChainProblem) * ns);
    std::memcpy(hs + o_lp, B.lp.data(), sizeof(DmLanczosProblem) * ns);
    int2 *up = reinterpret_cast<int2 *>(hs + o_up);
    int2 *sw = reinterpret_cast<int2 *>(hs + o_sw);
    int2 *nr = reinterpret_cast<int2 *>(hs + o_nr);
    int4 *sp = reinterpret_cast<int4 *>(hs + o_st);
    // the deepest trees first: their climbs and sweeps are the longest chains
    std::vector<int> order(B.act);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return B.cp[a].H.L > B.cp[b].H.L; });
    for (int p : order) {
        for (int b = 0; b < B.shape[p].climbs; ++b) *up++ = make_int2(p, b);
        for (int b = 0; b < B.shape[p].sweeps; ++b) *sw++ = make_int2(p, b);
        for (int b = 0; b < B.shape[p].items; ++b) *nr++ = make_int2(p, b);
        for (int b = 0; b < B.sblk[p]; ++b) *sp++ = make_int4(p, b, B.sblk[p], 0);
    }
    DmStart *ss = reinterpret_cast<DmStart *>(hs + o_ss);
    int2 *sm = reinterpret_cast<int2 *>(hs + o_sm);
    for (int i = 0; i < B.n_start; ++i) {
        const int p = B.starting[(size_t)i];
        const dm_ctx *h = B.h[p];
        const DmLanczos &Lz = h->lz;
        DmStart d{};
        d.perm = h->perm;
        d.N = Lz.N;
        d.key = dm_start_key(h->cfg.seed);
        d.z = Lz.z;
        d.V = Lz.V;
        d.nrm2 = Lz.nrm2;
        d.h = Lz.h;
        d.hlen = 2 * B.lp[p].hstride;
        d.jv = B.djv + p;
        ss[i] = d;
        const int nb = dm_finish_blocks(Lz.N);
        for (int b = 0; b < nb; ++b) *sm++ = make_int2(i, b);
    }
    // stream-ordered: kernels queued before still read the previous contents
    DM_CUDA(cudaMemcpyAsync(B.blob, hs, bytes, cudaMemcpyHostToDevice, B.st));
    DM_CUDA(cudaEventRecord(B.ev_stage[c], B.st));
    B.cur ^= 1;
    B.dcp = reinterpret_cast<const DmChainProblem *>(B.blob + o_cp);
    B.dlp = reinterpret_cast<const DmLanczosProblem *>(B.blob + o_lp);
    B.dup = reinterpret_cast<const int2 *>(B.blob + o_up);
    B.dsw = reinterpret_cast<const int2 *>(B.blob + o_sw);
    B.dnr = reinterpret_cast<const int2 *>(B.blob + o_nr);
    B.dst = reinterpret_cast<const int4 *>(B.blob + o_st);
    B.dss = reinterpret_cast<const DmStart *>(B.blob + o_ss);
    B.dsm = reinterpret_cast<const int2 *>(B.blob + o_sm);
    B.dirty = false;
    return DM_OK;
}

// Ritz vectors of the finished problems F (one set of launches for all of them)
int batch_finish(DmBatchSolver &B, const std::vector<DmFinish> &F) {
    if (F.empty()) return DM_OK;
    int m_hi = 1, k_hi = 1;
    std::vector<int2> map;
    for (size_t f = 0; f < F.size(); ++f) {
        m_hi = F[f].m > m_hi ? F[f].m : m_hi;
        k_hi = F[f].k > k_hi ? F[f].k : k_hi;
        const int nb = dm_finish_blocks(F[f].N);
        for (int b = 0; b < nb; ++b) map.push_back(make_int2((int)f, b));
    }
    const size_t o_map = a16(sizeof(DmFinish) * F.size());
    const size_t bytes = o_map + sizeof(int2) * map.size();
    if (B.ev_fstage) DM_CUDA(cudaEventSynchronize(B.ev_fstage));
    else DM_CUDA(cudaEventCreateWithFlags(&B.ev_fstage, cudaEventDisableTiming));
    if (bytes > B.c_fstage) {
        if (B.fstage) cudaFreeHost(B.fstage);
        B.fstage = nullptr;
        B.c_fstage = 0;
        if (cudaMallocHost(reinterpret_cast<void **>(&B.fstage), 2 * bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(DM_ENOMEM, "batched eigensolver: pinned staging of %zu bytes failed", 2 * bytes);
        }
        B.c_fstage = 2 * bytes;
    }
    if (bytes > B.c_fblob) {
        DM_CUDA(cudaStreamSynchronize(B.st));  // earlier launches may still read the old buffer
        if (B.fblob) cudaFree(B.fblob);
        B.fblob = nullptr;
        B.c_fblob = 0;
        if (cudaMalloc(reinterpret_cast<void **>(&B.fblob), 2 * bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(DM_ENOMEM, "batched eigensolver: cudaMalloc of %zu bytes failed", 2 * bytes);
        }
        B.c_fblob = 2 * bytes;
    }
    std::memcpy(B.fstage, F.data(), sizeof(DmFinish) * F.size());
    std::memcpy(B.fstage + o_map, map.data(), sizeof(int2) * map.size());
    DM_CUDA(cudaMemcpyAsync(B.fblob, B.fstage, bytes, cudaMemcpyHostToDevice, B.st));
    DM_CUDA(cudaEventRecord(B.ev_fstage, B.st));
    DM_CUDA(dm_lanczos_finish_batch(reinterpret_cast<const DmFinish *>(B.fblob), (int)F.size(),
                                    reinterpret_cast<const int2 *>(B.fblob + o_map), (int)map.size(), m_hi, k_hi,
                                    B.st));
    return DM_OK;
}

// read the check in flight and finish the problems it decides: their Ritz-vector launches are
// queued and they wait in B.fin for the next call
int batch_collect(DmBatchSolver &B) {
    if (B.pend.empty()) return DM_OK;
    DM_CUDA(cudaEventSynchronize(B.ev_chk));
    const int nd = (int)B.pend.size(), khi = B.pend_khi;
    const double *hth = B.hres, *hrs = hth + (size_t)nd * khi, *hbt = hrs + (size_t)nd * khi;
    bool left = false;
    std::vector<DmFinish> F;
    for (int i = 0; i < nd; ++i) {
        const int p = B.pend[i], m = B.pend_m[i];
        dm_ctx *h = B.h[p];
        const int k = B.k[p];
        const double *tp = hth + (size_t)i * khi, *rp = hrs + (size_t)i * khi;
        const double scale = std::fabs(tp[0]) > 0 ? std::fabs(tp[0]) : 1.0;
        bool ok = true;
        for (int j = 0; j < k; ++j)
            if (!(rp[j] <= h->cfg.conv_tol * scale)) ok = false;
        const bool breakdown = hbt[i] <= 1e-12 * scale;
        if (!(ok || breakdown || B.state[p] == kLeaving)) continue;
        // finished after m steps: Ritz vectors in original point order from the first m basis
        // columns (Lz.theta holds this check's values; a later step does not touch them)
        const DmLanczos &Lz = h->lz;
        DmFinish f{};
        f.alpha = Lz.alpha;
        f.beta = Lz.beta;
        f.theta = Lz.theta;
        f.Y = Lz.Y;
        f.twork = Lz.twork;
        f.colsum = Lz.colsum;
        f.Yf = Lz.Yf;
        f.phi = Lz.phi;
        f.evecs = h->evecs;
        f.V = Lz.V;
        f.ldv = Lz.ldv;
        f.N = Lz.N;
        f.perm = h->perm;
        f.best = Lz.best;
        f.neg = Lz.neg;
        f.ldy = Lz.m_max;
        f.m = m;
        f.k = k;
        F.push_back(f);
        DmBatchDone d;
        d.h = h;
        d.tag = B.tag[p];
        d.status = (ok || breakdown) ? DM_OK : DM_ENOCONV;
        d.iters = m;
        d.k = k;
        d.theta.assign(tp, tp + k);
        d.evecs = h->evecs;
        B.fin.push_back(std::move(d));
        h->last_k = k;
        h->stats.lanczos_iters = m;
        h->stats.converged = (ok || breakdown) ? 1 : 0;
        h->stats.matvec_calls = 0;
        h->stats.ms_matvec = 0.f;
        if (B.state[p] == kStepping) B.dirty = true;
        B.state[p] = kFree;
        B.h[p] = nullptr;
        --B.in_use;
        left = true;
    }
    B.pend.clear();
    B.pend_m.clear();
    DM_CHECK(batch_finish(B, F));
    if (left) {
        std::vector<int> keep;
        for (int p : B.act)
            if (B.state[p] == kStepping) keep.push_back(p);
        B.act.swap(keep);
        cudaEvent_t &e = B.ev_done[B.par];
        if (!e) DM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        DM_CUDA(cudaEventRecord(e, B.st));
        for (DmBatchDone &d : B.fin) d.ready = e;
    }
    return DM_OK;
}

}  // namespace

DmBatchSolver *dm_batch_create(int device, cudaStream_t st) {
    DmBatchSolver *B = new DmBatchSolver();
    B->device = device;
    B->st = st;
    return B;
}

void dm_batch_destroy(DmBatchSolver *B) { delete B; }

int dm_batch_active(const DmBatchSolver *B) { return B ? B->in_use + (int)B->fin.size() : 0; }

int dm_batch_reserve(DmBatchSolver *B, int n) {
    if (!B || n < 0) return fail(DM_EINVAL, "batched eigensolver: bad reserve");
    return batch_slots(*B, (size_t)n);
}

int dm_batch_prepare(dm_handle h, cudaEvent_t *ready) {
    if (!h || !ready) return fail(DM_EINVAL, "batched eigensolver: NULL argument");
    if (!h->compressed) return fail(DM_ESTATE, "batched eigensolver: handle not compressed");
    DM_CHECK(set_device(h));
    DM_CHECK(ensure_lanczos(h));
    *ready = nullptr;
    DM_CUDA(cudaEventCreateWithFlags(ready, cudaEventDisableTiming));
    DM_CUDA(cudaEventRecord(*ready, h->stream));
    return DM_OK;
}

int dm_batch_add(DmBatchSolver *B, dm_handle h, int k, void *tag, cudaEvent_t ready, cudaStream_t adopt) {
    if (!B || !h) return fail(DM_EINVAL, "batched eigensolver: NULL argument");
    if (!h->compressed || !h->lz_ready) return fail(DM_ESTATE, "batched eigensolver: handle not prepared");
    if (k < 1 || k > dm_lanczos_kmax() || k >= h->N || k > h->cfg.m_max)
        return fail(DM_EINVAL, "batched eigensolver: k out of range");
    if (h->device != B->device) return fail(DM_EINVAL, "batched eigensolver: handle on another device");
    int slot = -1;
    for (size_t i = 0; i < B->state.size(); ++i)
        if (B->state[i] == kFree) {
            slot = (int)i;
            break;
        }
    if (slot < 0) {
        slot = (int)B->state.size();
        DM_CHECK(batch_slots(*B, (size_t)slot + 1));
        B->h.push_back(nullptr);
        B->k.push_back(0);
        B->cap.push_back(0);
        B->jh.push_back(0);
        B->first.push_back(0);
        B->every.push_back(1);
        B->state.push_back(kFree);
        B->sblk.push_back(1);
        B->shm.push_back(0);
        B->tag.push_back(nullptr);
        B->shape.push_back(DmBatchShape{});
        B->cp.push_back(DmChainProblem{});
        B->lp.push_back(DmLanczosProblem{});
    }
    // everything queued for the handle before it was prepared runs first
    if (ready) DM_CUDA(cudaStreamWaitEvent(B->st, ready, 0));
    // the handle's own stream: idle from here on (the solver works on its own stream)
    if (adopt) h->stream = adopt;
    DmLanczos &Lz = h->lz;
    const DmHmat H = h->hmat();
    const int qt = dm_step_tile_quads(Lz.m_max);
    B->h[slot] = h;
    B->k[slot] = k;
    B->cap[slot] = (int)(h->cfg.m_max < h->N ? h->cfg.m_max : h->N);
    B->jh[slot] = 0;
    B->first[slot] = (5 * k + 3) / 4 + 5;
    B->every[slot] = h->cfg.check_every > 0 ? h->cfg.check_every : 1;
    B->tag[slot] = tag;
    B->shape[slot] = dm_batch_shape(H, h->near_mode);
    B->shm[slot] = dm_step_batch_smem(Lz.m_max);
    DmChainProblem &c = B->cp[slot];
    c.H = H;
    c.x = Lz.V;
    c.xstep = Lz.ldv;
    c.y = Lz.z;
    c.permuted = 1;
    c.near_mode = h->near_mode;
    c.near_rows = B->shape[slot].item_rows;
    c.climb_smem = B->shape[slot].climb_smem;
    c.chain_smem = 0;
    DmLanczosProblem &l = B->lp[slot];
    l.V = Lz.V;
    l.ldv = Lz.ldv;
    l.z = Lz.z;
    l.h = Lz.h;
    l.hstride = dm_lanczos_hstride(Lz.m_max);
    l.alpha = Lz.alpha;
    l.beta = Lz.beta;
    l.m_max = Lz.m_max;
    l.qt = qt;
    l.theta = Lz.theta;
    l.resid = Lz.resid;
    l.k = k;
    const int64_t qn = Lz.ldv >> 2;
    const int nb = (int)((qn + qt - 1) / qt);
    B->sblk[slot] = nb < 1 ? 1 : (nb > 304 ? 304 : nb);
    B->starting.push_back(slot);  // its start vector (and step counter) set with the others joining now
    B->state[slot] = kStepping;
    ++B->in_use;
    B->act.push_back(slot);
    B->dirty = true;
    return DM_OK;
}

int dm_batch_step(DmBatchSolver *B, std::vector<DmBatchDone> &done) {
    if (!B) return fail(DM_EINVAL, "batched eigensolver: NULL solver");
    const cudaStream_t st = B->st;
    if (!B->act.empty()) {
        if (B->dirty) DM_CHECK(batch_rebuild(*B));
        if (B->n_start > 0) {
            DM_CUDA(dm_lanczos_start_batch(B->dss, B->n_start, B->dsm, B->n_smap, st));
            B->starting.clear();
            B->n_start = 0;
        }
        DM_CUDA(dm_hmatvec_batch(B->dcp, B->dup, B->n_up, B->smem_up, B->dsw, B->n_sw, B->smem_sw, B->dnr, B->n_nr,
                                 B->smem_nr, B->djv, st));
        DM_CUDA(dm_lanczos_step_batch(B->dlp, B->dst, B->n_st, B->djv, B->darr, B->smem_step, st));
    }
    // the problems finished at the last call: their vectors come before this step
    for (DmBatchDone &d : B->fin) done.push_back(std::move(d));
    B->fin.clear();
    B->par ^= 1;
    // the previous step's check has been computed while this step was queued: read it
    DM_CHECK(batch_collect(*B));
    ++B->gstep;
    // checks due after this step
    std::vector<int> due;
    int m_hi = 0, k_hi = 1;
    bool leaving = false;
    for (int p : B->act) {
        if (B->state[p] != kStepping) continue;
        const int m = ++B->jh[p];
        const bool at_cap = m >= B->cap[p];
        // checks on the solver's own step count modulo check_every, so that problems joining
        // at different steps are checked in the same launches (fewer Ritz launches per step)
        if ((m >= B->first[p] && B->gstep % B->every[p] == 0) || at_cap) {
            due.push_back(p);
            m_hi = m > m_hi ? m : m_hi;
            k_hi = B->k[p] > k_hi ? B->k[p] : k_hi;
        }
        if (at_cap) {
            // no room for another basis vector: off the step list now, finished by its check
            B->state[p] = kLeaving;
            leaving = true;
        }
    }
    if (leaving) {
        std::vector<int> keep;
        for (int p : B->act)
            if (B->state[p] == kStepping) keep.push_back(p);
        B->act.swap(keep);
        B->dirty = true;
    }
    if (due.empty()) return DM_OK;
    const int nd = (int)due.size();
    for (int i = 0; i < nd; ++i) B->hdue[i] = due[i];
    double *th = B->dres, *rs = th + (size_t)nd * k_hi, *bt = rs + (size_t)nd * k_hi;
    if (!B->ev_chk) DM_CUDA(cudaEventCreateWithFlags(&B->ev_chk, cudaEventDisableTiming));
    DM_CUDA(cudaMemcpyAsync(B->ddue, B->hdue, sizeof(int) * nd, cudaMemcpyHostToDevice, st));
    DM_CUDA(dm_lanczos_ritz_batch(B->dlp, B->ddue, nd, B->djv, m_hi, k_hi, th, rs, bt, st));
    DM_CUDA(cudaMemcpyAsync(B->hres, B->dres, sizeof(double) * (size_t)nd * (2 * k_hi + 1), cudaMemcpyDeviceToHost,
                            st));
    DM_CUDA(cudaEventRecord(B->ev_chk, st));
    B->pend = due;
    B->pend_m.clear();
    for (int p : due) B->pend_m.push_back(B->jh[p]);
    B->pend_khi = k_hi;
    return DM_OK;
}

namespace {

// idle batched solvers kept per device between dm_eigs_batch calls: their device, pinned and
// slot arrays are allocated once rather than per call
std::mutex g_batch_mu;
std::vector<DmBatchSolver *> g_batch_pool;

struct BatchLease {
    DmBatchSolver *B = nullptr;
    BatchLease(int device, cudaStream_t st) {
        {
            std::lock_guard<std::mutex> lk(g_batch_mu);
            for (size_t i = 0; i < g_batch_pool.size(); ++i)
                if (g_batch_pool[i]->device == device) {
                    B = g_batch_pool[i];
                    g_batch_pool.erase(g_batch_pool.begin() + (long)i);
                    break;
                }
        }
        if (B) {
            B->st = st;  // idle and synchronised when it was returned to the pool
        } else {
            B = dm_batch_create(device, st);
        }
    }
    ~BatchLease() {
        if (!B) return;
        if (dm_batch_active(B) == 0 && B->act.empty() && B->pend.empty()) {
            cudaStreamSynchronize(B->st);
            B->st = nullptr;  // the caller's stream may be destroyed with its handle
            std::lock_guard<std::mutex> lk(g_batch_mu);
            g_batch_pool.push_back(B);
        } else {
            dm_batch_destroy(B);  // left mid-solve by an error: not reusable
        }
    }
    DmBatchSolver *get() const { return B; }
};

}  // namespace

extern "C" {

int dm_eigs_batch(dm_handle *hs, int32_t count, int32_t k, double *evals, float **evecs, int32_t *status) {
    if (!hs || !evals) return fail(DM_EINVAL, "dm_eigs_batch: NULL handles or evals");
    if (count < 1) return fail(DM_EINVAL, "dm_eigs_batch: count must be >= 1");
    if (k < 1 || k > dm_lanczos_kmax()) return fail(DM_EINVAL, "dm_eigs_batch: k must be in [1, %d]", dm_lanczos_kmax());
    for (int i = 0; i < count; ++i) {
        dm_ctx *h = hs[i];
        if (!h) return fail(DM_EINVAL, "dm_eigs_batch: handle %d is NULL", i);
        if (!h->compressed) return fail(DM_ESTATE, "dm_eigs_batch: handle %d is not compressed", i);
        if (k >= h->N || k > h->cfg.m_max) return fail(DM_EINVAL, "dm_eigs_batch: k too large for handle %d", i);
        if (h->device != hs[0]->device) return fail(DM_EINVAL, "dm_eigs_batch: handles on different devices");
        for (int j = 0; j < i; ++j)
            if (hs[j] == h) return fail(DM_EINVAL, "dm_eigs_batch: handle %d appears twice", i);
    }
    DM_CHECK(set_device(hs[0]));
    const cudaStream_t st = hs[0]->stream;
    // an idle solver of this device from the pool (its buffers grown by earlier calls), else a new one
    BatchLease B(hs[0]->device, st);
    if (!B.get()) return fail(DM_ENOMEM, "dm_eigs_batch: no batched solver");
    DM_CHECK(dm_batch_reserve(B.get(), count));
    PhaseTimer t(st);
    for (int i = 0; i < count; ++i) {
        cudaEvent_t ready = nullptr;
        int e = dm_batch_prepare(hs[i], &ready);
        if (e == DM_OK) e = dm_batch_add(B.get(), hs[i], k, reinterpret_cast<void *>((intptr_t)i), ready, nullptr);
        if (ready) cudaEventDestroy(ready);
        DM_CHECK(e);
    }
    std::vector<DmBatchDone> done;
    while (dm_batch_active(B.get()) > 0) DM_CHECK(dm_batch_step(B.get(), done));
    DM_CUDA(cudaStreamSynchronize(st));
    const float ms = t.stop();
    std::vector<double> ev_all((size_t)count * k, 0.0);
    std::vector<int> conv(count, 0);
    for (const DmBatchDone &d : done) {
        const int p = (int)reinterpret_cast<intptr_t>(d.tag);
        std::copy(d.theta.begin(), d.theta.end(), ev_all.begin() + (size_t)p * k);
        conv[p] = d.status == DM_OK;
    }
    if (is_device_ptr(evals))
        DM_CUDA(cudaMemcpy(evals, ev_all.data(), sizeof(double) * ev_all.size(), cudaMemcpyHostToDevice));
    else
        std::copy(ev_all.begin(), ev_all.end(), evals);
    bool all_conv = true;
    for (int p = 0; p < count; ++p) {
        dm_ctx *h = hs[p];
        if (evecs && evecs[p]) DM_CHECK(copy_out(h, evecs[p], h->evecs, sizeof(float) * (size_t)k * h->N));
        if (status) status[p] = conv[p] ? DM_OK : DM_ENOCONV;
        h->stats.ms_eigs = ms;
        if (!conv[p]) all_conv = false;
    }
    for (int p = 0; p < count; ++p) DM_CUDA(cudaStreamSynchronize(hs[p]->stream));
    return all_conv ? DM_OK : fail(DM_ENOCONV, "dm_eigs_batch: some handles did not converge within m_max");
}

int dm_eigs(dm_handle h, int32_t k, double *evals, float *evecs) {
    if (!h) return fail(DM_EINVAL, "handle is NULL");
    if (!h->compressed) return fail(DM_ESTATE, "dm_eigs before dm_compress");
    if (!evals) return fail(DM_EINVAL, "evals is NULL");
    if (k < 1 || k >= h->N) return fail(DM_EINVAL, "k must be in [1, N)");
    if (k > dm_lanczos_kmax()) return fail(DM_EINVAL, "k must be <= %d", dm_lanczos_kmax());
    if (k > h->cfg.m_max) return fail(DM_EINVAL, "k must be <= m_max");
    DM_CHECK(set_device(h));
    DM_CHECK(ensure_lanczos(h));
    if (h->cfg.block_size >= 2) return eigs_block(h, k, evals, evecs);
    PhaseTimer t(h->stream);
    DmLanczos &Lz = h->lz;
    const DmHmat H = h->hmat();
    int m_cap = h->cfg.m_max;
    if (m_cap > h->N) m_cap = (int)h->N;
    DM_CUDA(dm_lanczos_start(Lz, h->perm, h->cfg.seed, h->stream));
    std::vector<double> th(k), rs(k);
    double bj = 0.0;
    int m = 0;
    bool converged = false, ritz_current = false;
    std::vector<cudaEvent_t> ev_mv;
    const bool prof = h->cfg.profile != 0;
    double *hk = check_staging((size_t)2 * dm_lanczos_kmax() + 1);
    if (!hk) return fail(DM_ENOMEM, "pinned host staging for the convergence checks");
    if (!h->ev_chk) DM_CUDA(cudaEventCreateWithFlags(&h->ev_chk, cudaEventDisableTiming));
    // on a device of its own, a check runs on a second stream while the next step runs on
    // the first; on a shared device it runs in order on the handle's stream
    const bool overlap = h->cfg.shared_device == 0;
    if (overlap && !h->cstream) DM_CUDA(cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking));
    if (overlap && !h->ev_step) DM_CUDA(cudaEventCreateWithFlags(&h->ev_step, cudaEventDisableTiming));
    // one Lanczos step j: the H-matvec of basis vector j, then its orthogonalisation
    auto launch_step = [&](int j) -> int {
        if (prof) {
            cudaEvent_t e0, e1;
            DM_CUDA(cudaEventCreate(&e0));
            DM_CUDA(cudaEventCreate(&e1));
            ev_mv.push_back(e0);
            ev_mv.push_back(e1);
            DM_CUDA(cudaEventRecord(e0, h->stream));
        }
        DM_CUDA(dm_hmatvec(H, h->near_mode, Lz.V + (size_t)j * Lz.ldv, Lz.z, true, h->stream));
        if (prof) DM_CUDA(cudaEventRecord(ev_mv.back(), h->stream));
        DM_CUDA(dm_lanczos_orth(Lz, j, h->cfg.shared_device != 0, h->stream));
        return DM_OK;
    };
    int launched = 0;  // steps enqueued so far
    for (int j = 0; j < m_cap; ++j) {
        if (j >= launched) {
            DM_CHECK(launch_step(j));
            launched = j + 1;
        }
        m = j + 1;
        ritz_current = false;
        const bool last = (m == m_cap);
        // convergence checks from m = ceil(5k/4) + 5 on (the wanted pairs rarely converge
        // earlier; 32 steps for k = 20 on the 100k s-curve), then every check_every steps: each
        // check is an FP64 tridiagonal eigensolve whose results the host reads back. With a
        // device of its own, the check runs on the second stream after step j while step
        // j + 1 is already queued on the first, so neither the check nor the host's wait holds
        // up the Lanczos steps; when the check converges, that step's results (basis vector
        // m + 1, alpha_m, beta_m) are never read. At this point the last step queued is j.
        const int first0 = (5 * k + 3) / 4 + 5 > k + 4 ? (5 * k + 3) / 4 + 5 : k + 4;
        const int first = first0 < m_cap ? first0 : m_cap;
        if (m >= first && ((m - first) % h->cfg.check_every == 0 || last)) {
            cudaStream_t cs = h->stream;
            if (overlap) {
                DM_CUDA(cudaEventRecord(h->ev_step, h->stream));
                DM_CUDA(cudaStreamWaitEvent(h->cstream, h->ev_step, 0));
                cs = h->cstream;
            }
            DM_CUDA(dm_lanczos_ritz(Lz, m, k, h->cfg.conv_tol, cs));
            DM_CUDA(cudaMemcpyAsync(hk, Lz.theta, sizeof(double) * k, cudaMemcpyDeviceToHost, cs));
            DM_CUDA(cudaMemcpyAsync(hk + k, Lz.resid, sizeof(double) * k, cudaMemcpyDeviceToHost, cs));
            DM_CUDA(cudaMemcpyAsync(hk + 2 * k, Lz.beta + j, sizeof(double), cudaMemcpyDeviceToHost, cs));
            DM_CUDA(cudaEventRecord(h->ev_chk, cs));
            if (overlap && !last && launched == j + 1) {
                DM_CHECK(launch_step(j + 1));
                launched = j + 2;
            }
            DM_CUDA(cudaEventSynchronize(h->ev_chk));
            for (int i = 0; i < k; ++i) {
                th[i] = hk[i];
                rs[i] = hk[k + i];
            }
            bj = hk[2 * k];
            ritz_current = true;
            const double scale = std::fabs(th[0]) > 0 ? std::fabs(th[0]) : 1.0;
            bool ok = true;
            for (int i = 0; i < k; ++i)
                if (!(rs[i] <= h->cfg.conv_tol * scale)) ok = false;
            if (ok || bj <= 1e-12 * scale) {
                converged = true;
                break;
            }
        }
    }
    // the vectors below read theta from the last check
    if (overlap) DM_CUDA(cudaStreamWaitEvent(h->stream, h->ev_chk, 0));
    if (!ritz_current) {
        DM_CUDA(dm_lanczos_ritz(Lz, m, k, h->cfg.conv_tol, h->stream));
        DM_CUDA(cudaMemcpyAsync(th.data(), Lz.theta, sizeof(double) * k, cudaMemcpyDeviceToHost, h->stream));
    }
    DM_CUDA(dm_lanczos_vectors(Lz, m, k, h->perm, h->evecs, h->stream));
    DM_CUDA(cudaStreamSynchronize(h->stream));
    {
        int err = 0;
        DM_CUDA(cudaMemcpyAsync(&err, Lz.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        DM_CUDA(cudaStreamSynchronize(h->stream));
        if (err) {
            DM_CUDA(cudaMemsetAsync(Lz.err, 0, sizeof(int), h->stream));
            DM_CUDA(cudaStreamSynchronize(h->stream));
            return fail(DM_ETIMEOUT, "a grid barrier of the Lanczos step gave up waiting");
        }
    }
    if (is_device_ptr(evals)) DM_CUDA(cudaMemcpyAsync(evals, th.data(), sizeof(double) * k, cudaMemcpyHostToDevice, h->stream));
    else
        for (int i = 0; i < k; ++i) evals[i] = th[i];
    if (evecs) DM_CHECK(copy_out(h, evecs, h->evecs, sizeof(float) * (size_t)k * h->N));
    DM_CUDA(cudaStreamSynchronize(h->stream));
    h->stats.matvec_calls = 0;
    h->stats.ms_matvec = 0.f;
    for (size_t e = 0; e + 1 < ev_mv.size(); e += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev_mv[e], ev_mv[e + 1]) == cudaSuccess) {
            h->stats.ms_matvec += ms;
            h->stats.matvec_calls += 1;
        }
        cudaEventDestroy(ev_mv[e]);
        cudaEventDestroy(ev_mv[e + 1]);
    }
    h->last_k = k;
    h->stats.lanczos_iters = m;
    h->stats.converged = converged ? 1 : 0;
    h->stats.ms_eigs = t.stop();
    return converged ? DM_OK : fail(DM_ENOCONV, "Lanczos did not converge in %d steps", m);
}

int dm_tune_leaf(dm_handle h, double tol, int32_t max_rank, int32_t k, const int32_t *candidates, int32_t ncand,
                 int32_t *best_leaf, float *cost_ms) {
    if (!h || !candidates || !best_leaf) return fail(DM_EINVAL, "NULL argument");
    if (ncand < 1 || k < 1) return fail(DM_EINVAL, "need at least one candidate and k >= 1");
    DM_CHECK(set_device(h));
    float *xv = nullptr, *yv = nullptr;
    std::vector<float> costs((size_t)ncand);
    int best = -1;
    for (int c = 0; c < ncand; ++c) {
        DM_CHECK(dm_compress(h, tol, candidates[c], max_rank));
        h->resolve_laps();
        const float ms_c = h->stats.ms_tree + h->stats.ms_skeleton + h->stats.ms_pack;
        if (!xv) {
            // vectors live with the structure group (freed by the next compression)
            DM_CHECK(ensure_io(h, h->N));
            xv = h->io_x;
            yv = h->io_y;
            DM_CUDA(cudaMemsetAsync(xv, 0, sizeof(float) * (size_t)h->N, h->stream));
        }
        const DmHmat H = h->hmat();
        std::vector<float> ts;
        cudaEvent_t e0, e1;
        DM_CUDA(cudaEventCreate(&e0));
        DM_CUDA(cudaEventCreate(&e1));
        for (int r = 0; r < 6; ++r) {
            DM_CUDA(cudaEventRecord(e0, h->stream));
            DM_CUDA(dm_hmatvec(H, h->near_mode, xv, yv, true, h->stream));
            DM_CUDA(cudaEventRecord(e1, h->stream));
            DM_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            DM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (r > 0) ts.push_back(ms);  // the first call warms up
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        std::sort(ts.begin(), ts.end());
        const float ms_mv = ts[ts.size() / 2];
        costs[(size_t)c] = ms_c + (float)(2 * k + 20) * ms_mv;
        if (best < 0 || costs[(size_t)c] < costs[(size_t)best]) best = c;
    }
    if (best != ncand - 1) DM_CHECK(dm_compress(h, tol, candidates[best], max_rank));
    *best_leaf = candidates[best];
    if (cost_ms)
        for (int c = 0; c < ncand; ++c) cost_ms[c] = costs[(size_t)c];
    return DM_OK;
}

int dm_coords(dm_handle h, int32_t k, int32_t t, float *psi) {
    if (!h) return fail(DM_EINVAL, "handle is NULL");
    if (h->last_k == 0) return fail(DM_ESTATE, "dm_coords before dm_eigs");
    if (k < 1 || k > h->last_k) return fail(DM_EINVAL, "k must be in [1, %d]", h->last_k);
    if (t < 0) return fail(DM_EINVAL, "t must be >= 0");
    if (!psi) return fail(DM_EINVAL, "psi is NULL");
    DM_CHECK(set_device(h));
    const int64_t n = h->N * k;
    const bool pd = is_device_ptr(psi);
    float *dst = psi;
    if (!pd) {
        DM_CHECK(ensure_io(h, n));
        dst = h->io_y;
    }
    DM_CUDA(dm_launch_coords(h->evecs, h->lz.theta, h->dg, h->N, k, t, dst, h->stream));
    if (!pd) DM_CUDA(cudaMemcpyAsync(psi, dst, sizeof(float) * n, cudaMemcpyDeviceToHost, h->stream));
    DM_CUDA(cudaStreamSynchronize(h->stream));
    return DM_OK;
}

int dm_intrinsic_dim(const double *evals, int32_t k, int32_t t, double delta, int32_t *d, int32_t *at_k) {
    if (!evals || !d) return fail(DM_EINVAL, "evals or d is NULL");
    if (k < 2) return fail(DM_EINVAL, "k must be >= 2 (the trivial eigenvalue and at least one more)");
    if (t < 1) return fail(DM_EINVAL, "t must be >= 1");
    if (!(delta > 0.0 && delta < 1.0)) return fail(DM_EINVAL, "delta must be in (0, 1)");
    for (int l = 0; l < k; ++l)
        if (std::isnan(evals[l])) return fail(DM_EINVAL, "eigenvalue %d is NaN", l);
    // |lambda_l|^t > delta |lambda_1|^t, compared as t log(|lambda_l| / |lambda_1|) > log(delta)
    // so that large t neither underflows nor overflows
    const double l1 = std::fabs(evals[1]), ld = std::log(delta);
    int best = 0;
    if (l1 > 0.0)
        for (int l = 1; l < k; ++l) {
            const double r = std::fabs(evals[l]) / l1;
            if (r > 0.0 && (double)t * std::log(r) > ld) best = l;
        }
    *d = best;
    if (at_k) *at_k = (best == k - 1) ? 1 : 0;
    return DM_OK;
}

int dm_get_stats(dm_handle h, dm_stats *st) {
    if (!h || !st) return fail(DM_EINVAL, "NULL argument");
    resolve_create_time(h);
    h->resolve_laps();
    *st = h->stats;
    return DM_OK;
}

int dm_get_eps(dm_handle h, double *eps) {
    if (!h || !eps) return fail(DM_EINVAL, "NULL argument");
    *eps = h->eps;
    return DM_OK;
}

int dm_get_degrees(dm_handle h, double *q, double *dg, double *s) {
    if (!h) return fail(DM_EINVAL, "handle is NULL");
    DM_CHECK(set_device(h));
    const size_t b = sizeof(double) * (size_t)h->N;
    if (q) DM_CHECK(copy_out(h, q, h->q, b));
    if (dg) DM_CHECK(copy_out(h, dg, h->dg, b));
    if (s) DM_CHECK(copy_out(h, s, h->s, b));
    DM_CUDA(cudaStreamSynchronize(h->stream));
    return DM_OK;
}

int dm_get_tree(dm_handle h, int32_t *L, int32_t *perm) {
    if (!h) return fail(DM_EINVAL, "handle is NULL");
    if (!h->compressed) return fail(DM_ESTATE, "no compressed structure");
    DM_CHECK(set_device(h));
    if (L) *L = h->L;
    if (perm) {
        DM_CHECK(copy_out(h, perm, h->perm, sizeof(int32_t) * (size_t)h->N));
        DM_CUDA(cudaStreamSynchronize(h->stream));
    }
    return DM_OK;
}

int dm_get_hmatrix(dm_handle h, int32_t *ranks, int32_t *skel, float *P) {
    if (!h) return fail(DM_EINVAL, "handle is NULL");
    if (!h->compressed) return fail(DM_ESTATE, "no compressed structure");
    DM_CHECK(set_device(h));
    const int nnodes = (1 << (h->L + 1)) - 1;
    if (ranks) DM_CHECK(copy_out(h, ranks, h->ranks, sizeof(int32_t) * nnodes));
    if (skel) DM_CHECK(copy_out(h, skel, h->skel, sizeof(int32_t) * (size_t)nnodes * h->max_rank));
    if (P)
        DM_CUDA(cudaMemcpy2DAsync(P, sizeof(float) * h->cmax, h->P, sizeof(float) * h->ldp, sizeof(float) * h->cmax,
                                  (size_t)nnodes * h->max_rank, cudaMemcpyDefault, h->stream));
    DM_CUDA(cudaStreamSynchronize(h->stream));
    return DM_OK;
}

int dm_load_hmatrix(dm_handle h, int32_t L, int32_t max_rank, const int32_t *perm, const int32_t *ranks,
                    const int32_t *skel, const float *P) {
    if (!h) return fail(DM_EINVAL, "handle is NULL");
    if (!perm || !ranks || !skel || !P) return fail(DM_EINVAL, "NULL structure array");
    if (L < 0 || L > 20 || ((int64_t)1 << L) > h->N) return fail(DM_EINVAL, "bad depth %d", L);
    if (max_rank < 1 || max_rank > 1024) return fail(DM_EINVAL, "bad max_rank %d", max_rank);
    if (is_device_ptr(perm) || is_device_ptr(ranks) || is_device_ptr(skel) || is_device_ptr(P))
        return fail(DM_EINVAL, "dm_load_hmatrix takes host buffers");
    DM_CHECK(set_device(h));
    const int nnodes = (1 << (L + 1)) - 1;
    const int leaf_max = (int)((h->N + ((int64_t)1 << L) - 1) >> L);
    const int cmax = leaf_max > 2 * max_rank ? leaf_max : 2 * max_rank;
    // ---- validate on the host
    std::vector<char> seen((size_t)h->N, 0);
    for (int64_t i = 0; i < h->N; ++i) {
        const int32_t v = perm[i];
        if (v < 0 || v >= h->N || seen[(size_t)v]) return fail(DM_EINVAL, "perm is not a permutation");
        seen[(size_t)v] = 1;
    }
    if (ranks[0] != 0) return fail(DM_EINVAL, "root rank must be 0");
    for (int node = nnodes - 1; node >= 1; --node) {
        int64_t st, sz;
        dm_node_range(h->N, node, &st, &sz);
        const int lvl = dm_level_of(node);
        const int r = ranks[node];
        const int64_t c = (lvl == L) ? sz : (int64_t)ranks[2 * node + 1] + ranks[2 * node + 2];
        if (r < 0 || r > max_rank || r > c) return fail(DM_EINVAL, "node %d: rank %d out of range", node, r);
        for (int t = 0; t < r; ++t) {
            const int32_t p = skel[(int64_t)node * max_rank + t];
            bool ok = false;
            if (lvl == L) ok = p >= st && p < st + sz;
            else {
                for (int child = 2 * node + 1; child <= 2 * node + 2 && !ok; ++child)
                    for (int u = 0; u < ranks[child] && !ok; ++u) ok = skel[(int64_t)child * max_rank + u] == p;
            }
            if (!ok) return fail(DM_EINVAL, "node %d: skeleton %d is not a candidate", node, p);
        }
        for (int t = 0; t < r; ++t)
            for (int64_t j = 0; j < c; ++j)
                if (!std::isfinite(P[((int64_t)node * max_rank + t) * cmax + j]))
                    return fail(DM_EINVAL, "node %d: non-finite P", node);
    }
    DM_CHECK(alloc_structure(h, L, max_rank));
    h->tol = -1.0;
    resolve_near_mode(h);
    int32_t *pa = nullptr;
    DM_CHECK(h->alloc(&pa, (size_t)h->N, G_STRUCT));
    h->perm = pa;
    DM_CUDA(cudaMemcpyAsync(h->perm, perm, sizeof(int32_t) * (size_t)h->N, cudaMemcpyHostToDevice, h->stream));
    DM_CUDA(cudaMemcpyAsync(h->ranks, ranks, sizeof(int32_t) * nnodes, cudaMemcpyHostToDevice, h->stream));
    DM_CUDA(cudaMemcpyAsync(h->skel, skel, sizeof(int32_t) * (size_t)nnodes * max_rank, cudaMemcpyHostToDevice,
                            h->stream));
    DM_CUDA(cudaMemcpy2DAsync(h->P, sizeof(float) * h->ldp, P, sizeof(float) * cmax, sizeof(float) * cmax,
                              (size_t)nnodes * max_rank, cudaMemcpyHostToDevice, h->stream));
    DM_CUDA(dm_permute_points(h->Xs, h->sf, h->perm, h->N, h->d, h->Xp, h->sp, h->stream));
    DM_CHECK(finish_structure(h));
    DM_CUDA(cudaStreamSynchronize(h->stream));
    return DM_OK;
}

}  // extern "C"
