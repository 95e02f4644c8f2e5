// k_tree.cu -- geometry-oblivious balanced partition tree, built level by level on the device.
//
// The tree is the partition behind the H-matrix form of Eq. 2.18 (block-diagonal
// near field D on the leaves, low-rank far field UV between siblings). Split rule
// of a node whose points are in increasing original index (the paper leaves the
// rule to GOFMM; this is the reading the oracle implements as well):
//   anchor i0 = its first point; p = farthest point from i0 and q = farthest from p
//   in the Gram distance of W (largest squared distance, lowest index on ties);
//   key_i = W_iq - W_ip; the ceil(n/2) smallest (key, index) go left; both
//   children keep increasing original index.
// All decisions are taken in FP64 with the same operation order as the oracle, so
// both build the same tree (at high dimension from an FP64 copy of the points made once,
// which saves the FP64 pipe two conversions per coordinate). The O(n) FP64 passes of every level are cut into
// 512-point items spread over all SMs (FP64 is a narrow pipe on this GPU); the
// exact median and the stable partition run one CTA per node on integer keys.
#include <vector>

#include "dm_internal.cuh"

namespace {

constexpr int kItemPoints = 512;
constexpr int kTreeThreads = 256;

struct TreeItem {
    int node;
    int first_item;  // first item of this node in the level's list
    int nitems;      // items of this node
    int pad;
    long long lo, hi;  // positions [lo, hi)
};

struct Cand {
    unsigned long long val;  // bit pattern of a non-negative double (orders like the value)
    int idx;                 // original point index
};

__device__ __forceinline__ bool cand_better(const Cand &a, const Cand &b) {
    return a.val > b.val || (a.val == b.val && a.idx < b.idx);
}

__device__ __forceinline__ Cand warp_best(Cand c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Cand other;
        other.val = __shfl_xor_sync(DM_FULL, c.val, o);
        other.idx = __shfl_xor_sync(DM_FULL, c.idx, o);
        if (cand_better(other, c)) c = other;
    }
    return c;
}

// best over the block; result valid in every thread
__device__ Cand block_best(Cand c) {
    __shared__ unsigned long long sv[32];
    __shared__ int si[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    c = warp_best(c);
    __syncthreads();
    if (lane == 0) { sv[w] = c.val; si[w] = c.idx; }
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    Cand r;
    r.val = 0ull;
    r.idx = 0x7fffffff;
    if (lane < nw) { r.val = sv[lane]; r.idx = si[lane]; }
    r = warp_best(r);
    return r;
}

// source point of an item: the node's anchor (prev == nullptr) or the best candidate of the previous pass
__device__ int item_source(const TreeItem &it, const TreeItem *items, const Cand *prev, const int32_t *perm) {
    if (prev == nullptr) return perm[items[it.first_item].lo];
    Cand c;
    c.val = 0ull;
    c.idx = 0x7fffffff;
    for (int t = threadIdx.x; t < it.nitems; t += blockDim.x) {
        Cand o = prev[it.first_item + t];
        if (cand_better(o, c)) c = o;
    }
    return block_best(c).idx;
}

// farthest point (largest FP64 squared distance) from the item's source; optionally
// store W = exp(-r2/eps) per position for the key pass
template <class T>
__global__ void __launch_bounds__(kTreeThreads) farthest_kernel(const TreeItem *__restrict__ items,
                                                               const T *__restrict__ X, int d,
                                                               const int32_t *__restrict__ perm,
                                                               const Cand *__restrict__ prev,
                                                               Cand *__restrict__ out, double *__restrict__ wbuf,
                                                               double eps) {
    const TreeItem it = items[blockIdx.x];
    const int src = item_source(it, items, prev, perm);
    const T *xs = X + (int64_t)src * d;
    Cand best;
    best.val = 0ull;
    best.idx = 0x7fffffff;
    for (long long pos = it.lo + threadIdx.x; pos < it.hi; pos += blockDim.x) {
        const int i = perm[pos];
        const double r2 = dm_sqdist64(xs, X + (int64_t)i * d, d);
        Cand c;
        c.val = (unsigned long long)__double_as_longlong(r2);
        c.idx = i;
        if (cand_better(c, best)) best = c;
        if (wbuf) wbuf[pos] = exp(-r2 / eps);
    }
    best = block_best(best);
    if (threadIdx.x == 0) out[blockIdx.x] = best;
}

// key_i = W_iq - W_ip as order-preserving 64-bit integers
template <class T>
__global__ void __launch_bounds__(kTreeThreads) key_kernel(const TreeItem *__restrict__ items,
                                                          const T *__restrict__ X, int d,
                                                          const int32_t *__restrict__ perm,
                                                          const Cand *__restrict__ candq,
                                                          const double *__restrict__ wbuf, double eps,
                                                          uint64_t *__restrict__ keys) {
    const TreeItem it = items[blockIdx.x];
    const int q = item_source(it, items, candq, perm);
    const T *xq = X + (int64_t)q * d;
    for (long long pos = it.lo + threadIdx.x; pos < it.hi; pos += blockDim.x) {
        const int i = perm[pos];
        const double r2 = dm_sqdist64(xq, X + (int64_t)i * d, d);
        const double key = __dsub_rn(exp(-r2 / eps), wbuf[pos]);
        keys[pos] = dm_order_key(key);
    }
}

// exclusive prefix count of `flag` over the block (and the block total)
__device__ __forceinline__ int block_exclusive_count(bool flag, int *total, int *warp_tot) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned b = __ballot_sync(DM_FULL, flag);
    const int in_warp = __popc(b & ((1u << lane) - 1u));
    __syncthreads();
    if (lane == 0) warp_tot[w] = __popc(b);
    __syncthreads();
    int off = 0, tot = 0;
    const int nw = blockDim.x >> 5;
    for (int k = 0; k < nw; ++k) {
        const int v = warp_tot[k];
        if (k < w) off += v;
        tot += v;
    }
    *total = tot;
    return off + in_warp;
}

// one CTA per node: exact median by radix select, then a stable partition
__global__ void __launch_bounds__(1024) split_kernel(int first_node, int64_t N, const int32_t *__restrict__ perm_in,
                                                     const uint64_t *__restrict__ keys,
                                                     int32_t *__restrict__ perm_out) {
    __shared__ unsigned hist[256];
    __shared__ int warp_tot[32];
    int64_t st, sz;
    dm_node_range(N, first_node + (int)blockIdx.x, &st, &sz);
    const int64_t nl = (sz + 1) / 2;
    if (sz <= 1) {
        if (sz == 1 && threadIdx.x == 0) perm_out[st] = perm_in[st];
        return;
    }
    const uint64_t *k = keys + st;
    int64_t below;
    const uint64_t T = dm_cta_select([k](int64_t i) { return k[i]; }, sz, nl - 1, hist, &below);
    const int64_t need_eq = nl - below;  // equal keys that go left, first ones in index order
    int64_t left_off = 0, right_off = 0, eq_seen = 0;
    for (int64_t base = 0; base < sz; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool valid = i < sz;
        const uint64_t key = valid ? k[i] : ~0ull;
        const bool is_eq = valid && key == T;
        int tot_eq;
        const int eq_rank = block_exclusive_count(is_eq, &tot_eq, warp_tot);
        const bool left = valid && (key < T || (is_eq && eq_seen + eq_rank < need_eq));
        int tot_left;
        const int lrank = block_exclusive_count(left, &tot_left, warp_tot);
        if (valid) {
            const int32_t v = perm_in[st + i];
            if (left) perm_out[st + left_off + lrank] = v;
            else perm_out[st + nl + right_off + ((int)threadIdx.x - lrank)] = v;
        }
        const int tile = (int)((int64_t)blockDim.x < sz - base ? (int64_t)blockDim.x : sz - base);
        left_off += tot_left;
        right_off += tile - tot_left;
        eq_seen += tot_eq;
    }
}

// ---- the split of large nodes across many CTAs (levels whose nodes exceed kBigNode points):
// the same rule as split_kernel -- threshold T = the (ceil(n/2) - 1)-th smallest key by an
// exact radix select (8-bit digits from the top), then a stable partition -- but the
// histogram of every digit pass and the partition run over the level's 512-point items, with
// per-node state in global memory; the partition ranks come from per-item counts.
constexpr int64_t kBigNode = 8192;

struct SplitSel {
    unsigned long long prefix;  // digits chosen so far
    long long k;                // rank still to find among the keys matching prefix
    long long below;            // keys of the node smaller than the prefix's range
    long long pad;
};

__global__ void split_sel_init_kernel(SplitSel *S, int first_node, int count, int64_t N, unsigned *hist) {
    const int n = blockIdx.x;
    if (n >= count) return;
    if (threadIdx.x == 0) {
        int64_t st, sz;
        dm_node_range(N, first_node + n, &st, &sz);
        S[n].prefix = 0ull;
        S[n].k = (sz + 1) / 2 - 1;
        S[n].below = 0;
    }
    for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[n * 256 + b] = 0u;
}

__global__ void __launch_bounds__(512) split_hist_kernel(const TreeItem *__restrict__ items,
                                                         const uint64_t *__restrict__ keys,
                                                         const SplitSel *__restrict__ S, unsigned *hist,
                                                         int first_node, int shift) {
    __shared__ unsigned sh[256];
    const TreeItem it = items[blockIdx.x];
    const int n = it.node - first_node;
    const unsigned long long mask = shift >= 56 ? 0ull : (~0ull << (shift + 8));
    const unsigned long long pre = S[n].prefix & mask;
    for (int b = threadIdx.x; b < 256; b += blockDim.x) sh[b] = 0u;
    __syncthreads();
    for (long long pos = it.lo + threadIdx.x; pos < it.hi; pos += blockDim.x) {
        const uint64_t key = keys[pos];
        if ((key & mask) == pre) atomicAdd(&sh[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x)
        if (sh[b]) atomicAdd(hist + n * 256 + b, sh[b]);
}

// One block of 256 threads per node (thread b owns digit bin b): the digit is the first bin
// b <= 254 whose inclusive count exceeds the rank k still sought, else 255; the keys of the
// bins before it move from k to `below`. A block scan of the 256 counts replaces a serial
// walk over the bins (one dependent global load per bin).
__global__ void __launch_bounds__(256) split_step_kernel(SplitSel *S, unsigned *hist, int shift) {
    const int n = blockIdx.x, b = threadIdx.x, lane = b & 31, warp = b >> 5;
    __shared__ long long wsum[8];
    __shared__ int s_b;
    __shared__ long long s_acc;
    const long long h = (long long)hist[n * 256 + b];
    long long x = h;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(DM_FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    if (b == 0) s_b = 255;
    __syncthreads();
    long long off = 0;
    for (int w = 0; w < warp; ++w) off += wsum[w];
    const long long incl = off + x, excl = incl - h;
    const long long k = S[n].k;
    if (b < 255 && incl > k) atomicMin(&s_b, b);
    __syncthreads();
    if (b == s_b) s_acc = excl;
    __syncthreads();
    if (b == 0) {
        S[n].k -= s_acc;
        S[n].below += s_acc;
        S[n].prefix |= (unsigned long long)s_b << shift;
    }
    hist[n * 256 + b] = 0u;
}

// per item: keys below the threshold and keys equal to it
__global__ void __launch_bounds__(512) split_count_kernel(const TreeItem *__restrict__ items,
                                                          const uint64_t *__restrict__ keys,
                                                          const SplitSel *__restrict__ S, int first_node,
                                                          int2 *__restrict__ icnt) {
    __shared__ int warp_tot[32];
    const TreeItem it = items[blockIdx.x];
    const uint64_t T = S[it.node - first_node].prefix;
    const long long pos = it.lo + threadIdx.x;
    const bool valid = pos < it.hi;
    const uint64_t key = valid ? keys[pos] : ~0ull;
    int nlt, neq;
    block_exclusive_count(valid && key < T, &nlt, warp_tot);
    block_exclusive_count(valid && key == T, &neq, warp_tot);
    if (threadIdx.x == 0) icnt[blockIdx.x] = make_int2(nlt, neq);
}

// stable partition: left = keys below T, then the first (ceil(n/2) - below) keys equal to T in
// position order; an element's destination follows from the counts of the items before it
__global__ void __launch_bounds__(512) split_scatter_kernel(const TreeItem *__restrict__ items,
                                                            const uint64_t *__restrict__ keys,
                                                            const SplitSel *__restrict__ S,
                                                            const int2 *__restrict__ icnt, int first_node,
                                                            int64_t N, const int32_t *__restrict__ perm_in,
                                                            int32_t *__restrict__ perm_out) {
    __shared__ int warp_tot[32];
    __shared__ long long s_lt, s_eq;
    const TreeItem it = items[blockIdx.x];
    const int n = it.node - first_node;
    int64_t st, sz;
    dm_node_range(N, it.node, &st, &sz);
    const int64_t nl = (sz + 1) / 2;
    const uint64_t T = S[n].prefix;
    const long long need_eq = nl - S[n].below;
    if (threadIdx.x == 0) { s_lt = 0; s_eq = 0; }
    __syncthreads();
    long long lt_b = 0, eq_b = 0;
    for (int t = it.first_item + (int)threadIdx.x; t < (int)blockIdx.x; t += blockDim.x) {
        const int2 c = icnt[t];
        lt_b += c.x;
        eq_b += c.y;
    }
    atomicAdd(reinterpret_cast<unsigned long long *>(&s_lt), (unsigned long long)lt_b);
    atomicAdd(reinterpret_cast<unsigned long long *>(&s_eq), (unsigned long long)eq_b);
    __syncthreads();
    const long long pos = it.lo + threadIdx.x;
    const bool valid = pos < it.hi;
    const uint64_t key = valid ? keys[pos] : ~0ull;
    const bool lt = valid && key < T, eq = valid && key == T;
    int tot;
    const int lt_rank = block_exclusive_count(lt, &tot, warp_tot);
    const int eq_rank = block_exclusive_count(eq, &tot, warp_tot);
    if (!valid) return;
    const long long gl_lt = s_lt + lt_rank, gl_eq = s_eq + eq_rank;
    const bool left = lt || (eq && gl_eq < need_eq);
    const long long left_before = gl_lt + (gl_eq < need_eq ? gl_eq : need_eq);
    const long long i_node = pos - st;
    const long long dest = left ? st + left_before : st + nl + (i_node - left_before);
    perm_out[dest] = perm_in[pos];
}

}  // namespace

cudaError_t dm_tree_build(const float *X, const double *X64, int64_t N, int d, double eps, int L, int32_t *perm_a,
                          int32_t *perm_b, int32_t **perm_out, DmTreeWork *w, cudaStream_t st) {
    // item lists of every level, built on the host from the (deterministic) node ranges
    std::vector<TreeItem> items;
    std::vector<int> level_first(L + 1, 0);
    for (int lvl = 0; lvl < L; ++lvl) {
        level_first[lvl] = (int)items.size();
        const int first = (1 << lvl) - 1, count = 1 << lvl;
        for (int kk = 0; kk < count; ++kk) {
            int64_t s0, sz;
            dm_node_range(N, first + kk, &s0, &sz);
            const int nit = (int)((sz + kItemPoints - 1) / kItemPoints);
            const int f = (int)items.size() - level_first[lvl];  // relative to the level's list
            for (int t = 0; t < nit; ++t) {
                TreeItem it;
                it.node = first + kk;
                it.first_item = f;
                it.nitems = nit;
                it.pad = 0;
                it.lo = s0 + (int64_t)t * kItemPoints;
                it.hi = s0 + (int64_t)(t + 1) * kItemPoints < s0 + sz ? s0 + (int64_t)(t + 1) * kItemPoints : s0 + sz;
                items.push_back(it);
            }
        }
    }
    level_first[L] = (int)items.size();
    if ((int)items.size() > w->max_items) return cudaErrorInvalidValue;
    cudaError_t e;
    TreeItem *ditems = reinterpret_cast<TreeItem *>(w->items);
    if (!items.empty()) {
        e = cudaMemcpyAsync(ditems, items.data(), sizeof(TreeItem) * items.size(), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
    }
    Cand *c1 = reinterpret_cast<Cand *>(w->cand1);
    Cand *c2 = reinterpret_cast<Cand *>(w->cand2);
    int32_t *in = perm_a, *out = perm_b;
    for (int lvl = 0; lvl < L; ++lvl) {
        const int f = level_first[lvl], n = level_first[lvl + 1] - level_first[lvl];
        const TreeItem *li = ditems + f;  // first_item fields are relative to this pointer
        if (X64) {
            farthest_kernel<double><<<n, kTreeThreads, 0, st>>>(li, X64, d, in, nullptr, c1, nullptr, eps);
            farthest_kernel<double><<<n, kTreeThreads, 0, st>>>(li, X64, d, in, c1, c2, w->wbuf, eps);
            key_kernel<double><<<n, kTreeThreads, 0, st>>>(li, X64, d, in, c2, w->wbuf, eps, w->keys);
        } else {
            farthest_kernel<float><<<n, kTreeThreads, 0, st>>>(li, X, d, in, nullptr, c1, nullptr, eps);
            farthest_kernel<float><<<n, kTreeThreads, 0, st>>>(li, X, d, in, c1, c2, w->wbuf, eps);
            key_kernel<float><<<n, kTreeThreads, 0, st>>>(li, X, d, in, c2, w->wbuf, eps, w->keys);
        }
        dm_count_launches(2);
        dm_count_launches(1);
        int64_t s0, sz0;
        dm_node_range(N, (1 << lvl) - 1, &s0, &sz0);
        if (sz0 > kBigNode && w->sel && (1 << lvl) <= w->max_big) {
            // large nodes: select and partition over the level's items
            SplitSel *S = reinterpret_cast<SplitSel *>(w->sel);
            const int first = (1 << lvl) - 1, count = 1 << lvl;
            split_sel_init_kernel<<<count, 256, 0, st>>>(S, first, count, N, w->hist);
            dm_count_launches(1);
            for (int shift = 56; shift >= 0; shift -= 8) {
                split_hist_kernel<<<n, 512, 0, st>>>(li, w->keys, S, w->hist, first, shift);
                split_step_kernel<<<count, 256, 0, st>>>(S, w->hist, shift);
                dm_count_launches(2);
            }
            int2 *icnt = reinterpret_cast<int2 *>(w->icnt);
            split_count_kernel<<<n, 512, 0, st>>>(li, w->keys, S, first, icnt);
            split_scatter_kernel<<<n, 512, 0, st>>>(li, w->keys, S, icnt, first, N, in, out);
            dm_count_launches(2);
        } else {
            split_kernel<<<1 << lvl, 1024, 0, st>>>((1 << lvl) - 1, N, in, w->keys, out);
            dm_count_launches(1);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        int32_t *t = in;
        in = out;
        out = t;
    }
    *perm_out = in;
    return cudaSuccess;
}

size_t dm_tree_items_bound(int64_t N, int L) {
    size_t n = 0;
    for (int lvl = 0; lvl < L; ++lvl) n += (size_t)((N + kItemPoints - 1) / kItemPoints) + ((size_t)1 << lvl);
    return n;
}
size_t dm_tree_item_bytes() { return sizeof(TreeItem); }
size_t dm_tree_sel_bytes() { return sizeof(SplitSel); }
int64_t dm_tree_big_node() { return kBigNode; }
size_t dm_tree_cand_bytes() { return sizeof(Cand); }
