// dm_serve.cu -- request server: independent diffusion-map solves admitted as slots and
// device memory free up. Each slot builds a request's kernel and compression (dm_create,
// dm_compress) on its own CUDA stream, so that concurrently running builds overlap on the GPU;
// single-vector eigensolves then join a batched solver (one per size class), whose thread
// advances every resident request's Lanczos iteration in the same launches, each request at
// its own step, and finishes each one when its own convergence check says so (continuous
// batching at step level). Block Lanczos requests run their eigensolve on their slot.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "dm_internal.cuh"

int dm_lanczos_kmax();

namespace {

inline uint64_t r256(uint64_t b) { return (b + 255) & ~uint64_t(255); }

// solver lanes by request size: lane l takes requests of at most kLaneN[l] points (the last
// lane the rest); lower lanes run on higher-priority streams
constexpr int kLanes = 4;
constexpr int64_t kLaneN[kLanes - 1] = {5000, 15000, 40000};
inline int lane_of(int64_t N) {
    int l = 0;
    while (l < kLanes - 1 && N > kLaneN[l]) ++l;
    return l;
}

enum JobState { kQueued = 0, kRunning = 1, kDone = 2 };

struct Job;
struct Handoff {
    Job *j;
    dm_handle h;
    cudaEvent_t ready;
};

struct Job {
    dm_ticket id = 0;
    dm_request req{};
    std::vector<float> points;
    uint64_t bytes = 0;
    JobState state = kQueued;
    std::vector<double> evals;
    std::vector<float> evecs;
    std::string error;
    dm_result res{};
};

struct Server {
    std::mutex mu;
    std::condition_variable cv;
    bool running = false, stopping = false;
    int device = 0;
    uint64_t budget = 0, used = 0;
    int capacity = 65536;
    int busy = 0;
    dm_ticket next_id = 1;
    std::deque<Job *> queue;
    std::map<dm_ticket, std::unique_ptr<Job>> jobs;
    std::vector<std::thread> workers;
    // batched eigensolvers, one per size class (lane_of), so that small requests are not held
    // to the step time of large ones: each with its thread and the requests handed to it
    struct Lane {
        std::thread th;
        std::condition_variable cv;
        std::deque<Handoff> handoff;
    };
    Lane lanes[kLanes];
    bool workers_done = false;
    // slot streams, then each lane's solver stream and result stream; destroyed after every
    // thread has ended (the slots' allocations are freed on their streams, possibly by a
    // solver's thread)
    std::vector<cudaStream_t> streams;
    std::chrono::steady_clock::time_point t0;

    double now_ms() const {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
};

Server g_srv;

bool valid_request(const dm_request *r) {
    return r && r->points && r->N >= 2 && r->d >= 1 && r->alpha >= 0.0 && r->tol >= 0.0 && r->leaf_size >= 1 &&
           r->max_rank >= 1 && r->max_rank <= 256 && r->k >= 1 && r->k < r->N && r->k <= dm_lanczos_kmax() &&
           r->N <= (int64_t)0x7fffffff && r->block_size >= 0 && r->block_size <= 16;
}

// pick the first queued job that fits (caller holds the lock); nullptr if none
Job *admit_locked(Server &S) {
    for (auto it = S.queue.begin(); it != S.queue.end(); ++it) {
        Job *j = *it;
        if (S.used + j->bytes <= S.budget || S.used == 0) {
            S.queue.erase(it);
            return j;
        }
    }
    return nullptr;
}

// stream-ordered allocations on the slot's stream: no device-wide synchronisation
// between concurrently running solves (plain cudaFree would serialise them)
void *slot_alloc(size_t bytes, void *user) {
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, reinterpret_cast<cudaStream_t>(user)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}
void slot_free(void *p, size_t, void *user) { cudaFreeAsync(p, reinterpret_cast<cudaStream_t>(user)); }

// completed request: release its memory and publish the result (takes the lock)
void finish_job(Job *j, int status) {
    {
        std::lock_guard<std::mutex> lk(g_srv.mu);
        j->res.status = status;
        g_srv.used -= j->bytes;
        j->points.clear();
        j->points.shrink_to_fit();
        j->res.done_ms = g_srv.now_ms();
        j->res.k = j->req.k;
        j->res.N = j->req.N;
        j->res.evals = j->evals.empty() ? nullptr : j->evals.data();
        j->res.evecs = j->evecs.empty() ? nullptr : j->evecs.data();
        j->res.error = j->error.c_str();
        j->state = kDone;
    }
    g_srv.cv.notify_all();
}

// build the request's kernel and compression on the slot's stream; single-vector solves are
// handed to the batched solver (returns false), block solves run here (returns true)
bool run_job(Job *j, cudaStream_t stream, int *status) {
    dm_config cfg;
    dm_config_default(&cfg);
    cfg.seed = j->req.seed;
    cfg.stream = stream;
    cfg.device = g_srv.device;
    cfg.alloc = slot_alloc;
    cfg.free = slot_free;
    cfg.alloc_user = stream;
    cfg.shared_device = 1;  // other slots run concurrently: no cooperative launches
    // a convergence check of a block solve runs in order on the slot's stream and the slot's
    // thread waits for it: check every second step, not every step
    cfg.check_every = 2;
    cfg.block_size = j->req.block_size;
    dm_handle h = nullptr;
    const int k = j->req.k;
    int st = dm_create(j->points.data(), j->req.N, j->req.d, j->req.eps, j->req.alpha, &cfg, &h);
    if (st == DM_OK) st = dm_compress(h, j->req.tol, j->req.leaf_size, j->req.max_rank);
    {
        std::lock_guard<std::mutex> lk(g_srv.mu);
        j->res.built_ms = g_srv.now_ms();
    }
    if (st == DM_OK && j->req.block_size < 2) {
        cudaEvent_t ready = nullptr;
        st = dm_batch_prepare(h, &ready);
        if (st == DM_OK) {
            Server::Lane &ln = g_srv.lanes[lane_of(j->req.N)];
            {
                std::lock_guard<std::mutex> lk(g_srv.mu);
                ln.handoff.push_back(Handoff{j, h, ready});
            }
            ln.cv.notify_one();
            return false;
        }
        if (ready) cudaEventDestroy(ready);
    } else if (st == DM_OK) {
        j->evals.assign((size_t)k, 0.0);
        if (j->req.want_vectors) j->evecs.assign((size_t)k * (size_t)j->req.N, 0.f);
        st = dm_eigs(h, k, j->evals.data(), j->req.want_vectors ? j->evecs.data() : nullptr);
        dm_stats s{};
        dm_get_stats(h, &s);
        j->res.lanczos_iters = s.lanczos_iters;
    }
    if (st != DM_OK && st != DM_ENOCONV) j->error = dm_last_error();
    if (h) dm_destroy(h);
    *status = st;
    return true;
}

void worker_main(cudaStream_t stream) {
    cudaSetDevice(g_srv.device);
    for (;;) {
        Job *j = nullptr;
        {
            std::unique_lock<std::mutex> lk(g_srv.mu);
            g_srv.cv.wait(lk, [&] {
                if (g_srv.stopping) return true;
                for (Job *q : g_srv.queue)
                    if (g_srv.used + q->bytes <= g_srv.budget || g_srv.used == 0) return true;
                return false;
            });
            if (g_srv.stopping) break;
            j = admit_locked(g_srv);
            if (!j) continue;
            g_srv.used += j->bytes;
            g_srv.busy += 1;
            j->state = kRunning;
            j->res.start_ms = g_srv.now_ms();
        }
        int st = DM_OK;
        const bool finished = run_job(j, stream, &st);
        {
            std::lock_guard<std::mutex> lk(g_srv.mu);
            g_srv.busy -= 1;
        }
        if (finished) finish_job(j, st);
    }
}

// the batched eigensolver: takes handed-over requests between steps, advances every resident
// one by a step, and finishes those whose check decided (results copied to the host, handle
// destroyed, memory released); ends when the slots have ended and nothing is resident
void solver_main(int lane, cudaStream_t stream, cudaStream_t out) {
    cudaSetDevice(g_srv.device);
    Server::Lane &ln = g_srv.lanes[lane];
    std::unique_ptr<DmBatchSolver, void (*)(DmBatchSolver *)> B(dm_batch_create(g_srv.device, stream),
                                                                dm_batch_destroy);
    std::vector<std::pair<Job *, dm_handle>> resident;
    std::vector<DmBatchDone> done;
    auto drop = [&](Job *j, dm_handle h, int st, const char *why) {
        j->error = why ? why : dm_last_error();
        dm_destroy(h);
        finish_job(j, st);
    };
    for (;;) {
        std::deque<Handoff> in;
        {
            std::unique_lock<std::mutex> lk(g_srv.mu);
            ln.cv.wait(lk, [&] {
                return !ln.handoff.empty() || dm_batch_active(B.get()) > 0 || g_srv.workers_done;
            });
            in.swap(ln.handoff);
            if (in.empty() && dm_batch_active(B.get()) == 0 && g_srv.workers_done) break;
        }
        for (Handoff &x : in) {
            // the handle's own stream becomes `out`, where its results are read and its wait
            // before destruction ends at once
            const int st = dm_batch_add(B.get(), x.h, x.j->req.k, x.j, x.ready, out);
            cudaEventDestroy(x.ready);
            if (st == DM_OK) {
                resident.emplace_back(x.j, x.h);
            } else {
                drop(x.j, x.h, st, nullptr);
            }
        }
        if (dm_batch_active(B.get()) == 0) continue;
        done.clear();
        const int st = dm_batch_step(B.get(), done);
        for (DmBatchDone &d : done) {
            Job *j = static_cast<Job *>(d.tag);
            j->evals = d.theta;
            j->res.lanczos_iters = d.iters;
            int rs = d.status;
            // on `out`, after the vectors: the step queued after them keeps running meanwhile
            cudaError_t ce = cudaStreamWaitEvent(out, d.ready, 0);
            if (ce == cudaSuccess && j->req.want_vectors) {
                j->evecs.assign((size_t)d.k * (size_t)j->req.N, 0.f);
                ce = cudaMemcpyAsync(j->evecs.data(), d.evecs, sizeof(float) * j->evecs.size(), cudaMemcpyDeviceToHost,
                                     out);
            }
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(out);
            if (ce != cudaSuccess) {
                cudaGetLastError();
                rs = DM_ECUDA;
                j->error = "reading the eigenvectors failed";
            }
            dm_destroy(d.h);
            for (size_t i = 0; i < resident.size(); ++i)
                if (resident[i].first == j) {
                    resident.erase(resident.begin() + (long)i);
                    break;
                }
            finish_job(j, rs);
        }
        if (st != DM_OK) {
            // the step failed: every resident request fails with it; start over empty
            const std::string why = dm_last_error();
            for (auto &r : resident) drop(r.first, r.second, st, why.c_str());
            resident.clear();
            B.reset(dm_batch_create(g_srv.device, stream));
        }
    }
}

}  // namespace

extern "C" {

uint64_t dm_request_bytes(const dm_request *r) {
    if (!r || r->N < 2 || r->d < 1 || r->leaf_size < 1 || r->max_rank < 1) return 0;
    const uint64_t N = (uint64_t)r->N, d = (uint64_t)r->d, R = (uint64_t)r->max_rank;
    const int L = dm_depth_for(r->N, r->leaf_size);
    const uint64_t nleaves = 1ull << L, nnodes = (2ull << L) - 1;
    const uint64_t leaf_max = (N + nleaves - 1) / nleaves;
    const uint64_t ldk = (leaf_max + 3) & ~3ull;
    const uint64_t cmax = leaf_max > 2 * R ? leaf_max : 2 * R;
    const uint64_t ldp = (cmax + 3) & ~3ull, rmax = 2 * R + 10, ldr = (rmax + 3) & ~3ull;
    const uint64_t mmax = 300, kmax = (uint64_t)dm_lanczos_kmax(), ldv = (N + 63) & ~63ull;
    uint64_t b = 0;
    // points, degrees and scalings
    b += 2 * r256(4 * N * d) + 5 * r256(8 * N) + 3 * r256(4 * N);
    // the FP64 copy of the points held until the tree is built (high dimension)
    if (r->d >= kWideMinD) b += r256(8 * N * d);
    // compressed structure
    b += r256(4 * nnodes) + r256(4 * nnodes * R) + r256(4 * nnodes * R * ldp) + r256(4 * N * d) + r256(4 * N);
    b += 2 * r256(4 * N) + r256(4 * nleaves * leaf_max * ldk) + r256(4 * (nleaves > 1 ? nleaves - 1 : 1) * R * R);
    b += 2 * r256(4 * nnodes * R) + r256(4 * N) + r256(4 * nnodes) + r256(4 * nleaves * leaf_max * ((R + 3) & ~3ull));
    // transient workspaces of the compression (skeletonization is the largest)
    b += r256(4 * nleaves * cmax * ldr) + r256(4 * nleaves * R * cmax) + r256(4 * nleaves * R * ldr);
    // the upper tree's shared-memory images (at most one cluster's shared memory)
    b += r256((uint64_t)kTreeMaxCtas * kTreeSmemBudget) + r256(16 * nnodes) + 256;
    // Lanczos basis, Ritz vectors and small arrays
    b += r256(4 * (mmax + 1) * ldv) + r256(4 * ldv) + 2 * r256(4 * kmax * N);
    b += r256(8 * kmax * 6 * mmax) + r256(8 * kmax * mmax) + r256(4 * kmax * mmax) + 16 * 256;
    if (r->block_size >= 2) {
        // block Lanczos: work block, projection partials (2 per SM), T and its reduction, and
        // the block H-matvec's padded vectors and skeleton weights
        const uint64_t bs = (uint64_t)r->block_size;
        b += r256(4 * bs * ldv) + r256(4 * 2 * 152 * (mmax + 1) * bs) + 2 * r256(8 * mmax * mmax);
        b += 2 * r256(4 * bs * nleaves * ldk) + 2 * r256(4 * nnodes * R * bs) + 8 * 256;
    }
    return b;
}

int dm_serve_start(const dm_serve_config *cfg) {
    std::lock_guard<std::mutex> lk(g_srv.mu);
    if (g_srv.running) return dm_fail_msg(DM_ESTATE, "server already running");
    int dev = cfg && cfg->device >= 0 ? cfg->device : -1;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return dm_fail_msg(DM_ECUDA, "no CUDA device available");
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || dev >= ndev) {
        cudaGetLastError();
        return dm_fail_msg(DM_ECUDA, "no CUDA device available");
    }
    g_srv.device = dev;
    {
        // keep freed blocks in this process's pool between requests
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    }
    g_srv.budget = cfg && cfg->hbm_budget_bytes ? cfg->hbm_budget_bytes : 150ull * 1000 * 1000 * 1000;
    g_srv.capacity = cfg && cfg->queue_capacity > 0 ? cfg->queue_capacity : 65536;
    const int slots = cfg && cfg->slots > 0 ? cfg->slots : 4;
    g_srv.used = 0;
    g_srv.busy = 0;
    g_srv.stopping = false;
    g_srv.workers_done = false;
    g_srv.t0 = std::chrono::steady_clock::now();
    if (cudaSetDevice(dev) != cudaSuccess) {
        cudaGetLastError();
        return dm_fail_msg(DM_ECUDA, "cannot select the CUDA device");
    }
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    cudaGetLastError();
    for (int i = 0; i < slots + 2 * kLanes; ++i) {
        cudaStream_t s = nullptr;
        // solver streams (slots + 2 l) by lane: the smallest requests' lane at the highest priority
        int prio = prio_lo;
        if (i >= slots && (i - slots) % 2 == 0) {
            const int l = (i - slots) / 2;
            prio = prio_hi + (prio_lo - prio_hi) * l / (kLanes - 1);  // numerically lower = higher
        }
        if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, prio) != cudaSuccess) {
            cudaGetLastError();
            for (cudaStream_t q : g_srv.streams) cudaStreamDestroy(q);
            g_srv.streams.clear();
            return dm_fail_msg(DM_ECUDA, "stream creation failed");
        }
        g_srv.streams.push_back(s);
    }
    for (int i = 0; i < slots; ++i) g_srv.workers.emplace_back(worker_main, g_srv.streams[(size_t)i]);
    for (int l = 0; l < kLanes; ++l)
        g_srv.lanes[l].th = std::thread(solver_main, l, g_srv.streams[(size_t)(slots + 2 * l)],
                                        g_srv.streams[(size_t)(slots + 2 * l + 1)]);
    g_srv.running = true;
    return DM_OK;
}

int dm_serve_stop(void) {
    std::vector<std::thread> ws;
    {
        std::lock_guard<std::mutex> lk(g_srv.mu);
        if (!g_srv.running) return dm_fail_msg(DM_ESTATE, "server not running");
        g_srv.stopping = true;
        for (Job *j : g_srv.queue) {
            j->res.status = DM_ESTATE;
            j->error = "server stopped before the request ran";
            j->res.error = j->error.c_str();
            j->state = kDone;
        }
        g_srv.queue.clear();
        ws.swap(g_srv.workers);
    }
    g_srv.cv.notify_all();
    // the slots finish the builds they are on (single-vector ones still go to the solver),
    // then the solver finishes every resident request
    for (auto &t : ws) t.join();
    {
        std::lock_guard<std::mutex> lk(g_srv.mu);
        g_srv.workers_done = true;
    }
    for (auto &l : g_srv.lanes) {
        l.cv.notify_all();
        if (l.th.joinable()) l.th.join();
    }
    for (cudaStream_t s : g_srv.streams) cudaStreamDestroy(s);
    g_srv.streams.clear();
    std::lock_guard<std::mutex> lk(g_srv.mu);
    g_srv.jobs.clear();
    g_srv.running = false;
    g_srv.stopping = false;
    g_srv.workers_done = false;
    return DM_OK;
}

int dm_submit(const dm_request *r, dm_ticket *t) {
    if (!t) return dm_fail_msg(DM_EINVAL, "ticket pointer is NULL");
    if (!valid_request(r)) return dm_fail_msg(DM_EINVAL, "invalid request (sizes, k, ranks, tolerances)");
    auto j = std::make_unique<Job>();
    j->req = *r;
    j->points.assign(r->points, r->points + (size_t)r->N * (size_t)r->d);
    j->req.points = nullptr;
    j->bytes = dm_request_bytes(r);
    std::lock_guard<std::mutex> lk(g_srv.mu);
    if (!g_srv.running || g_srv.stopping) return dm_fail_msg(DM_ESTATE, "server not running");
    if ((int)g_srv.queue.size() >= g_srv.capacity) return dm_fail_msg(DM_EBUSY, "request queue full");
    j->id = g_srv.next_id++;
    j->res.submit_ms = g_srv.now_ms();
    j->res.error = j->error.c_str();
    *t = j->id;
    g_srv.queue.push_back(j.get());
    g_srv.jobs[j->id] = std::move(j);
    g_srv.cv.notify_all();
    return DM_OK;
}

int dm_poll(dm_ticket t, dm_result *r, int32_t *done) {
    std::lock_guard<std::mutex> lk(g_srv.mu);
    auto it = g_srv.jobs.find(t);
    if (it == g_srv.jobs.end()) return dm_fail_msg(DM_EINVAL, "unknown ticket");
    const bool fin = it->second->state == kDone;
    if (done) *done = fin ? 1 : 0;
    if (fin && r) *r = it->second->res;
    return DM_OK;
}

int dm_release(dm_ticket t) {
    std::lock_guard<std::mutex> lk(g_srv.mu);
    auto it = g_srv.jobs.find(t);
    if (it == g_srv.jobs.end()) return dm_fail_msg(DM_EINVAL, "unknown ticket");
    if (it->second->state != kDone) return dm_fail_msg(DM_EBUSY, "request still queued or running");
    g_srv.jobs.erase(it);
    return DM_OK;
}

}  // extern "C"
