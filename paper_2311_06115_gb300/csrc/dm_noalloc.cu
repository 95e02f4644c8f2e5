// dm_noalloc.cu -- degree vectors without any device allocation.
//
// Some callers cannot let a library call cudaMalloc: code that runs under a
// framework which owns every byte of device memory and forbids side
// allocations, services whose memory budget is fixed up front, and callers
// that must not take cudaMalloc's implicit device-wide synchronisation on a hot
// path. dm_degrees_noalloc serves them: it computes the same q, dg and s as
// dm_create into buffers the caller owns, and keeps its intermediate arrays in
// the fixed scratch array below instead of allocating.
#include <mutex>

#include "dm_internal.cuh"

namespace {

// Scratch of dm_degrees_noalloc. It is a module-scope device array, so every GPU
// that loads this library holds it until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array, looked up once per device with that
// device current. In host code the array's name is only a host-side stand-in.
// The cached address belongs to the device's primary context as it was at the
// first call: after cudaDeviceReset (which reloads this module) it is stale, so
// a process that resets a device must not call dm_degrees_noalloc on it again.
std::mutex g_scratch_mu;
void *g_scratch_addr[256];

int scratch_for_current_device(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return DM_ECUDA;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return DM_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return DM_OK;
}

// 1: device (or managed) memory of device `dev`; 0: host memory or unknown; -1: device
// memory of another GPU (its kernels would make peer or illegal accesses).
int on_device(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (a.type == cudaMemoryTypeManaged) return 1;
    if (a.type != cudaMemoryTypeDevice) return 0;
    return a.device == dev ? 1 : -1;
}

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

size_t dm_noalloc_scratch_need(int64_t N, int d) {
    // pre-scaled points (FP32), q^-alpha (FP64 and FP32), s (FP32)
    return align256(sizeof(float) * (size_t)N * d) + align256(sizeof(double) * (size_t)N) +
           align256(sizeof(float) * (size_t)N) + align256(sizeof(float) * (size_t)N);
}

extern "C" int dm_degrees_noalloc(const float *points, int64_t N, int32_t d, double eps, double alpha, double *q,
                                  double *dg, double *s, void *stream) {
    if (!points || !q || !dg || !s) return dm_fail_msg(DM_EINVAL, "dm_degrees_noalloc: NULL pointer");
    if (N < 2 || d < 1 || !(eps > 0.0) || !(alpha >= 0.0))
        return dm_fail_msg(DM_EINVAL, "dm_degrees_noalloc: needs N >= 2, d >= 1, eps > 0, alpha >= 0");
    if (dm_noalloc_scratch_need(N, d) > kNoAllocScratchBytes)
        return dm_fail_msg(DM_EINVAL, "dm_degrees_noalloc: N * (4 d + 16) bytes exceed the 16 MiB scratch array");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return dm_fail_msg(DM_ECUDA, "dm_degrees_noalloc: no current device");
    int where[4] = {on_device(points, dev), on_device(q, dev), on_device(dg, dev), on_device(s, dev)};
    for (int w : where) {
        if (w == 0) return dm_fail_msg(DM_EINVAL, "dm_degrees_noalloc: points, q, dg and s must be device memory");
        if (w < 0)
            return dm_fail_msg(DM_EINVAL,
                               "dm_degrees_noalloc: a buffer is on another device than the current one");
    }
    void *base = nullptr;
    if (scratch_for_current_device(&base) != DM_OK)
        return dm_fail_msg(DM_ECUDA, "dm_degrees_noalloc: cudaGetSymbolAddress of the scratch array failed");
    unsigned char *b = static_cast<unsigned char *>(base);
    float *Xs = reinterpret_cast<float *>(b);
    b += align256(sizeof(float) * (size_t)N * d);
    double *qa = reinterpret_cast<double *>(b);
    b += align256(sizeof(double) * (size_t)N);
    float *qaf = reinterpret_cast<float *>(b);
    b += align256(sizeof(float) * (size_t)N);
    float *sf = reinterpret_cast<float *>(b);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // every scratch word read below is written first in this call; q and dg are
    // zeroed by the degree passes themselves
    if (dm_launch_scale_points(points, N, d, eps, Xs, st) != cudaSuccess ||
        dm_launch_degree_pass(Xs, N, d, nullptr, q, st) != cudaSuccess ||
        dm_launch_finish_degrees(N, alpha, q, qa, qaf, st) != cudaSuccess ||
        dm_launch_degree_pass(Xs, N, d, qaf, dg, st) != cudaSuccess ||
        dm_launch_finish_scaling(N, qa, dg, s, sf, st) != cudaSuccess)
        return dm_fail_msg(DM_ECUDA, "dm_degrees_noalloc: kernel launch failed");
    return DM_OK;
}
