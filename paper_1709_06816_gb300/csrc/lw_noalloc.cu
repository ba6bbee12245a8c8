// lw_noalloc.cu -- lw_cluster_noalloc: the merge kernel without any allocation.
//
// Some callers cannot allocate device memory at the moment they want a
// clustering: code running under a memory pool or arena that forbids
// cudaMalloc/cudaFree (allocation can synchronise the device or fail
// mid-run), plug-ins inside a host application that owns all allocations,
// and real-time loops that must not call the allocator at all.  This entry
// point serves them: the caller passes its own device buffers for the
// matrix and the outputs, and the kernel's scratch (row-minimum keys,
// cluster sizes, exchange records, barrier and status words) lives in one
// file-scope __device__ array of fixed size, allocated once when the library
// is loaded on a device and kept until the process exits.
//
// Nothing here calls cudaMalloc, cudaFree, cudaMallocHost or any allocating
// library routine.  The only set-up is cudaGetSymbolAddress on the first call
// per device (see include/lw.h for the rules that follow from that).

#include "../../include/lw.h"
#include "lw_internal.h"

#include <mutex>

namespace {

// Largest n this entry point accepts and the scratch that serves it: cluster
// sizes 4n, per-CTA records and refill lists (about 8.5 KB per CTA of a
// full-device grid), barrier, status and stats words.
constexpr long long kNoAllocMaxN = LW_NOALLOC_MAX_N;
constexpr size_t kScratchBytes = 2 * 1024 * 1024;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device (first call per device
// looks it up).  In host code `g_scratch` names a host-side stand-in, not
// device memory, so it is never passed to a kernel directly.
cudaError_t scratch_address(int device, void **out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess)
            return e;
        g_scratch_ptr[device] = p;
    }
    *out = g_scratch_ptr[device];
    return cudaSuccess;
}

bool is_device_memory(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" lw_status lw_cluster_noalloc(float *dist, int64_t n, int linkage, int32_t *merges_out,
                                        float *heights_out, void *cuda_stream)
{
    if (n < 1 || n > kNoAllocMaxN || linkage < LW_SINGLE || linkage > LW_CENTROID)
        return LW_ERR_INVALID_ARG;
    if (n == 1)
        return LW_OK;
    if (!dist || !merges_out || !heights_out || !is_device_memory(dist) ||
        !is_device_memory(merges_out) || !is_device_memory(heights_out))
        return LW_ERR_INVALID_ARG;
    int device = 0, num_sms = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices ||
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        return LW_ERR_CUDA;
    }
    // the same grid policy as lw_cluster: one CTA for small matrices, every SM otherwise
    int G = n <= 4096 ? 1 : num_sms;
    const long long nb = (n + lw::kRowBlock - 1) / lw::kRowBlock;
    if (G > nb)
        G = (int)nb;
    while (G < num_sms && !lw::merge_config_ok(n, G, num_sms))
        ++G;
    if (!lw::merge_config_ok(n, G, num_sms))
        return LW_ERR_INVALID_ARG;
    const lw::WorkspaceLayout L = lw::workspace_layout(n, G);
    if (L.total > kScratchBytes)
        return LW_ERR_INVALID_ARG;

    void *base = nullptr;
    if (scratch_address(device, &base) != cudaSuccess) {
        cudaGetLastError();
        return LW_ERR_CUDA;
    }
    char *ws = static_cast<char *>(base);
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

    lw::MergeParams p;
    p.D = dist;
    p.TL = nullptr;
    p.stamp = nullptr;
    p.full = 0;
    p.n = n;
    p.pitch = n;
    p.linkage = linkage;
    p.G = G;
    p.aligned16 = ((uintptr_t)dist & 15u) == 0;
    p.merges = merges_out;
    p.heights = heights_out;
    lw::bind_workspace(p, ws, L);
    p.stats = reinterpret_cast<long long *>(ws + L.stats);
    p.timeout_ns = 5000ull * 1000000ull;
    p.skip_arrive_cta = -1;
    p.timing = 0;

    // the scratch keeps the previous call's contents: the barrier,
    // status and stats words must start at zero
    if (cudaMemsetAsync(ws + L.zero, 0, L.total - L.zero, stream) != cudaSuccess ||
        lw::launch_merge(p, lw::kThreads, stream) != cudaSuccess) {
        cudaGetLastError();
        return LW_ERR_CUDA;
    }
    int status[4] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(status, p.status, sizeof status, cudaMemcpyDeviceToHost, stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess) {
        cudaGetLastError();
        return LW_ERR_CUDA;
    }
    switch (status[0]) {
    case 0: return LW_OK;
    case lw::kErrInput: return LW_ERR_INVALID_INPUT;
    case lw::kErrTimeout: return LW_ERR_TIMEOUT;
    default: return LW_ERR_CUDA;
    }
}
