// lw_noalloc.cu -- lw_cluster_noalloc: the merge kernel without any allocation.
//
// Some callers cannot allocate device memory at the moment they want a
// clustering: code running under a memory pool or arena that forbids
// cudaMalloc/cudaFree (allocation can synchronise the device or fail
// mid-run), plug-ins inside a host application that owns all allocations,
// and real-time loops that must not call the allocator at all.  This entry
// point serves them: the caller passes its own device buffers for the
// matrix and the outputs, and the kernel's global scratch (cluster sizes,
// per-CTA exchange records and pair minima, refill lists, barrier, status
// and counter words) lives in one file-scope __device__ array of fixed size.
// The array comes into being on a device when the library's device code is
// loaded there -- with CUDA's lazy module loading, during the first call on
// that device -- and stays until the process exits.  The row caches live in
// shared memory.  The working matrix is the caller's packed triangle (the
// row-log layout would need memory of its own).
//
// Nothing here calls cudaMalloc, cudaFree, cudaMallocHost or any allocating
// library routine.  Each call looks the array's device address up with
// cudaGetSymbolAddress (see include/lw.h for the rules that follow).

#include "../../include/lw.h"
#include "lw_internal.h"


namespace {

// Largest n this entry point accepts and the scratch that serves it
// (workspace_layout): cluster sizes 4n B; per CTA a 240 B record and 512 B of
// pair minima; 16 KB of refill lists; barrier, status and counter words.  At
// n = 16384 on a 256-CTA grid that is about 275 KB; the array holds 2 MB,
// and every call checks its layout against that size.
constexpr long long kNoAllocMaxN = LW_NOALLOC_MAX_N;
constexpr size_t kScratchBytes = 2 * 1024 * 1024;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch on the current device.  In host code
// `g_scratch` names a host-side stand-in, not device memory, so it is never
// passed to a kernel directly.  The address is looked up on every call (it
// allocates nothing, and stays right after a device reset reloads the module).
cudaError_t scratch_address(void **out)
{
    return cudaGetSymbolAddress(out, g_scratch);
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
    if (cudaGetDevice(&device) != cudaSuccess ||
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
    if (scratch_address(&base) != cudaSuccess) {
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
    lw::check_range(p, dist, (unsigned long long)n * (unsigned long long)(n - 1) / 2 * sizeof(float));
    lw::check_range(p, merges_out, 8ull * (unsigned long long)(n - 1));
    lw::check_range(p, heights_out, 4ull * (unsigned long long)(n - 1));
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
