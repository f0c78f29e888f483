// fs_amplitudes_noalloc: the amplitude evaluation of fs_amplitudes for
// callers that cannot allocate device memory -- for instance code running
// where every device allocation must go through a pool it does not own, or
// inside a plugin that must not grow the process's device footprint at call
// time.  Instead of cudaMalloc it uses one file-scope device array of
// FS_NOALLOC_SCRATCH_BYTES bytes as the whole device workspace (programs,
// bit strings, checkpoint table, partial sums, counters and the staged
// amplitudes).  The array exists once per device that loads this module and
// stays allocated until the process exits.
#include <cstdio>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/feynsparse.h"
#include "fs_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_scratch[FS_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_scratch_dev[MAX_DEVICES] = {};   // device address of g_scratch, per device

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// The host-side name g_scratch is only a stand-in for the device array; its
// device address comes from cudaGetSymbolAddress, taken once per device with
// that device current.
int scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fs::set_error(FS_ERR_CUDA, "cudaGetDevice failed");
    if (dev < 0 || dev >= MAX_DEVICES) return fs::set_error(FS_ERR_INVALID, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return fs::set_error(FS_ERR_CUDA, "cudaGetSymbolAddress of the static scratch array failed");
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return FS_OK;
}

}  // namespace

extern "C" FS_API int fs_amplitudes_noalloc(fs_circuit* c, const uint64_t* outputs, size_t n_out,
                                            double eps, double* amp_out, void* stream)
{
    if (!c || (n_out && (!outputs || !amp_out))) return fs::set_error(FS_ERR_INVALID, "NULL argument");
    if (n_out == 0) return FS_OK;
    void* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    fs_batch* b = nullptr;
    rc = fs_batch_create(&b);
    if (rc) return rc;
    fs::batch_forbid_host_alloc(b);
    size_t ws = 0;
    // keep the autotuned checkpoint table (and the live list of pruned
    // requests) inside a quarter of the scratch, and the per-item partial or
    // subtree sums (16 B each) inside another quarter
    fs_options opt = {};
    opt.table_budget_bytes = FS_NOALLOC_SCRATCH_BYTES / 4;
    opt.max_items = FS_NOALLOC_SCRATCH_BYTES / 4 / 16;
    // the precompiled kernels: the generated engine would load a freshly
    // compiled module onto the device, which allocates
    opt.engine = 1;
    rc = fs_batch_set_options(b, &opt);
    if (!rc) rc = fs_batch_add(b, c, outputs, n_out, eps, nullptr);
    if (!rc) rc = fs_batch_plan(b, &ws);
    const size_t amp_off = align256(ws);
    const size_t need = amp_off + 2 * sizeof(double) * n_out;
    if (!rc && need > (size_t)FS_NOALLOC_SCRATCH_BYTES) {
        char msg[200];
        snprintf(msg, sizeof msg, "request needs %zu bytes of device scratch; the static scratch of "
                 "fs_amplitudes_noalloc holds %zu bytes (use fs_amplitudes or a batch instead)",
                 need, (size_t)FS_NOALLOC_SCRATCH_BYTES);
        rc = fs::set_error(FS_ERR_TOO_LARGE, msg);
    }
    unsigned char* base = (unsigned char*)scratch;
    cudaStream_t s = (cudaStream_t)stream;
    if (!rc) rc = fs_batch_upload(b, base, ws, stream);
    if (!rc) rc = fs_batch_run(b, base, (double*)(base + amp_off), stream);
    if (!rc) rc = fs_batch_finish(b, base, stream, nullptr, 0);
    if (!rc) {
        if (cudaMemcpyAsync(amp_out, base + amp_off, 2 * sizeof(double) * n_out,
                            cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            rc = fs::set_error(FS_ERR_CUDA, "copy of the amplitudes to the host failed");
    }
    fs_batch_destroy(b);
    return rc;
}
