// nao_integrate_h_noalloc: the FP64 Hamiltonian integration with its evaluation scratch in a
// fixed, file-scope device array instead of memory obtained from cudaMalloc.
//
// Some callers cannot allocate device memory at the point where they integrate: an
// application whose own memory manager owns all device memory, or a latency-bound loop that
// must not call cudaMalloc/cudaFree (which can synchronise the device). This entry point
// makes no allocation of any kind: it evaluates the basis functions into the static array
// below and runs the same evaluation and contraction kernels as nao_integrate_h with NAO_FP64.
//
// Limits and sharing:
//   - the array holds NAO_NOALLOC_SCRATCH_BYTES; the handle's evaluation chunks must fit
//     (create the handle with options.scratch_bytes <= NAO_NOALLOC_SCRATCH_BYTES), otherwise
//     the call fails with NAO_ERR_INVALID_ARG and enqueues nothing;
//   - every GPU that loads the library holds the array until the process exits;
//   - all calls on a device share the one array and it keeps the last call's contents:
//     the evaluation kernel writes every entry the contraction later reads (padding
//     included), so nothing has to be cleared; H_dev is zeroed by the call itself;
//   - the call writes the handle's device pointer table (H, v) like every other call on the
//     handle;
//   - calls whose work overlaps on the GPU (other streams, other handles) race on the array;
//   - the first call on a device looks up the array's device address (cudaGetSymbolAddress,
//     with that device current); make that first call before any stream capture. The address
//     is cached for the life of the process: a device reset (or a new primary context) can move
//     the array, after which this entry point must not be called on that device again.
#include <mutex>
#include <string>

#include "nao_internal.h"

namespace {

constexpr size_t kNoallocDoubles = NAO_NOALLOC_SCRATCH_BYTES / sizeof(double);

static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[kMaxDevices] = {};

nao_status noalloc_fail(nao_status s, const std::string &msg) {
    nao_set_last_error(msg);
    return s;
}

// Device address of the array on the current device (looked up once per device).
nao_status noalloc_address(int dev, double **out) {
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(NAO_ERR_UNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return noalloc_fail(NAO_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        }
        g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return NAO_OK;
}

}  // namespace

extern "C" nao_status nao_integrate_h_noalloc(nao_grid *g, const double *v_dev, uint32_t terms, double *H_dev,
                                              void *cuda_stream) {
    if (!g) return noalloc_fail(NAO_ERR_INVALID_ARG, "handle is NULL");
    if (g->n_sys != 1) return noalloc_fail(NAO_ERR_INVALID_ARG, "the handle holds more than one system");
    if (!H_dev) return noalloc_fail(NAO_ERR_INVALID_ARG, "H_dev is NULL");
    if (terms == 0 || (terms & ~3u)) return noalloc_fail(NAO_ERR_INVALID_ARG, "bad terms");
    if ((uint64_t)g->scratch_elems > (uint64_t)kNoallocDoubles)
        return noalloc_fail(NAO_ERR_INVALID_ARG,
                            "the handle's evaluation chunks need " + std::to_string(g->scratch_elems * 8) +
                                " bytes of scratch; nao_integrate_h_noalloc holds " +
                                std::to_string(NAO_NOALLOC_SCRATCH_BYTES) +
                                " (create the handle with options.scratch_bytes <= NAO_NOALLOC_SCRATCH_BYTES)");
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return noalloc_fail(NAO_ERR_CUDA, "cudaGetDevice failed");
    if (prev != g->device && cudaSetDevice(g->device) != cudaSuccess) return noalloc_fail(NAO_ERR_CUDA, "cudaSetDevice failed");
    double *scratch = nullptr;
    nao_status st = noalloc_address(g->device, &scratch);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaSuccess;
    if (st == NAO_OK) {
        // this call's H and v pointers, into the handle's device pointer table (written by a
        // kernel that carries the values in its arguments; no allocation)
        const size_t n = (size_t)g->n_sys;
        g->h_tab[0] = H_dev;
        g->h_tab[n] = const_cast<double *>(v_dev);
        e = launch_set_pointers(g->d_tab, g->h_tab.data(), 1, s);
        if (e == cudaSuccess) e = launch_set_pointers(g->d_tab + n, g->h_tab.data() + n, 1, s);
    }
    if (st == NAO_OK && e == cudaSuccess) e = launch_zero_h(g->sys, g->d_zero_tasks, (int32_t)g->zero_tasks.size(), s);
    for (size_t c = 0; st == NAO_OK && e == cudaSuccess && c < g->chunks.size(); c++) {
        const Chunk &ch = g->chunks[c];
        e = launch_eval(g->sys, ch.b0, ch.b1, NAO_FP64, true, scratch, s);
        if (e == cudaSuccess)
            e = launch_h_simt(g->sys, NAO_FP64, g->d_hwork + ch.hw0, ch.hw1 - ch.hw0, scratch, terms, s);
    }
    if (st == NAO_OK && e == cudaSuccess)
        e = launch_mirror(g->sys, g->d_mirror_tasks, (int32_t)g->mirror_tasks.size(), s);
    if (st == NAO_OK && e == cudaSuccess) {
        e = cudaEventRecord(g->ev_last, s);  // the end of this call's work, for destroy and sync
        if (e == cudaSuccess) g->used = true;
    }
    if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
    if (st != NAO_OK) return st;
    if (e != cudaSuccess) return noalloc_fail(NAO_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return NAO_OK;
}
