// Allocation-free FP64 field sum (lbm_field_sum_noalloc, declared in include/lbm.h).
//
// Some callers cannot allocate device memory at the moment they need a reduction: code that
// runs inside a memory-pool-managed framework which forbids cudaMalloc outside its allocator,
// plug-ins running with a fixed device-memory budget, or sections that must not allocate for
// latency reasons.  This entry point serves them: the caller passes the input field and gets the
// sum back, and the working memory the reduction needs (per-block partial sums, the last-block
// ticket and the result) is a file-scope device array, reserved when the library is loaded and
// kept on every GPU that loads the library until the process exits.
//
// The reduction is the same deterministic two-level scheme as the library's other FP64 sums:
// each block adds its elements in a fixed order and writes its partial; the block that finishes
// last (atomic ticket) adds the partials in index order.  The result therefore depends only on
// the input and the grid size, which is fixed by the input length.
#include <mutex>
#include <stdint.h>
#include <stdio.h>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/lbm.h"

// error message of lbm_last_error (defined with the rest of the C-ABI)
extern "C" void gb300lbm_set_error(const char* msg);

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 1024;   // capacity of the scratch array in block partials

// Scratch layout (all 256-byte aligned inside the array):
//   [0, kMaxBlocks)    double2 block partials (sum, 0)
//   kMaxBlocks         double2 result
//   kMaxBlocks + 1     unsigned ticket (first 4 bytes of the slot)
struct Scratch {
    double2 partial[kMaxBlocks];
    double2 result;
    unsigned ticket;
    unsigned pad[3];
};
static __device__ __align__(256) Scratch g_noalloc_scratch;

__global__ void __launch_bounds__(kThreads) k_field_sum_noalloc(const float* __restrict__ a, long long n,
                                                               Scratch* sc) {
    __shared__ double s[kThreads / 32];
    __shared__ int is_last;
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads)
        acc += (double)a[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += s[w];
        sc->partial[blockIdx.x] = make_double2(t, 0.0);
        __threadfence();
        is_last = atomicAdd(&sc->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double t = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += kThreads) t += __ldcg(&sc->partial[k]).x;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) r += s[w];
        sc->result = make_double2(r, 0.0);
        sc->ticket = 0u;
    }
}

// Device address of the scratch array, looked up once per device with that device current.
// (In host code the array's name is only a host-side handle, never a device address.)
std::mutex g_mu;
void* g_scratch_addr[128] = {nullptr};

int scratch_for_current_device(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
        gb300lbm_set_error("lbm_field_sum_noalloc: no usable current device");
        return LBM_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            gb300lbm_set_error("lbm_field_sum_noalloc: cudaGetSymbolAddress of the scratch array failed");
            return LBM_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return LBM_OK;
}

// The input must be device (or managed) memory of the current device, and the n floats from
// `field` must lie inside one allocation: a host pointer, another GPU's pointer or a range past
// the end of the buffer would make the kernel read memory it does not own.  The allocation's
// extent comes from the driver (cuMemGetAddressRange); where that query is unavailable only the
// pointer's kind and device are checked.
typedef CUresult (*AddressRangeFn)(CUdeviceptr*, size_t*, CUdeviceptr);

int check_field(const float* field, long long n) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        gb300lbm_set_error("lbm_field_sum_noalloc: no usable current device");
        return LBM_ECUDA;
    }
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, field) != cudaSuccess) {
        cudaGetLastError();
        gb300lbm_set_error("lbm_field_sum_noalloc: field is not a pointer the CUDA runtime knows");
        return LBM_EINVAL;
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) {
        gb300lbm_set_error("lbm_field_sum_noalloc: field must be device or managed memory, not host memory");
        return LBM_EINVAL;
    }
    if (at.type == cudaMemoryTypeDevice && at.device != dev) {
        char m[160];
        snprintf(m, sizeof(m), "lbm_field_sum_noalloc: field lives on device %d, the current device is %d", at.device,
                 dev);
        gb300lbm_set_error(m);
        return LBM_EINVAL;
    }
    static AddressRangeFn range_fn = nullptr;
    static bool looked_up = false;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!looked_up) {
            void* fn = nullptr;
            cudaDriverEntryPointQueryResult q;
            if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &fn, 12000, cudaEnableDefault, &q) ==
                    cudaSuccess &&
                q == cudaDriverEntryPointSuccess)
                range_fn = (AddressRangeFn)fn;
            cudaGetLastError();
            looked_up = true;
        }
    }
    if (range_fn) {
        CUdeviceptr base = 0;
        size_t size = 0;
        if (range_fn(&base, &size, (CUdeviceptr)(uintptr_t)field) == CUDA_SUCCESS) {
            const unsigned long long begin = (unsigned long long)(uintptr_t)field;
            const unsigned long long end = begin + 4ull * (unsigned long long)n;
            if (end > (unsigned long long)base + size) {
                char m[200];
                snprintf(m, sizeof(m),
                         "lbm_field_sum_noalloc: %lld floats run %llu bytes past the end of the allocation holding "
                         "field",
                         n, end - ((unsigned long long)base + size));
                gb300lbm_set_error(m);
                return LBM_EINVAL;
            }
        }
    }
    return LBM_OK;
}

int cuda_fail(const char* what, cudaError_t e) {
    char m[200];
    snprintf(m, sizeof(m), "lbm_field_sum_noalloc: %s: %s", what, cudaGetErrorString(e));
    gb300lbm_set_error(m);
    return LBM_ECUDA;
}

}  // namespace

extern "C" int lbm_field_sum_noalloc(const float* field, long long n, double* sum_out, void* cuda_stream) {
    if (!sum_out || n < 0 || (n > 0 && !field)) {
        gb300lbm_set_error("lbm_field_sum_noalloc: NULL pointer or negative n");
        return LBM_EINVAL;
    }
    if (n > LBM_NOALLOC_MAX_ELEMENTS) {
        char m[160];
        snprintf(m, sizeof(m), "lbm_field_sum_noalloc: n = %lld exceeds the maximum of %lld elements", n,
                 (long long)LBM_NOALLOC_MAX_ELEMENTS);
        gb300lbm_set_error(m);
        return LBM_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the call synchronises its stream and copies the result to pageable host memory, so it can
    // never be part of a captured graph; made during a capture it would invalidate the capture
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return cuda_fail("cudaStreamIsCapturing", e);
    if (cap != cudaStreamCaptureStatusNone) {
        gb300lbm_set_error("lbm_field_sum_noalloc: the stream is being captured; call it outside stream capture");
        return LBM_ESTATE;
    }
    if (n == 0) {
        *sum_out = 0.0;
        return LBM_OK;
    }
    int rc = check_field(field, n);
    if (rc != LBM_OK) return rc;
    void* p = nullptr;
    rc = scratch_for_current_device(&p);
    if (rc != LBM_OK) return rc;
    Scratch* sc = (Scratch*)p;
    // the ticket is zero here: it starts at zero and every completed launch resets it
    long long blocks = (n + kThreads - 1) / kThreads;
    if (blocks > kMaxBlocks) blocks = kMaxBlocks;
    k_field_sum_noalloc<<<(unsigned)blocks, kThreads, 0, st>>>(field, n, sc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("kernel launch", e);
    double2 r;
    e = cudaMemcpyAsync(&r, &sc->result, sizeof(r), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail("result copy", e);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail("stream synchronisation", e);
    *sum_out = r.x;
    return LBM_OK;
}
