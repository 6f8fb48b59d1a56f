// Host-side helpers shared by the library's C-ABI translation units (internal).
#pragma once
#include <stddef.h>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/lbm.h"
#include "lbm_device.cuh"

namespace gb300lbm {

// record a printf-style message for lbm_last_error and return status
int fail(int status, const char* fmt, ...);
size_t align256(size_t v);
size_t pop_bytes(int precision);
// T_c of the Peng-Robinson EOS from the rounded constants (Sec. IV.A)
double critical_T(const lbm_params* p);
// LBM_OK or LBM_EINVAL (message recorded) for a parameter set
int validate(const lbm_params* p);
// device-side constants of a parameter set (geometry, storage layout, model constants)
DevParams make_dev(const lbm_params* p);
bool is_device_ptr(const void* ptr);
// elements of one population buffer (all slots, ghost cells and padding included)
inline size_t pop_elems(const DevParams& d) { return (size_t)d.splane * d.nz; }

// NVTX range over the enclosing scope, named for the call (visible in Nsight Systems / Compute
// timelines; a no-op unless a tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace gb300lbm

#define GB300_CK(call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return ::gb300lbm::fail(LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)
