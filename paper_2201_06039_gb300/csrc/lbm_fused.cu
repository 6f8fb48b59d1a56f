// Fused z-marching variant of the lattice update (one kernel per step).
#include "lbm_launch.h"

namespace gb300lbm {

bool fused_supported(const DevParams&) { return false; }

cudaError_t launch_fused(const DevParams&, int, const StateBufs&, const double*, double*, int, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace gb300lbm
