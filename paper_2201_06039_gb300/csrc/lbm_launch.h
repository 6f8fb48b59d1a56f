// Host-side launchers of the lattice kernels (internal to the library; the public
// C-ABI is include/lbm.h).
#pragma once
#include <cuda_runtime.h>
#include "lbm_device.cuh"

namespace gb300lbm {

// Device buffers of one lattice state (populations are structure-of-arrays).
struct StateBufs {
    const void* fsrc;      // populations read this step
    const void* gsrc;
    void* fdst;            // populations written this step
    void* gdst;
    int pull_f, pull_g;    // 0: state is post-streaming at the node (right after init)
    float2* psirho;        // per node (psi, rho)
    float* phis;           // phi_s history, read and rewritten in place
    double2* partial;      // per-block partial sums of the deterministic reduction
    unsigned* counter;     // last-block counter of the reduction (kept at 0 between launches)
    int* flag;             // non-finite flag
};

int reduce_blocks_psi(const DevParams& P);

cudaError_t launch_init(const DevParams& P, int precision, void* f, void* g, const float* rho,
                        const float* T, const float* u, cudaStream_t s);

// psi/EOS pass: rho, T, psi of every node; optional FP64 sums (rho, T) into sums[0..1].
cudaError_t launch_psi(const DevParams& P, int precision, const StateBufs& B, double* sums,
                       cudaStream_t s);

// stream-collide pass of the two-pass variant.
cudaError_t launch_collide(const DevParams& P, int precision, const StateBufs& B,
                           const double* sums_cur, int first, cudaStream_t s);

// fused z-marching variant (psi of the tile halo recomputed from the populations).
cudaError_t launch_fused(const DevParams& P, int precision, const StateBufs& B,
                         const double* sums_cur, double* sums_next, int first, cudaStream_t s);
bool fused_supported(const DevParams& P);

// macroscopic moments (needs the psi pass on the same state first).
cudaError_t launch_moments(const DevParams& P, int precision, const StateBufs& B,
                           const double* sums_cur, float* rho, float* ux, float* uy, float* uz,
                           float* T, cudaStream_t s);

// deterministic FP64 sum of a float field into out[0] (out[1] = 0).
cudaError_t launch_sum_field(const float* a, int n, double2* partial, unsigned* counter,
                             double* out, cudaStream_t s);

int max_partials(const DevParams& P);

}  // namespace gb300lbm
