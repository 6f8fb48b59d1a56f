// Host-side launchers of the lattice kernels (internal to the library; the public
// C-ABI is include/lbm.h).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include "lbm_device.cuh"

namespace gb300lbm {

// Device buffers of one lattice state (populations are structure-of-arrays).
struct StateBufs {
    const void* src;       // populations read this step (26 slots: f and g, see fslot / gslot)
    void* dst;             // populations written this step
    int src_index;         // which of the two population buffers src is (tensor maps are per buffer)
    int pull_f, pull_g;    // 0: state is post-streaming at the node (right after init)
    float2* psirho;        // per node (psi, rho)
    float* phis;           // phi_s history, read and rewritten in place
    double2* partial;      // per-block partial sums of the deterministic reduction
    unsigned* counter;     // last-block counter of the reduction (kept at 0 between launches)
    int* flag;             // non-finite flag
    float4* vel;           // per node u (finite-difference div u only; NULL otherwise)
};

int reduce_blocks_psi(const DevParams& P);

cudaError_t launch_init(const DevParams& P, int precision, void* pops, const float* rho, const float* T,
                        const float* u, cudaStream_t s);

// psi/EOS pass: rho, T, psi of every node; optional FP64 sums (rho, T) into sums[0..1].
cudaError_t launch_psi(const DevParams& P, int precision, const StateBufs& B, double* sums,
                       cudaStream_t s);

// stream-collide pass of the two-pass variant.
// u = (sum e f + F/2) / rho of every node into B.vel (finite-difference div u)
cudaError_t launch_wall_params(const DevParams& P, float2* par, cudaStream_t s);
cudaError_t launch_wall_map(const DevParams& P, const float* phi, const float* drho, float2* par, int* bad,
                            int write, cudaStream_t s);
cudaError_t launch_wall_table(const DevParams& P, int precision, const void* fs, int pull_f, float2* tab,
                              cudaStream_t s);
cudaError_t launch_velocity(const DevParams& P, int precision, const StateBufs& B, const double* sums_cur,
                            cudaStream_t s);
cudaError_t launch_collide(const DevParams& P, int precision, const StateBufs& B,
                           const double* sums_cur, int first, cudaStream_t s);

// Tensor maps of the two population buffers for the TMA variant: the load windows (4D x, y, z,
// slot; boxes (TX + 2 * 16 bytes of columns) x (TY + 4) x 1 x 14 and x 6 over the padded storage) and the output tile
// (4D x, slot, y, z over the real nodes only; boxes TX x 26 x TY x 1, and TX x 26 x (rows of the
// last tile row) x 1 in mout_top); and the number of SMs for its persistent grid.
struct TmaMaps {
    CUtensorMap m14[2], m6[2], mout[2], mout_top[2];
    // ghost stores (4D x, slot, y, z over the whole padded plane): edge-column box gw x 26 x TY (and
    // x rows of the last tile row), edge-row box TX x 26 x 2 (and x columns of the last tile
    // column), corner box gw x 26 x 2, gw = 16 bytes of columns
    CUtensorMap mgcol[2], mgcol_top[2], mgrow[2], mgrow_right[2], mgcor[2];
    // ghost cells after a TMA step: 1 the edge tiles store them by TMA, 2 the edge nodes store their
    // periodic images directly (FP32 lattices whose nx is no multiple of the 16-byte band, or with
    // one tile across an axis), 0 the refresh kernel writes them
    int ghosts;
    bool ok;
    int sms;
    int shape, zchunk, items;   // plan of tma_plan_for
};

// Tensor maps and plan of the TMA kernel for one lattice whose two population buffers start at
// buf0 / buf1: the tile shape and z-chunk of tma_plan_for (forced_shape / forced_zchunk >= 0 / > 0
// pin them; the model spreads the items over model_ctas persistent CTAs, the device's SM count if
// <= 0).  false (maps->ok false) if the lattice does not qualify, the shape does not fit the
// device, or the plan has more than max_items items (the capacity of the caller's partial-sum
// buffer).
bool build_tma_maps(const DevParams& d, int precision, void* buf0, void* buf1, int model_ctas, int forced_shape,
                    int forced_zchunk, int max_items, TmaMaps* maps);

// fused z-marching variant (psi of the tile halo recomputed from the populations); uses the
// TMA kernel when maps are given and the lattice / state qualify (see tma_eligible).
// *ghosts_written (nullable) tells whether the launch also refreshed the ghost cells of dst.
cudaError_t launch_fused(const DevParams& P, int precision, const StateBufs& B, const double* sums_cur,
                         double* sums_next, int first, cudaStream_t s, const TmaMaps* maps,
                         bool* ghosts_written = nullptr);
bool fused_supported(const DevParams& P);
// CTAs (partial sums) of one generic fused launch on P
long long fused_blocks(const DevParams& P);
bool tma_eligible(const DevParams& P, int precision);
// refresh the ghost columns / rows of a population buffer from their periodic images
cudaError_t launch_ghosts(const DevParams& P, int precision, void* pops, cudaStream_t s);
// tile shapes 0: 32 x 8, 1: 40 x 7, 2: 32 x 12, 3: 24 x 16 (window boxes tma_box_w x tma_box_h per
// population slot)
// forced_shape >= 0 / forced_zchunk > 0 pin the shape / the z-chunk of the plan
void tma_plan_for(const DevParams& P, int ctas, int forced_shape, int forced_zchunk, int* shape, int* zchunk,
                  int* items);
int tma_num_shapes();
// the plan model's node rate of a tile shape (relative to 32 x 8)
double tma_rate(int shape);
// up to max z-chunks of a shape, best modelled first (returns how many)
int tma_zchunk_candidates(const DevParams& P, int ctas, int shape, int* zcs, int max);
size_t tma_smem_bytes(int shape, int precision);
int tma_box_w(int shape, int precision);
int tma_box_h(int shape);
int tma_tile_w(int shape);
int tma_ghost_mode(const DevParams& P, int shape, int precision);
int tma_ghost_cols(int precision);
int tma_tile_h(int shape);

// macroscopic moments (needs the psi pass on the same state first).
cudaError_t launch_moments(const DevParams& P, int precision, const StateBufs& B,
                           const double* sums_cur, float* rho, float* ux, float* uy, float* uz,
                           float* T, cudaStream_t s);

// deterministic FP64 sum of a float field into out[0] (out[1] = 0).
cudaError_t launch_sum_field(const float* a, int n, double2* partial, unsigned* counter,
                             double* out, cudaStream_t s);

int max_partials(const DevParams& P);

// ---------------------------------------------------------------- batched ensemble
// Geometry of one instance (device table).  Instance k owns the elements [pop_off, pop_off + its
// population-buffer size) of each population buffer (same padded layout as a single lattice) and nodes
// [field_off, field_off + N) of the dense fields; its items are item0 .. item0 + n_items - 1.
struct BatchInst {
    int nx, ny, nz, Ws, Hs;
    int item0, n_items, pad_;
    long long pop_off, field_off;
    double inv_N;
};
// One work item: tile column (x0, y0) of 32 x TY nodes, planes [z0, z1) of instance inst.
struct BatchItem {
    int inst, x0, y0, z0, z1, pad_;
};
// Batched fused update.  B.counter points at two unsigned counters (work, ticket) that must be
// zero before the first launch (every launch leaves them at zero); B.partial holds one double2
// per item; sums_cur / sums_next hold (sum rho, sum T) per instance.  ty: tile rows (4 or 8).
cudaError_t launch_fused_batch(const DevParams& P, int precision, int ty, const BatchInst* insts,
                               const BatchItem* items, int n_items, int n_inst, const StateBufs& B,
                               const double* sums_cur, double* sums_next, int first, int ctas, cudaStream_t s);
// resident CTAs per SM of the batched kernel (0 if it cannot launch)
int batch_ctas_per_sm(int precision, int ty);
int batch_tile_rows(int ty);

}  // namespace gb300lbm
