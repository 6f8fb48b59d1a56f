// Fused z-marching variants of the lattice update: one kernel per time step.
//
// A CTA owns a 32 x 8 tile of (x, y) columns and marches through a chunk of z-planes.  For
// every plane it
//   psi pass : pulls the 26 populations of each tile node and of the one-node halo ring around
//              the tile, forms rho = sum f (Eq. 10), T = sum g (Eq. 20) and psi (Eq. 8 with the
//              Peng-Robinson EOS, Eq. 49), and keeps (psi, rho) in a shared-memory plane ring;
//   collision: for the previous plane: interaction force (Eq. 7) and grad rho from the ring,
//              buoyancy, D3Q19 MRT collision (Eqs. 3-6, 9, 10), div u (Eq. 48), grad T (Eq. 45),
//              phi_s (Eq. 18), source Q (Eq. 23), D3Q7 MRT collision (Eqs. 38-43); stores f*,
//              g+ and phi_s.
// psi and rho never go to HBM: the halo ring is recomputed from the populations.  rho_ave of
// the buoyancy force is the deterministic FP64 mean of this step's rho, used by the next step.
//
// k_fused     : generic (any faces, any storage precision, frozen f or g, first step).
// k_fused_tma : FP32 or shifted 16-bit storage, f-periodic x and y faces (any z faces).  A
//               producer warp fetches each plane's pulls for the whole tile + halo with three TMA
//               tensor copies (one per e_z group of population slots) into a multi-stage
//               shared-memory pipeline guarded by mbarriers; psi warps and collision warps read
//               every pull as one shared-memory load at a fixed offset.  FP32 planes leave through
//               TMA tensor stores, 16-bit planes through direct stores of the collision threads.
//               Persistent CTAs take (z-chunk, tile) items round robin.
#include <cuda.h>
#include "lbm_launch.h"

namespace gb300lbm {

namespace {

constexpr int TX = 32;
constexpr int kTY = 8;

template <int TY, int QT = 7> struct FusedShape {
    static constexpr int kInterior = TX * TY;
    static constexpr int kPops = 19 + QT;   // populations of a node (f and the thermal lattice's g)
    static constexpr int kHaloNodes = 2 * (TX + 2) + 2 * TY;
    static constexpr int kHaloThreads = ((kHaloNodes + 31) / 32) * 32;
    static constexpr int kThreads = kInterior + kHaloThreads;
    static constexpr int kRingW = TX + 2, kRingH = TY + 2;
    static constexpr int kRingPlane = kRingW * kRingH;
    static constexpr size_t kStageFloats = (size_t)kPops * kInterior;
    static constexpr size_t kSmemBytes = 2 * kStageFloats * sizeof(float) + 3 * kRingPlane * sizeof(float2);
};

// coordinate of the node whose (psi, rho) fills a ring slot at coordinate c (may be -1 or n):
// wrap for periodic (f) faces, mirror (= clamp for one layer) for walls and outflow faces.
__device__ __forceinline__ int map_coord(int c, int n, int bc_lo, int bc_hi) {
    if (c < 0) return f_wraps(bc_lo) ? c + n : 0;
    if (c >= n) return f_wraps(bc_hi) ? c - n : n - 1;
    return c;
}

// ring slot (lx, ly) of a thread: tile nodes first (one warp per row), then the halo ring
template <int TY>
__device__ __forceinline__ void slot_of(int tid, int& lx, int& ly) {
    using Sh = FusedShape<TY>;
    lx = -1;
    ly = -1;
    if (tid < Sh::kInterior) {
        lx = (tid & 31) + 1;
        ly = (tid >> 5) + 1;
    } else {
        int h = tid - Sh::kInterior;
        if (h < TX + 2) { lx = h; ly = 0; }
        else if (h < 2 * (TX + 2)) { lx = h - (TX + 2); ly = TY + 1; }
        else if (h < Sh::kHaloNodes) { int k = h - 2 * (TX + 2); lx = (k & 1) ? TX + 1 : 0; ly = 1 + (k >> 1); }
    }
}

// interaction force sum_a w psi(x+e) e and grad rho from the (psi, rho) ring planes: each
// neighbour's (psi, rho) pair is added to the (F, grad rho) pair of every axis it lies along with
// one paired FP32 fma (per lane the same rounding as two scalar fmas), in the velocity order of
// Eq. 2 (the two-pass kernels' stencil adds in the same order, so every variant agrees bit for bit)
struct RingStencil {
    float Fx, Fy, Fz, gx, gy, gz;
};
__device__ __forceinline__ RingStencil ring_stencil(const float2* rm, const float2* r0, const float2* rp, int slot,
                                                   int W) {
    float2 ax = make_float2(0.f, 0.f), ay = ax, az = ax;
#define GB300_NB(PL, DX, DY, DZ, WGT)                                                          \
    {                                                                                          \
        const float2 q = PL[slot + (DY) * W + (DX)];                                           \
        if (DX) ax = __ffma2_rn(make_float2((DX) * (WGT), (DX) * (WGT)), q, ax);                 \
        if (DY) ay = __ffma2_rn(make_float2((DY) * (WGT), (DY) * (WGT)), q, ay);                 \
        if (DZ) az = __ffma2_rn(make_float2((DZ) * (WGT), (DZ) * (WGT)), q, az);                 \
    }
    const float w1 = 1.f / 6.f, w2 = 1.f / 12.f;
    GB300_NB(r0, 1, 0, 0, w1) GB300_NB(r0, -1, 0, 0, w1) GB300_NB(r0, 0, 1, 0, w1) GB300_NB(r0, 0, -1, 0, w1)
    GB300_NB(rp, 0, 0, 1, w1) GB300_NB(rm, 0, 0, -1, w1)
    GB300_NB(r0, 1, 1, 0, w2) GB300_NB(r0, -1, -1, 0, w2) GB300_NB(r0, 1, -1, 0, w2) GB300_NB(r0, -1, 1, 0, w2)
    GB300_NB(rp, 1, 0, 1, w2) GB300_NB(rm, -1, 0, -1, w2) GB300_NB(rm, 1, 0, -1, w2) GB300_NB(rp, -1, 0, 1, w2)
    GB300_NB(rp, 0, 1, 1, w2) GB300_NB(rm, 0, -1, -1, w2) GB300_NB(rm, 0, 1, -1, w2) GB300_NB(rp, 0, -1, 1, w2)
#undef GB300_NB
    return RingStencil{ax.x, ay.x, az.x, ax.y, ay.y, az.y};
}

__device__ __forceinline__ void kahan_add(float& sum, float& c, float v) {
    float y = v - c, t = sum + y;
    c = (t - sum) - y;
    sum = t;
}

// barrier 0 = the whole block; other ids = named barrier over the first nthreads threads
__device__ __forceinline__ void sync_threads(int bar_id, int nthreads) {
    if (bar_id == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(nthreads) : "memory");
}

// FP64 sum of (a, b) over the NT threads of the barrier group, written to partial[index]
template <int NT>
__device__ void block_partial(double a, double b, double2* partial, int index, int tid, int bar_id, double* sa,
                              double* sb) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((tid & 31) == 0) { sa[tid >> 5] = a; sb[tid >> 5] = b; }
    sync_threads(bar_id, NT);
    if (tid == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < NT / 32; ++w) { ta += sa[w]; tb += sb[w]; }
        partial[index] = make_double2(ta, tb);
    }
    sync_threads(bar_id, NT);
}

// The last block of the grid to arrive adds partial[0..n) in index order into out[0..1] and
// resets the ticket: the result depends only on the partials, never on block scheduling.
template <int NT>
__device__ void finish_sums(const double2* partial, int n, unsigned* counter, double* out, int tid, int bar_id,
                            double* sa, double* sb, int* is_last) {
    if (tid == 0) {
        __threadfence();
        unsigned ticket = atomicAdd(counter, 1u);
        *is_last = ticket == gridDim.x * gridDim.y * gridDim.z - 1;
    }
    sync_threads(bar_id, NT);
    if (!*is_last) return;
    __threadfence();
    double ta = 0.0, tb = 0.0;
    for (int k = tid; k < n; k += NT) {
        double2 q = __ldcg(partial + k);
        ta += q.x;
        tb += q.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ta += __shfl_down_sync(0xffffffffu, ta, o);
        tb += __shfl_down_sync(0xffffffffu, tb, o);
    }
    if ((tid & 31) == 0) { sa[tid >> 5] = ta; sb[tid >> 5] = tb; }
    sync_threads(bar_id, NT);
    if (tid == 0) {
        double ra = 0.0, rb = 0.0;
        for (int w = 0; w < NT / 32; ++w) { ra += sa[w]; rb += sb[w]; }
        out[0] = ra;
        out[1] = rb;
        *counter = 0u;
    }
}

// ================================================================ generic fused kernel
// One tile column: the (x, y) tile at (x0, y0), planes [z0, z1), by all threads of the block.
// Adds the tile's rho and T to the Kahan pairs (r_sum, r_c), (t_sum, t_c) of the owner threads
// and ORs a non-finite / psi-domain failure into bad.
template <typename S, int TY, bool kWet, int QT = 7>
__device__ __forceinline__ void fused_column(const DevParams& P, const S* __restrict__ src, S* __restrict__ dst,
                                             int pull_f, int pull_g, float rho_ave, float* __restrict__ phis,
                                             int first, int x0, int y0, int z0, int z1, float* stage, float2* ring,
                                             float& r_sum, float& r_c, float& t_sum, float& t_c, int& bad) {
    using Sh = FusedShape<TY, QT>;
    const int tid = threadIdx.x;
    int lx, ly;
    slot_of<TY>(tid, lx, ly);
    const bool interior = tid < Sh::kInterior;
    const int gx = x0 + lx - 1, gy = y0 + ly - 1;
    const bool slot_used = lx >= 0 && gx >= -1 && gx <= P.nx && gy >= -1 && gy <= P.ny;
    const int mx = slot_used ? map_coord(gx, P.nx, P.bc[0], P.bc[1]) : 0;
    const int my = slot_used ? map_coord(gy, P.ny, P.bc[2], P.bc[3]) : 0;
    const bool owner = interior && gx < P.nx && gy < P.ny;
    const int slot = slot_used ? bbase(P, ly * Sh::kRingW + lx, 0, 0, Sh::kRingPlane) : 0;

    auto psi_pass = [&](int zp) {
        if (!slot_used) return;
        if (kWet && zp < 0 && P.wet) {   // solid layer below a wetting -z wall: virtual (psi, rho)
            ring[((zp + 3) % 3) * Sh::kRingPlane + slot] = wall_entry(P, mx, my);
            return;
        }
        const bool in_chunk = zp >= z0 && zp < z1;
        const int mz = map_coord(zp, P.nz, P.bc[4], P.bc[5]);
        const int i = sidx(P, mx, my, mz);
        Nbr n = make_nbr(P, mx, my, mz);
        float f[19], g[QT];
        load_f<S>(P, src, pull_f, i, mx, my, mz, n, f);
        Therm<QT>::template load<S>(P, src, pull_g, i, mx, my, mz, n, g);
        float rho = sum19(f), T = Therm<QT>::sum(g);
        float psi2 = psi_squared(P, rho, T);
        ring[((zp + 3) % 3) * Sh::kRingPlane + slot] = make_float2(psi_of(psi2), rho);
        if (owner && in_chunk) {
            float* st = stage + ((zp - z0) & 1) * Sh::kStageFloats + tid;
#pragma unroll
            for (int a = 0; a < 19; ++a) st[a * Sh::kInterior] = f[a];
#pragma unroll
            for (int a = 0; a < QT; ++a) st[(19 + a) * Sh::kInterior] = g[a];
            kahan_add(r_sum, r_c, rho);
            kahan_add(t_sum, t_c, T);
            bad |= !(psi2 > 0.f) || !isfinite(rho) || !isfinite(T);
        }
    };

    auto collide = [&](int z) {
        if (!owner) return;
        const int x = gx, y = gy;
        const int i = sidx(P, x, y, z), d = (int)bidx(P, node_of(P, x, y, z), P.N);
        const float* st = stage + ((z - z0) & 1) * Sh::kStageFloats + tid;
        float f[19], g[QT];
#pragma unroll
        for (int a = 0; a < 19; ++a) f[a] = st[a * Sh::kInterior];
#pragma unroll
        for (int a = 0; a < QT; ++a) g[a] = st[(19 + a) * Sh::kInterior];
        float rho = sum19(f), T = Therm<QT>::sum(g);
        const float2* rm = ring + ((z + 2) % 3) * Sh::kRingPlane;
        const float2* r0 = ring + (z % 3) * Sh::kRingPlane;
        const float2* rp = ring + ((z + 1) % 3) * Sh::kRingPlane;
        const float2 me = r0[slot];
        RingStencil rs = ring_stencil(rm, r0, rp, bbase(P, slot, -(Sh::kRingW + 1), Sh::kRingW + 1, Sh::kRingPlane),
                                      Sh::kRingW);
        const Forces F = total_force(P, me.x, rs.Fx, rs.Fy, rs.Fz, rho - rho_ave);
        NodeOut o = collide_f(P, f, rho, F.Fx, F.Fy, F.Fz, F.Fm2, me.x * me.x);
        float ph = Therm<QT>::collide(P, g, rho, T, o, rs.gx, rs.gy, rs.gz, phis[d], first);
        // frozen fields keep their stored values (no streaming, no collision)
        if (P.flow_off) {
#pragma unroll
            for (int a = 0; a < 19; ++a)
                f[a] = Codec<S>::load(src + (size_t)fslot(a) * P.Ns + bidx(P, i, P.Nidx), P.shift_f[a]);
        }
        if (P.thermal_off) Therm<QT>::template stored<S>(P, src, i, g);
        Therm<QT>::template store<S>(P, dst, i, f, g);
        phis[d] = ph;
    };

    psi_pass(z0 - 1);
    psi_pass(z0);
    __syncthreads();
    for (int z = z0; z < z1; ++z) {
        psi_pass(z + 1);
        __syncthreads();
        collide(z);
        __syncthreads();
    }
}

template <typename S, int TY, int QT>
__global__ void __launch_bounds__(FusedShape<TY, QT>::kThreads, 2)
k_fused(DevParams P, const S* __restrict__ src, S* __restrict__ dst, int pull_f, int pull_g,
        const double* __restrict__ sums_cur, double2* partial, unsigned* counter, double* sums_next,
        float* __restrict__ phis, int* flag, int first, int zchunk) {
    using Sh = FusedShape<TY, QT>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float* stage = reinterpret_cast<float*>(smem_raw);                       // [2][26][TY][32]
    float2* ring = reinterpret_cast<float2*>(stage + 2 * Sh::kStageFloats);  // [3][TY+2][34]
    __shared__ double red_a[Sh::kThreads / 32], red_b[Sh::kThreads / 32];
    __shared__ int is_last;

    const int tid = threadIdx.x;
    const int z0 = blockIdx.z * zchunk;
    float r_sum = 0.f, r_c = 0.f, t_sum = 0.f, t_c = 0.f;
    int bad = 0;
    const float rho_ave = buoyancy_ref(P, sums_cur[0], P.inv_N);
    fused_column<S, TY, true, QT>(P, src, dst, pull_f, pull_g, rho_ave, phis, first, blockIdx.x * TX, blockIdx.y * TY, z0,
                        min(P.nz, z0 + zchunk), stage, ring, r_sum, r_c, t_sum, t_c, bad);

    if (__syncthreads_or(bad) && tid == 0) atomicOr(flag, 1);
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    block_partial<Sh::kThreads>((double)r_sum - (double)r_c, (double)t_sum - (double)t_c, partial, bid, tid, 0,
                                red_a, red_b);
    finish_sums<Sh::kThreads>(partial, gridDim.x * gridDim.y * gridDim.z, counter, sums_next, tid, 0, red_a, red_b,
                              &is_last);
}

// ================================================================ batched ensemble
// Many independent lattices in one launch.  Persistent CTAs draw (instance, tile column) items
// from a table through an atomic work counter, so uneven instances balance themselves; every
// item runs the generic fused update above with the geometry of its instance and the shared
// model constants of P.  Per-item FP64 partials of (rho, T) are reduced per instance, in item
// order, by the last CTA to finish, which also re-arms both counters for the next launch.
template <typename S, int TY>
__global__ void __launch_bounds__(FusedShape<TY>::kThreads, 2)
k_fused_batch(DevParams P, const BatchInst* __restrict__ insts, const BatchItem* __restrict__ items, int n_items,
              int n_inst, const S* __restrict__ src, S* __restrict__ dst, int pull_f, int pull_g,
              const double* __restrict__ sums_cur, double2* partial, unsigned* counters, double* sums_next,
              float* __restrict__ phis, int* flag, int first) {
    using Sh = FusedShape<TY>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float* stage = reinterpret_cast<float*>(smem_raw);
    float2* ring = reinterpret_cast<float2*>(stage + 2 * Sh::kStageFloats);
    __shared__ double red_a[Sh::kThreads / 32], red_b[Sh::kThreads / 32];
    __shared__ int next_item, is_last;
    const int tid = threadIdx.x;
    int bad = 0;
    for (;;) {
        if (tid == 0) next_item = (int)atomicAdd(&counters[0], 1u);
        __syncthreads();
        const int it = next_item;
        __syncthreads();
        if (it >= n_items) break;
        const BatchItem w = items[it];
        const BatchInst I = insts[w.inst];
        DevParams Q = P;
        Q.nx = I.nx; Q.ny = I.ny; Q.nz = I.nz;
        Q.plane = I.nx * I.ny;
        Q.N = Q.plane * I.nz;
        Q.Ws = I.Ws; Q.Hs = I.Hs;
        Q.Rs = kSlots * I.Ws;
        Q.splane = Q.Rs * I.Hs;
        Q.Ns = I.Ws;
        Q.Nidx = Q.splane * I.nz - (kSlots - 1) * I.Ws;
        Q.inv_N = I.inv_N;
        Q.hot_cx = 0.5f * (float)I.nx;
        Q.hot_cy = 0.5f * (float)I.ny;
        float r_sum = 0.f, r_c = 0.f, t_sum = 0.f, t_c = 0.f;
        const float rho_ave = buoyancy_ref(P, sums_cur[2 * w.inst], I.inv_N);
        fused_column<S, TY, false>(Q, src + I.pop_off, dst + I.pop_off, pull_f, pull_g, rho_ave, phis + I.field_off, first,
                            w.x0, w.y0, w.z0, w.z1, stage, ring, r_sum, r_c, t_sum, t_c, bad);
        block_partial<Sh::kThreads>((double)r_sum - (double)r_c, (double)t_sum - (double)t_c, partial, it, tid, 0,
                                    red_a, red_b);
    }
    if (__syncthreads_or(bad) && tid == 0) atomicOr(flag, 1);
    if (tid == 0) {
        __threadfence();
        is_last = atomicAdd(&counters[1], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    for (int k = tid; k < n_inst; k += Sh::kThreads) {
        const BatchInst I = insts[k];
        double a = 0.0, b = 0.0;
        for (int j = I.item0; j < I.item0 + I.n_items; ++j) {
            const double2 q = __ldcg(partial + j);
            a += q.x;
            b += q.y;
        }
        sums_next[2 * k] = a;
        sums_next[2 * k + 1] = b;
    }
    if (tid == 0) {
        counters[0] = 0u;
        counters[1] = 0u;
    }
}

// ================================================================ TMA producer / consumer kernel
// Tile TX x TY.  Warps: producer, storer (FP32 only), compute warps (one tile node per thread:
// pull, psi, collision), one halo warp (psi of the one-node ring around the tile).
constexpr size_t align128(size_t v) { return (v + 127) / 128 * 128; }

template <int TX_, int TY_, typename S_ = float> struct TmaShape {
    using S = S_;
    static constexpr int kE = (int)sizeof(S);                        // bytes per stored population
    static constexpr int kInterior = TX_ * TY_;
    static constexpr int kHaloNodes = 2 * (TX_ + 2) + 2 * TY_;
    static constexpr int kSlotsAll = kInterior + kHaloNodes;        // ring slots with a psi value
    static constexpr int kCompWarps = (kInterior + 31) / 32;         // one tile node per thread
    static constexpr int kHaloWarps = 1;
    static constexpr int kHaloPerLane = (kHaloNodes + 31) / 32;      // halo slots of one halo lane
    static constexpr int kCompThreads = kCompWarps * 32, kHaloThreads = kHaloWarps * 32;
    // Output path: the collided plane goes to an output tile in shared memory and leaves by TMA
    // tensor stores issued by a storer warp (direct global stores by the compute threads measured
    // slower, for FP32 and for 16-bit storage alike).
    static constexpr int kLeadWarps = 2;                             // producer and storer warps first
    static constexpr int kThreads = 32 * kLeadWarps + kCompThreads + kHaloThreads;
    // registers per thread: warp w runs on SM sub-partition w % 4, whose register file holds 16K
    // registers; the per-thread count goes in steps of 8
    static constexpr int kWarpsPerSub = (kThreads / 32 + 3) / 4;
    static constexpr int kMaxRegs = (16384 / (32 * kWarpsPerSub)) / 8 * 8 > 255 ? 255
                                  : (16384 / (32 * kWarpsPerSub)) / 8 * 8;
    static constexpr int kRingW = TX_ + 2, kRingPlane = (TX_ + 2) * (TY_ + 2);
    // a window row starts kXOff columns left of the tile, on a 16-byte boundary
    static constexpr int kXOff = 16 / kE;
    static constexpr int kWinW = TX_ + 2 * kXOff;       // window columns x0-kXOff .. x0+TX+kXOff-1
    static constexpr int kWinH = TY_ + 4;               // window rows    y0-2 .. y0+TY+1
    static constexpr int kWin = kWinW * kWinH;          // elements per population slot
    // a stage holds the three slot groups (e_z = 0: slots 0-13, +1: 14-19, -1: 20-25), each
    // starting on a 128-byte boundary
    static constexpr size_t kGrp1 = align128((size_t)14 * kWin * kE);
    static constexpr size_t kGrp2 = kGrp1 + align128((size_t)6 * kWin * kE);
    static constexpr size_t kStageOne = kGrp2 + align128((size_t)6 * kWin * kE);
    // the collided plane and the periodic images of an edge tile are written into the stage whose
    // pulls were just made (the pulls of the plane above), and leave it by TMA tensor stores; the
    // stage is refilled once those stores have read it.  Inside a stage, from its start:
    //   out   [TY][26][TX]   the collided plane (a box of fewer rows reads a prefix of it)
    //   gcol  [TY][26][kGW]  kGW edge columns of an edge tile (kGW columns = 16 B)
    //   grow  [2][26][w]     its 2 edge rows (w = the tile's real columns)
    //   gcor  [2][26][kGW]   the kGW x 2 corner block
    // each laid out exactly as the box that stores it
    static constexpr int kGW = 16 / kE;
    static constexpr size_t kOutBytes = align128((size_t)kSlots * kInterior * kE);
    static constexpr size_t kGColOff = kOutBytes;
    static constexpr size_t kGRowOff = kGColOff + align128((size_t)TY_ * kSlots * kGW * kE);
    static constexpr size_t kGCorOff = kGRowOff + align128((size_t)2 * kSlots * TX_ * kE);
    static constexpr size_t kOutAllBytes = kGCorOff + align128((size_t)2 * kSlots * kGW * kE);
    static_assert(kOutAllBytes <= kStageOne, "the collided plane and its ghost images fit in a stage");
    // ring of (psi, rho) planes: planes z-1, z, z+1 of the collision and the plane pulled ahead
    static constexpr int kRing = 4;
    // as many stages as fit in one CTA's 227 KB beside the ring (at most 3 for FP32, 4 for 16-bit
    // storage; at least 3: a stage holds a plane's pulls and then the collided plane below it)
    static constexpr size_t kFixed = (size_t)kRing * (TX_ + 2) * (TY_ + 2) * sizeof(float2) + 2048;
    static constexpr int kStagesFit = (int)((227 * 1024 - kFixed) / kStageOne);
    static constexpr int kStagesCap = kE == 4 ? 3 : 4;
    static constexpr int kStages = kStagesFit > kStagesCap ? kStagesCap : kStagesFit;
    static_assert(kStages >= 3, "three stages of the tile's window fit in shared memory");
    static constexpr size_t kStageBytes = (size_t)kStages * kStageOne;
    static constexpr size_t kRingOff = kStageBytes;
    static constexpr size_t kSmem = kRingOff + (size_t)kRing * kRingPlane * sizeof(float2);
    // element offset of storage slot s inside a stage
    static constexpr __host__ __device__ int slot_off(int s) {
        return s < 14 ? s * kWin : s < 20 ? (int)(kGrp1 / kE) + (s - 14) * kWin : (int)(kGrp2 / kE) + (s - 20) * kWin;
    }
    // thread counts of the named barriers (see k_fused_tma)
    static constexpr int kCntRing = kCompThreads + kHaloThreads + 32;
    static constexpr int kCntOut = kCompThreads + 32;
    static constexpr int kCntEmpty = 64;
    static_assert(kStages <= 4, "three named barriers a stage, ids 2..13");
    static_assert(TX_ % 8 == 0 || kE == 4, "tile origins on 16-byte boundaries for 2-byte storage");
    static_assert(TX_ % 4 == 0, "tile origins on 16-byte boundaries");
    static_assert(kSmem <= 227 * 1024, "shared memory of one CTA");
};

// ring slot (lx, ly) of slot index q: tile nodes (row-major), then the halo ring
template <int TX_, int TY_>
__device__ __forceinline__ void tma_slot_of(int q, int& lx, int& ly) {
    using Sh = TmaShape<TX_, TY_, float>;
    lx = -1;
    ly = -1;
    if (q < Sh::kInterior) {
        lx = q % TX_ + 1;
        ly = q / TX_ + 1;
    } else {
        int h = q - Sh::kInterior;
        if (h < TX_ + 2) { lx = h; ly = 0; }
        else if (h < 2 * (TX_ + 2)) { lx = h - (TX_ + 2); ly = TY_ + 1; }
        else if (h < Sh::kHaloNodes) { int k = h - 2 * (TX_ + 2); lx = (k & 1) ? TX_ + 1 : 0; ly = 1 + (k >> 1); }
    }
}

constexpr unsigned kSpinLimit = 1u << 21;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// the waiting thread may sleep (up to about 1 us per call) until the phase completes, instead of
// spinning on the issue slots the other warps need
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(1000u)
        : "memory");
    return ok != 0;
}
// bounded wait: false after kSpinLimit polls (the caller records a timeout and stops waiting)
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    for (unsigned it = 0; it < kSpinLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_4d(void* smem_dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// tensor store of a shared-memory box (bulk async-group completion); the box is clipped at the
// tensor's bounds
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, const void* smem_src, int c0, int c1, int c2,
                                             int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(
            reinterpret_cast<unsigned long long>(map)),
        "r"(smem_u32(smem_src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// generic-proxy shared-memory writes of this thread become visible to the async (TMA) proxy
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// source plane of the e_z = +1 group (pulls from z-1) and of the e_z = -1 group (pulls from
// z+1); -1 at a wall face (all those links bounce back from the node itself)
__device__ __forceinline__ int src_plane_up(const DevParams& P, int mz) {
    if (mz > 0) return mz - 1;
    int bc = P.bc[4];
    return f_wraps(bc) ? P.nz - 1 : (bc == BC_OUTFLOW ? 0 : -1);
}
__device__ __forceinline__ int src_plane_dn(const DevParams& P, int mz) {
    if (mz < P.nz - 1) return mz + 1;
    int bc = P.bc[5];
    return f_wraps(bc) ? 0 : (bc == BC_OUTFLOW ? P.nz - 1 : -1);
}

// Stored population <-> FP32 (shifted 16-bit storage: stored = value - w_a ref, rounded to
// nearest even; the same operations as the generic kernels' Codec).
template <typename S> __device__ __forceinline__ float st_dec(S v, float sh);
template <> __device__ __forceinline__ float st_dec<float>(float v, float) { return v; }
template <> __device__ __forceinline__ float st_dec<__nv_bfloat16>(__nv_bfloat16 v, float sh) {
    return __bfloat162float(v) + sh;
}
template <> __device__ __forceinline__ float st_dec<__half>(__half v, float sh) { return __half2float(v) + sh; }
template <typename S> __device__ __forceinline__ S st_enc(float v, float sh);
template <> __device__ __forceinline__ float st_enc<float>(float v, float) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 st_enc<__nv_bfloat16>(float v, float sh) {
    return __float2bfloat16_rn(v - sh);
}
template <> __device__ __forceinline__ __half st_enc<__half>(float v, float sh) { return __float2half_rn(v - sh); }

// The 26 pulled populations of the node whose window cell is b (a pointer into a stage), with the
// boundary links of its plane mz patched: Eq. 50 for f at z walls (f*_abar of the node itself,
// read from global memory), Eq. 51 for g at non-periodic z faces (own g+_abar from global memory)
// and at thermal x / y faces (own g+_abar from the stage).
template <class Sh>
__device__ __forceinline__ void stage_pulls(const DevParams& P, const typename Sh::S* __restrict__ b,
                                            const typename Sh::S* __restrict__ src, int mx, int my, int mz,
                                            float f[19], float g[7]) {
    using S = typename Sh::S;
    constexpr int WW = Sh::kWinW;
#define GB300_SF(A) f[A] = st_dec<S>(b[Sh::slot_off(fslot(A)) - ey19(A) * WW - ex19(A)], P.shift_f[A]);
    GB300_SF(0) GB300_SF(1) GB300_SF(2) GB300_SF(3) GB300_SF(4) GB300_SF(5) GB300_SF(6) GB300_SF(7) GB300_SF(8)
    GB300_SF(9) GB300_SF(10) GB300_SF(11) GB300_SF(12) GB300_SF(13) GB300_SF(14) GB300_SF(15) GB300_SF(16)
    GB300_SF(17) GB300_SF(18)
#undef GB300_SF
#define GB300_SG(A) g[A] = st_dec<S>(b[Sh::slot_off(gslot(A)) - ey7(A) * WW - ex7(A)], P.shift_g[A]);
    GB300_SG(0) GB300_SG(1) GB300_SG(2) GB300_SG(3) GB300_SG(4) GB300_SG(5) GB300_SG(6)
#undef GB300_SG
    if (mz == 0 && P.bc[4] != BC_PERIODIC) {
        const int i = (int)bidx(P, sidx(P, mx, my, mz), P.Nidx);
        if (P.bc[4] == BC_WALL) {
            f[5] = Codec<S>::load(src + (size_t)fslot(6) * P.Ns + i, P.shift_f[6]);
            f[11] = Codec<S>::load(src + (size_t)fslot(12) * P.Ns + i, P.shift_f[12]);
            f[14] = Codec<S>::load(src + (size_t)fslot(13) * P.Ns + i, P.shift_f[13]);
            f[15] = Codec<S>::load(src + (size_t)fslot(16) * P.Ns + i, P.shift_f[16]);
            f[18] = Codec<S>::load(src + (size_t)fslot(17) * P.Ns + i, P.shift_f[17]);
        }
        g[5] = -Codec<S>::load(src + (size_t)gslot(6) * P.Ns + i, P.shift_g[6]) + 2.f * P.w1 * wall_T(P, 4, mx, my);
    }
    if (mz == P.nz - 1 && P.bc[5] != BC_PERIODIC) {
        const int i = (int)bidx(P, sidx(P, mx, my, mz), P.Nidx);
        if (P.bc[5] == BC_WALL) {
            f[6] = Codec<S>::load(src + (size_t)fslot(5) * P.Ns + i, P.shift_f[5]);
            f[12] = Codec<S>::load(src + (size_t)fslot(11) * P.Ns + i, P.shift_f[11]);
            f[13] = Codec<S>::load(src + (size_t)fslot(14) * P.Ns + i, P.shift_f[14]);
            f[16] = Codec<S>::load(src + (size_t)fslot(15) * P.Ns + i, P.shift_f[15]);
            f[17] = Codec<S>::load(src + (size_t)fslot(18) * P.Ns + i, P.shift_f[18]);
        }
        g[6] = -Codec<S>::load(src + (size_t)gslot(5) * P.Ns + i, P.shift_g[5]) + 2.f * P.w1 * wall_T(P, 5, mx, my);
    }
    if (P.bc[0] == BC_THERMAL_ONLY && mx == 0)
        g[1] = -st_dec<S>(b[Sh::slot_off(gslot(2))], P.shift_g[2]) + 2.f * P.w1 * wall_T(P, 0, mx, my);
    if (P.bc[1] == BC_THERMAL_ONLY && mx == P.nx - 1)
        g[2] = -st_dec<S>(b[Sh::slot_off(gslot(1))], P.shift_g[1]) + 2.f * P.w1 * wall_T(P, 1, mx, my);
    if (P.bc[2] == BC_THERMAL_ONLY && my == 0)
        g[3] = -st_dec<S>(b[Sh::slot_off(gslot(4))], P.shift_g[4]) + 2.f * P.w1 * wall_T(P, 2, mx, my);
    if (P.bc[3] == BC_THERMAL_ONLY && my == P.ny - 1)
        g[4] = -st_dec<S>(b[Sh::slot_off(gslot(3))], P.shift_g[3]) + 2.f * P.w1 * wall_T(P, 3, mx, my);
}

// named barriers of the TMA kernel (bar.sync / bar.arrive; 0 is __syncthreads): the waiting
// warps block in hardware and issue nothing while they wait.  Three per stage s (s < kStages <= 4).
constexpr int kBarComp = 1;
__device__ __forceinline__ int bar_ring(int s) { return 2 + s; }
__device__ __forceinline__ int bar_out_full(int s) { return 6 + s; }
__device__ __forceinline__ int bar_empty(int s) { return 10 + s; }
__device__ __forceinline__ void nb_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void nb_arrive(int id, int nthreads) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Warp roles: warp 0 = producer (TMA loads), warp 1 = storer (TMA stores), then the compute warps
// (thread t owns tile node t: it pulls the node's 26 populations once, writes the node's
// (psi, rho) into the ring, keeps the populations in registers and collides the node one plane
// later), then one halo warp (psi of the ring around the tile, kHaloPerLane slots a lane).
// Stage use k (plane p) goes through stage s = k % kStages:
//   full[s]        mbarrier: the TMA bytes of use k landed (producer -> compute, halo; bounded waits)
//   RING(s)        named: producer bar.arrive once use k's loads are issued; compute and halo
//                  bar.sync once they have pulled plane p and put its psi into the ring.  After it
//                  nobody reads the stage's window again, and the ring holds plane p.
//   OUT_FULL(s)    named: compute bar.arrive -> storer bar.sync.  For the uses that carry an output
//                  (p = z0 + 1 .. z1 of an item) the compute warps first write the collided plane
//                  p - 1 (and an edge tile's periodic images) into the stage itself.
//   EMPTY(s)       named, bar.sync by storer and producer: the tensor stores have read the stage
//                  and it may be refilled (the producer waits for use k before loading k + kStages).
// The collided plane thus leaves from the stage just pulled, so the compute warps never wait for
// a store to drain: the storer and the next loads have kStages - 1 planes of time for it.
// Stage uses and ring planes follow one plane counter k across the CTA's items.  Every role runs
// the same sequence of named-barrier operations whatever happens: an abort (a TMA wait that ran
// out) skips only the mbarrier waits, the copies and the work, so no barrier is left incomplete.
// No role laps another on a barrier: RING and EMPTY are synced by the roles that could run ahead
// (compute, halo; storer, producer), the producer's next arrival on RING(s) follows its EMPTY(s)
// sync of the previous use of s, and the compute warps' next arrival on OUT_FULL(s) follows their
// RING(s) sync of the next use of s, which needs that arrival of the producer.
template <int TX_, int TY_, typename S, bool kWet>
__global__ void __maxnreg__((TmaShape<TX_, TY_, S>::kMaxRegs))
k_fused_tma(const __grid_constant__ CUtensorMap map14, const __grid_constant__ CUtensorMap map6,
            const __grid_constant__ CUtensorMap map_out, const __grid_constant__ CUtensorMap map_out_top,
            const __grid_constant__ CUtensorMap map_gcol, const __grid_constant__ CUtensorMap map_gcol_top,
            const __grid_constant__ CUtensorMap map_grow, const __grid_constant__ CUtensorMap map_grow_right,
            const __grid_constant__ CUtensorMap map_gcor, int ghosts, DevParams P, const S* __restrict__ src,
            S* __restrict__ dst,
            const double* __restrict__ sums_cur, double2* partial, unsigned* counter, double* sums_next,
            float* __restrict__ phis, int* flag, int first, int zchunk, int tiles_x, int tiles_y, int n_items) {
    using Sh = TmaShape<TX_, TY_, S>;
    constexpr int kWinW = Sh::kWinW, kStages = Sh::kStages, kRing = Sh::kRing, kRP = Sh::kRingPlane;
    constexpr int kComp = Sh::kCompThreads, kGW = Sh::kGW;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // stage s: smem_raw + s * kStageOne (three slot groups of [slots][TY+4][TX+2 kXOff])
    // stage s: smem_raw + s * kStageOne; after its pulls it holds the collided plane below (out,
    // gcol, grow, gcor at kGColOff, kGRowOff, kGCorOff)
    float2* ring = reinterpret_cast<float2*>(smem_raw + Sh::kRingOff);           // [kRing][TY+2][TX+2]
    __shared__ __align__(8) unsigned long long full_bar[kStages], stall_bar;
    __shared__ double red_a[kComp / 32], red_b[kComp / 32];
    __shared__ int is_last;
    __shared__ volatile int abort_flag;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&full_bar[s], 1);
        mbar_init(&stall_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int ntiles = tiles_x * tiles_y;
    // bounded wait for the bytes of a stage use: a timeout raises the abort flag, after which no
    // role waits for a copy again
    auto wait_full = [&](int s, unsigned parity) {
        if (abort_flag) return;
        if (!mbar_wait(&full_bar[s], parity)) {
            abort_flag = 1;
            atomicOr(flag, 2);
        }
    };
    auto stage_of = [&](int s) { return reinterpret_cast<const S*>(smem_raw + (size_t)s * Sh::kStageOne); };

    if (warp == 0) {
        // ------------------------------------------------------------ producer (lane 0 issues)
        unsigned k = 0;
        for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
            const int chunk = item / ntiles, tile = item % ntiles;
            const int x0 = (tile % tiles_x) * TX_, y0 = (tile / tiles_x) * TY_;
            const int z0 = chunk * zchunk, z1 = min(P.nz, z0 + zchunk);
            // window origin in storage coordinates: (x0 - kXOff) + kGX, (y0 - 2) + kGY
            const int cx = x0 - Sh::kXOff + kGX, cy = y0;
            for (int p = z0 - 1; p <= z1; ++p, ++k) {
                const int s = k % kStages;
                if (k >= (unsigned)kStages) nb_sync(bar_empty(s), Sh::kCntEmpty);   // use k - kStages stored
                if (lane == 0) {
                    if (P.test_stall && k == 0) {
                        // timeout-path test: the first stage's data never comes; the producer waits
                        // (bounded) on a barrier nothing completes, then releases the stage empty
                        if (!mbar_wait(&stall_bar, 0u)) {
                            abort_flag = 1;
                            atomicOr(flag, 2);
                        }
                        mbar_arrive(&full_bar[s]);
                    } else if (abort_flag) {
                        mbar_arrive(&full_bar[s]);   // release the waiters without data
                    } else {
                        const int mz = map_coord(p, P.nz, P.bc[4], P.bc[5]);
                        const int zu = src_plane_up(P, mz), zd = src_plane_dn(P, mz);
                        const unsigned bytes =
                            (14u + (zu >= 0 ? 6u : 0u) + (zd >= 0 ? 6u : 0u)) * (unsigned)(Sh::kWin * Sh::kE);
                        unsigned char* st = smem_raw + (size_t)s * Sh::kStageOne;
                        mbar_expect_tx(&full_bar[s], bytes);
                        tma_load_4d(st, &map14, cx, cy, mz, 0, &full_bar[s]);
                        if (zu >= 0) tma_load_4d(st + Sh::kGrp1, &map6, cx, cy, zu, 14, &full_bar[s]);
                        if (zd >= 0) tma_load_4d(st + Sh::kGrp2, &map6, cx, cy, zd, 20, &full_bar[s]);
                    }
                }
                __syncwarp();
                nb_arrive(bar_ring(s), Sh::kCntRing);   // use k is under way
            }
        }
        // the last stage uses (every use of EMPTY is matched on both sides)
        const unsigned q0 = k > (unsigned)kStages ? k - kStages : 0u;
        for (unsigned q = q0; q < k; ++q) nb_sync(bar_empty(q % kStages), Sh::kCntEmpty);
        // copies still in flight land before the CTA exits (every use completes one phase; bounded)
        if (lane == 0)
            for (unsigned q = q0; q < k; ++q) mbar_wait(&full_bar[q % kStages], (q / kStages) & 1);
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------------------ storer (lane 0 issues)
        unsigned k = 0;
        for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
            const int chunk = item / ntiles, tile = item % ntiles;
            const int x0 = (tile % tiles_x) * TX_, y0 = (tile / tiles_x) * TY_;
            const int z0 = chunk * zchunk, z1 = min(P.nz, z0 + zchunk);
            // box (x, slot, y, z) at the tile origin (x a multiple of 4 floats); the last tile
            // row uses the map whose box holds exactly its rows, so a box never reaches past
            // ny; columns beyond nx fall outside the tensor and are not written
            const CUtensorMap* m = y0 + TY_ > P.ny ? &map_out_top : &map_out;
            // ghost cells written from this tile (storage coordinates; every box lies inside
            // the padded plane exactly): its 4 edge columns to the opposite ghost columns, its
            // 2 edge rows to the opposite ghost rows, and the corner block
            const bool left = ghosts == 1 && x0 == 0, right = ghosts == 1 && x0 + TX_ >= P.nx;
            const bool bottom = ghosts == 1 && y0 == 0, top = ghosts == 1 && y0 + TY_ >= P.ny;
            const int gx_col = right ? kGX - kGW : P.nx + kGX;    // destination of the column box
            const int gy_row = top ? kGY - 2 : P.ny + kGY;        // destination of the row box
            const CUtensorMap* mc = y0 + TY_ > P.ny ? &map_gcol_top : &map_gcol;
            const CUtensorMap* mr = x0 + TX_ > P.nx ? &map_grow_right : &map_grow;
            // ghost mode 2, nx no multiple of the 16-byte band: the last tile column stores its
            // nodes itself (a tensor store clipped at nx inside a 16-byte unit also writes the
            // ghost columns past nx, which the first tile column's nodes write)
            const bool direct_tile = ghosts == 2 && x0 + TX_ > P.nx && P.nx % kGW != 0;
            for (int p = z0 - 1; p <= z1; ++p, ++k) {
                const int s = k % kStages;
                nb_sync(bar_out_full(s), Sh::kCntOut);
                if (p > z0 && lane == 0 && !abort_flag && !direct_tile) {   // the stage holds collided plane p - 1
                    const int z = p - 1;
                    unsigned char* st = smem_raw + (size_t)s * Sh::kStageOne;
                    tma_store_4d(m, st, x0 + kGX, 0, y0 + kGY, z);
                    if (left || right) tma_store_4d(mc, st + Sh::kGColOff, gx_col, 0, y0 + kGY, z);
                    if (top || bottom) tma_store_4d(mr, st + Sh::kGRowOff, x0 + kGX, 0, gy_row, z);
                    if ((left || right) && (top || bottom))
                        tma_store_4d(&map_gcor, st + Sh::kGCorOff, gx_col, 0, gy_row, z);
                    bulk_commit();
                    bulk_wait_read_all();
                }
                __syncwarp();
                nb_sync(bar_empty(s), Sh::kCntEmpty);   // the stage may be refilled
            }
        }
        if (lane == 0) bulk_wait_all();   // the stores have completed before the CTA exits
        __syncwarp();
    } else if (warp < Sh::kLeadWarps + Sh::kCompWarps) {
        // ------------------------------------------------------------ compute
        const int ct = tid - 32 * Sh::kLeadWarps;
        const bool node_thread = ct < Sh::kInterior;
        const int lx = ct % TX_ + 1, ly = ct / TX_ + 1;
        // (the shared-memory offsets a thread reaches from these bases stay inside the ring plane,
        // each slot's window and the output tile; checked in bounds-checked builds)
        const int slot = node_thread ? bbase(P, ly * Sh::kRingW + lx, -(Sh::kRingW + 1), Sh::kRingW + 1, kRP)
                                     : ly * Sh::kRingW + lx;
        const int woff = node_thread ? bbase(P, (ly + 1) * kWinW + lx - 1 + Sh::kXOff, -(kWinW + 1), kWinW + 1,
                                             Sh::kWin)
                                     : 0;
        const float rho_ave = buoyancy_ref(P, sums_cur[0], P.inv_N);
        const int ooff = node_thread ? bbase(P, (ly - 1) * (kSlots * TX_) + (lx - 1), 0, (kSlots - 1) * TX_,
                                             kSlots * Sh::kInterior)
                                     : 0;   // the node's element in the out tile
        int bad = 0;
        unsigned k = 0;
        for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
            const int chunk = item / ntiles, tile = item % ntiles;
            const int x0 = (tile % tiles_x) * TX_, y0 = (tile / tiles_x) * TY_;
            const int z0 = chunk * zchunk, z1 = min(P.nz, z0 + zchunk);
            const int gx = x0 + lx - 1, gy = y0 + ly - 1;
            const bool owner = node_thread && gx < P.nx && gy < P.ny;
            // a tile slot just past the lattice edge (partial tile) holds the psi of the periodic
            // image or mirror node there, as the halo ring does
            const bool used = node_thread && gx <= P.nx && gy <= P.ny;
            const int mx = used ? map_coord(gx, P.nx, P.bc[0], P.bc[1]) : 0;
            const int my = used ? map_coord(gy, P.ny, P.bc[2], P.bc[3]) : 0;
            // this node's place in the ghost staging tiles of an edge tile (-1: none)
            const bool eright = ghosts == 1 && x0 + TX_ >= P.nx, eleft = ghosts == 1 && x0 == 0;
            const bool etop = ghosts == 1 && y0 + TY_ >= P.ny, ebottom = ghosts == 1 && y0 == 0;
            // ghost mode 2: this node's periodic images in the ghost columns (hx) and rows (hy)
            const bool hx = ghosts == 2 && owner && (gx < 2 || gx >= P.nx - 2);
            const bool hy = ghosts == 2 && owner && (gy < 2 || gy >= P.ny - 2);
            const int ix = gx < 2 ? gx + P.nx : gx - P.nx, iy = gy < 2 ? gy + P.ny : gy - P.ny;
            // ... and the last tile column of such a lattice stores its nodes directly (see storer)
            const bool direct_tile = ghosts == 2 && x0 + TX_ > P.nx && P.nx % kGW != 0;
            const int cx4 = !owner ? -1 : eright ? (gx >= P.nx - kGW ? gx - (P.nx - kGW) : -1)
                                        : eleft ? (gx < kGW ? gx : -1) : -1;
            const int ry2 = !owner ? -1 : etop ? (gy >= P.ny - 2 ? gy - (P.ny - 2) : -1)
                                        : ebottom ? (gy < 2 ? gy : -1) : -1;
            // the edge-row tile is as wide as the tile's real columns (the box reads it densely)
            const int rw = min(TX_, P.nx - x0);
            float r_sum = 0.f, r_c = 0.f, t_sum = 0.f, t_c = 0.f;
            // phi_s history of the thread's node, loaded one plane ahead of its use
            float ph_next = owner ? phis[bidx(P, node_of(P, gx, gy, z0), P.N)] : 0.f;

            // pull plane p (stage use k) into (fo, go), put the node's (psi, rho) into ring plane k
            auto pull_plane = [&](int p, float* fo, float* go, float& ro, float& To, float& po) {
                const int s = k % kStages;
                wait_full(s, (k / kStages) & 1);
                float2* rp = ring + (k % kRing) * kRP + slot;
                if (kWet && p < 0) {   // solid layer below a wetting -z wall: virtual (psi, rho)
                    if (used) *rp = wall_entry(P, mx, my);
                } else if (used) {
                    const int mz = map_coord(p, P.nz, P.bc[4], P.bc[5]);
                    stage_pulls<Sh>(P, stage_of(s) + woff, src, mx, my, mz, fo, go);
                    ro = sum19(fo);
                    To = sum7(go);
                    const float psi2 = psi_squared(P, ro, To);
                    po = psi_of(psi2);
                    *rp = make_float2(po, ro);
                    bad |= !(psi2 > 0.f) || !isfinite(ro) || !isfinite(To);
                }
                nb_sync(bar_ring(s), Sh::kCntRing);   // the window is read; the ring holds plane p
                ++k;
            };
            // one collided plane z: pull plane z + 1 (into the n-set), wait for the ring, collide
            // plane z (the c-set), store it
            auto iterate = [&](int z, float* fc, float* gc, float rc, float Tc, float pc, float* fn, float* gn,
                               float& rn, float& Tn, float& pn) {
                pull_plane(z + 1, fn, gn, rn, Tn, pn);   // ring: psi of planes z - 1, z, z + 1
                const int so = (k - 1) % kStages;       // the stage just pulled receives plane z
                const float ph_prev = ph_next;
                if (owner && z + 1 < z1) ph_next = phis[bidx(P, node_of(P, gx, gy, z + 1), P.N)];
                float ph = 0.f;
                if (owner) {
                    const float2* rm = ring + ((k - 3) % kRing) * kRP;
                    const float2* r0 = ring + ((k - 2) % kRing) * kRP;
                    const float2* rq = ring + ((k - 1) % kRing) * kRP;
                    const RingStencil rs = ring_stencil(rm, r0, rq, slot, Sh::kRingW);
                    kahan_add(r_sum, r_c, rc);
                    kahan_add(t_sum, t_c, Tc);
                    const Forces F = total_force(P, pc, rs.Fx, rs.Fy, rs.Fz, rc - rho_ave);
                    NodeOut o = collide_f(P, fc, rc, F.Fx, F.Fy, F.Fz, F.Fm2, pc * pc);
                    ph = collide_g(P, gc, rc, Tc, o, rs.gx, rs.gy, rs.gz, ph_prev, first);
                }
                {
                    S* const sb = reinterpret_cast<S*>(smem_raw + (size_t)so * Sh::kStageOne);
                    S* const outp = sb + ooff;
                    if (owner) {
                        S fe[19], ge[7];
#pragma unroll
                        for (int a = 0; a < 19; ++a) fe[a] = st_enc<S>(fc[a], P.shift_f[a]);
#pragma unroll
                        for (int a = 0; a < 7; ++a) ge[a] = st_enc<S>(gc[a], P.shift_g[a]);
                        if (direct_tile) {
                            S* q = dst + bidx(P, sidx(P, gx, gy, z), P.Nidx);
#pragma unroll
                            for (int a = 0; a < 19; ++a) q[(size_t)fslot(a) * P.Ns] = fe[a];
#pragma unroll
                            for (int a = 0; a < 7; ++a) q[(size_t)gslot(a) * P.Ns] = ge[a];
                        } else {
#pragma unroll
                            for (int a = 0; a < 19; ++a) outp[fslot(a) * TX_] = fe[a];
#pragma unroll
                            for (int a = 0; a < 7; ++a) outp[gslot(a) * TX_] = ge[a];
                        }
                        if (cx4 >= 0) {   // edge column: [TY][26][kGW]
                            S* q = sb + Sh::kGColOff / sizeof(S) + (ly - 1) * (kSlots * kGW) + cx4;
#pragma unroll
                            for (int a = 0; a < 19; ++a) q[fslot(a) * kGW] = fe[a];
#pragma unroll
                            for (int a = 0; a < 7; ++a) q[gslot(a) * kGW] = ge[a];
                        }
                        if (ry2 >= 0) {   // edge row: [2][26][rw]
                            S* q = sb + Sh::kGRowOff / sizeof(S) + ry2 * (kSlots * rw) + (lx - 1);
#pragma unroll
                            for (int a = 0; a < 19; ++a) q[fslot(a) * rw] = fe[a];
#pragma unroll
                            for (int a = 0; a < 7; ++a) q[gslot(a) * rw] = ge[a];
                        }
                        if (cx4 >= 0 && ry2 >= 0) {   // corner block: [2][26][kGW]
                            S* q = sb + Sh::kGCorOff / sizeof(S) + ry2 * (kSlots * kGW) + cx4;
#pragma unroll
                            for (int a = 0; a < 19; ++a) q[fslot(a) * kGW] = fe[a];
#pragma unroll
                            for (int a = 0; a < 7; ++a) q[gslot(a) * kGW] = ge[a];
                        }
                        if (hx || hy) {   // ghost mode 2: straight to the images in dst
                            auto put = [&](int qx, int qy) {
                                S* q = dst + bidx(P, sidx(P, qx, qy, z), P.Nidx);
#pragma unroll
                                for (int a = 0; a < 19; ++a) q[(size_t)fslot(a) * P.Ns] = fe[a];
#pragma unroll
                                for (int a = 0; a < 7; ++a) q[(size_t)gslot(a) * P.Ns] = ge[a];
                            };
                            if (hx) put(ix, gy);
                            if (hy) put(gx, iy);
                            if (hx && hy) put(ix, iy);
                        }
                    }
                    // this thread's out writes become visible to the tensor store (async proxy)
                    fence_proxy_async_smem();
                    nb_arrive(bar_out_full(so), Sh::kCntOut);
                }
                if (owner) phis[bidx(P, node_of(P, gx, gy, z), P.N)] = ph;
            };

            // the populations of the plane being collided (a) and of the plane pulled ahead (b)
            float fa[19], ga[7], ra = 0.f, Ta = 0.f, pa = 0.f;
            float fb[19], gb[7], rb = 0.f, Tb = 0.f, pb = 0.f;
            pull_plane(z0 - 1, fb, gb, rb, Tb, pb);   // psi only
            nb_arrive(bar_out_full((k - 1) % kStages), Sh::kCntOut);   // no output in this use
            pull_plane(z0, fa, ga, ra, Ta, pa);
            nb_arrive(bar_out_full((k - 1) % kStages), Sh::kCntOut);
            // one copy of the loop body (the instruction cache holds it; unrolled twice to swap the
            // two register sets it measured slower), so the pulled-ahead set is moved over
#pragma unroll 1
            for (int z = z0; z < z1; ++z) {
                iterate(z, fa, ga, ra, Ta, pa, fb, gb, rb, Tb, pb);
#pragma unroll
                for (int a = 0; a < 19; ++a) fa[a] = fb[a];
#pragma unroll
                for (int a = 0; a < 7; ++a) ga[a] = gb[a];
                ra = rb;
                Ta = Tb;
                pa = pb;
            }
            block_partial<kComp>((double)r_sum - (double)r_c, (double)t_sum - (double)t_c, partial, item, ct,
                                 kBarComp, red_a, red_b);
        }
        if (bad) atomicOr(flag, 1);
        finish_sums<kComp>(partial, n_items, counter, sums_next, ct, kBarComp, red_a, red_b, &is_last);
    } else {
        // ------------------------------------------------------------ halo psi (one warp)
        int bad = 0;
        unsigned k = 0;
        for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
            const int chunk = item / ntiles, tile = item % ntiles;
            const int x0 = (tile % tiles_x) * TX_, y0 = (tile / tiles_x) * TY_;
            const int z0 = chunk * zchunk, z1 = min(P.nz, z0 + zchunk);
            for (int p = z0 - 1; p <= z1; ++p, ++k) {
                const int s = k % kStages;
                float2* rp = ring + (k % kRing) * kRP;
                wait_full(s, (k / kStages) & 1);
                const S* st = stage_of(s);
                const int mz = map_coord(p, P.nz, P.bc[4], P.bc[5]);
                // kHaloPerLane slots a lane, rolled (one copy of the pull and EOS code); the slot
                // geometry is recomputed per plane rather than kept in an indexed array
#pragma unroll 1
                for (int j = 0; j < Sh::kHaloPerLane; ++j) {
                    const int q = Sh::kInterior + lane + 32 * j;
                    if (q >= Sh::kSlotsAll) break;
                    int lx, ly;
                    tma_slot_of<TX_, TY_>(q, lx, ly);
                    const int gx = x0 + lx - 1, gy = y0 + ly - 1;
                    if (gx < -1 || gx > P.nx || gy < -1 || gy > P.ny) continue;
                    const int mx = map_coord(gx, P.nx, P.bc[0], P.bc[1]);
                    const int my = map_coord(gy, P.ny, P.bc[2], P.bc[3]);
                    const int roff = bbase(P, ly * Sh::kRingW + lx, 0, 0, kRP);
                    if (kWet && p < 0) {   // virtual (psi, rho) of the solid layer below a wetting -z wall
                        rp[roff] = wall_entry(P, mx, my);
                        continue;
                    }
                    float f[19], g[7];
                    stage_pulls<Sh>(P, st + bbase(P, (ly + 1) * kWinW + lx - 1 + Sh::kXOff, -(kWinW + 1), kWinW + 1, Sh::kWin),
                                    src, mx, my, mz, f, g);
                    const float rho = sum19(f), T = sum7(g);
                    const float psi2 = psi_squared(P, rho, T);
                    rp[roff] = make_float2(psi_of(psi2), rho);
                    bad |= !(psi2 > 0.f) || !isfinite(rho) || !isfinite(T);
                }
                nb_sync(bar_ring(s), Sh::kCntRing);   // the window is read; the ring holds plane p
            }
        }
        if (bad) atomicOr(flag, 1);
    }
    __syncthreads();
}

// Ghost refresh after a step on the TMA path: every ghost cell (columns -2, -1, nx, nx+1 over all
// rows including the ghost rows, and rows -2, -1, ny, ny+1 over the real columns) receives the
// stored populations of its periodic image.  Threads [0, nA): one (row, slot) each, copying the
// column pairs (nx-2, nx-1) -> (-2, -1) and (0, 1) -> (nx, nx+1) (as one word pair when nx is
// even); threads [nA, nA + nB): one (ghost row, slot, 4-column group) each (one wide word when
// nx % 4 == 0).  Raw element bits are copied, so any storage type works.
template <int E> struct RawPair;
template <> struct RawPair<4> { using T = uint2; using Q = uint4; using W = unsigned; };
template <> struct RawPair<2> { using T = unsigned; using Q = uint2; using W = unsigned short; };
template <typename S>
__global__ void __launch_bounds__(256) k_ghosts(DevParams P, S* __restrict__ pops) {
    using R = RawPair<(int)sizeof(S)>;
    using T2 = typename R::T;
    using T4 = typename R::Q;
    using T1 = typename R::W;
    const int nA = (P.ny + 4) * kSlots;
    const int groups = (P.nx + 3) / 4;
    const int nB = 4 * kSlots * groups;
    const int t = blockIdx.x * 256 + threadIdx.x;
    const int z = blockIdx.y;
    if (t < nA) {
        const int a = t % kSlots, gy = t / kSlots - 2;
        const int iy = ((gy % P.ny) + P.ny) % P.ny;
        S* base = pops + (size_t)a * P.Ns;
        const int yrow = sidx(P, 0, gy, z), irow = sidx(P, 0, iy, z);
        if ((P.nx & 1) == 0) {
            const T2 hi = *reinterpret_cast<const T2*>(base + irow + P.nx - 2);
            const T2 lo = *reinterpret_cast<const T2*>(base + irow);
            *reinterpret_cast<T2*>(base + yrow - 2) = hi;
            *reinterpret_cast<T2*>(base + yrow + P.nx) = lo;
        } else {
            T1* b1 = reinterpret_cast<T1*>(base);
            const T1 h0 = b1[irow + P.nx - 2], h1 = b1[irow + P.nx - 1], l0 = b1[irow], l1 = b1[irow + 1];
            b1[yrow - 2] = h0;
            b1[yrow - 1] = h1;
            b1[yrow + P.nx] = l0;
            b1[yrow + P.nx + 1] = l1;
        }
    } else if (t < nA + nB) {
        const int u = t - nA;
        const int q = u % groups, a = (u / groups) % kSlots, k = u / (groups * kSlots);
        const int gy = k == 0 ? -2 : k == 1 ? -1 : k == 2 ? P.ny : P.ny + 1;
        const int iy = ((gy % P.ny) + P.ny) % P.ny;
        S* base = pops + (size_t)a * P.Ns;
        const int dst = sidx(P, 4 * q, gy, z), src = sidx(P, 4 * q, iy, z);
        if ((P.nx & 3) == 0) {
            *reinterpret_cast<T4*>(base + dst) = *reinterpret_cast<const T4*>(base + src);
        } else {
            T1* b1 = reinterpret_cast<T1*>(base);
            for (int c = 0; c < 4 && 4 * q + c < P.nx; ++c) b1[dst + c] = b1[src + c];
        }
    }
}

// Tile shapes of the TMA kernel (index = plan shape): 8 to 13 compute warps of one tile node a
// thread.  kTmaRate is each shape's node rate per CTA relative to 32 x 8 (a prior for the model
// below, which lbm_autotune replaces by measurement).  The 40-wide shapes tile lattices whose nx
// is a multiple of 40 (such as 200) without a partial tile column.
#define GB300_TMA_SHAPES(M) M(0, 32, 8) M(1, 40, 7) M(2, 32, 12) M(3, 24, 16) M(4, 40, 8) M(5, 40, 10)
constexpr int kNumTmaShapes = 6;
constexpr int kTmaTX[kNumTmaShapes] = {32, 40, 32, 24, 40, 40};
constexpr int kTmaTY[kNumTmaShapes] = {8, 7, 12, 16, 8, 10};
constexpr double kTmaRate[kNumTmaShapes] = {1.0, 1.0, 1.25, 1.12, 1.1, 1.25};

// Plan of the TMA kernel for a lattice: the tile shape and z-chunking with the least modelled
// time of the busiest CTA.  Items (tile, z-chunk) go round robin to the persistent CTAs; a plane
// of an item costs its tile nodes over the shape's rate, and an item about two planes more (its
// two psi-only planes and the pipeline's fill).  forced_shape / forced_zchunk (>= 0 / > 0) pin
// either choice.  lbm_autotune replaces the model by measurement.
void tma_plan(const DevParams& P, int ctas, int forced_shape, int forced_zchunk, int* shape, int* zchunk,
              int* items) {
    double best = -1.0;
    *shape = -1;
    for (int sh = 0; sh < kNumTmaShapes; ++sh) {
        if (forced_shape >= 0 && sh != forced_shape) continue;
        const int tx = kTmaTX[sh], ty = kTmaTY[sh];
        const int tiles = ((P.nx + tx - 1) / tx) * ((P.ny + ty - 1) / ty);
        for (int nch = 1; nch <= P.nz; ++nch) {
            int zc = (P.nz + nch - 1) / nch;
            if (forced_zchunk > 0) zc = forced_zchunk < P.nz ? forced_zchunk : P.nz;
            const int nchunks = (P.nz + zc - 1) / zc;
            if (forced_zchunk <= 0 && zc < 16 && nch > 1) break;
            const long long n = (long long)tiles * nchunks;
            const long long per_cta = (n + ctas - 1) / ctas;
            const double cost = (double)per_cta * tx * ty / kTmaRate[sh] * (zc + 2.0);
            if (best < 0 || cost < best) {
                best = cost;
                *shape = sh;
                *zchunk = zc;
                *items = (int)n;
            }
            if (forced_zchunk > 0) break;
        }
    }
}

// SM count of the current device (queried once per device)
int device_sms() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
    if (dev < 64 && cached[dev] > 0) return cached[dev];
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    if (dev < 64) cached[dev] = n;
    return n;
}

int zchunk_generic(const DevParams& P, int tiles) {
    const int target = device_sms() * 2 * 4;   // about four waves of two CTAs per SM
    int chunks = (target + tiles - 1) / tiles;
    int zc = (P.nz + chunks - 1) / chunks;
    if (zc < 8) zc = 8;
    if (zc > P.nz) zc = P.nz;
    return zc;
}

}  // namespace

long long fused_blocks(const DevParams& P) {
    int tiles = ((P.nx + TX - 1) / TX) * ((P.ny + kTY - 1) / kTY);
    int zc = zchunk_generic(P, tiles);
    return (long long)tiles * ((P.nz + zc - 1) / zc);
}

bool fused_supported(const DevParams& P) { return fused_blocks(P) <= (long long)max_partials(P); }

cudaError_t launch_ghosts(const DevParams& P, int precision, void* pops, cudaStream_t s) {
    const int per_plane = (P.ny + 4) * kSlots + 4 * kSlots * ((P.nx + 3) / 4);
    const dim3 grid((per_plane + 255) / 256, P.nz);
    if (precision == 0) k_ghosts<float><<<grid, 256, 0, s>>>(P, (float*)pops);
    else k_ghosts<__half><<<grid, 256, 0, s>>>(P, (__half*)pops);   // raw 2-byte copies (BF16 or FP16)
    return cudaGetLastError();
}

bool tma_eligible(const DevParams& P, int precision) {
    return precision >= 0 && precision <= 2 && P.qt == 7 && P.nx >= 4 && P.ny >= 4 && f_wraps(P.bc[0]) && f_wraps(P.bc[1]) &&
           f_wraps(P.bc[2]) && f_wraps(P.bc[3]) && !P.flow_off && !P.thermal_off && (!P.wet || precision == 0);
}

size_t tma_smem_bytes(int shape, int precision) {
#define GB300_SMEM(I, X, Y) \
    case I: return precision == 0 ? TmaShape<X, Y, float>::kSmem : TmaShape<X, Y, __half>::kSmem;
    switch (shape) { GB300_TMA_SHAPES(GB300_SMEM) }
#undef GB300_SMEM
    return (size_t)-1;
}

void tma_plan_for(const DevParams& P, int ctas, int forced_shape, int forced_zchunk, int* shape, int* zchunk,
                  int* items) {
    tma_plan(P, ctas, forced_shape, forced_zchunk, shape, zchunk, items);
}

int tma_num_shapes() { return kNumTmaShapes; }
double tma_rate(int shape) { return kTmaRate[shape]; }

int tma_zchunk_candidates(const DevParams& P, int ctas, int shape, int* zcs, int max) {
    // the z-chunks of the shape in increasing modelled cost (distinct, at least 16 planes unless
    // the column is shorter), the whole column included
    const int tx = kTmaTX[shape], ty = kTmaTY[shape];
    const long long tiles = (long long)((P.nx + tx - 1) / tx) * ((P.ny + ty - 1) / ty);
    int n = 0;
    double cost[64];
    int zc_of[64];
    for (int nch = 1; nch <= P.nz && n < 64; ++nch) {
        const int zc = (P.nz + nch - 1) / nch;
        if (zc < 16 && nch > 1) break;
        if (n > 0 && zc_of[n - 1] == zc) continue;
        const long long items = tiles * ((P.nz + zc - 1) / zc);
        cost[n] = (double)((items + ctas - 1) / ctas) * (zc + 2.0);
        zc_of[n++] = zc;
    }
    int out = 0;
    bool taken[64] = {false};
    while (out < max && out < n) {
        int b = -1;
        for (int i = 0; i < n; ++i)
            if (!taken[i] && (b < 0 || cost[i] < cost[b])) b = i;
        taken[b] = true;
        zcs[out++] = zc_of[b];
    }
    return out;
}

int tma_box_w(int shape, int precision) { return kTmaTX[shape] + 2 * (precision == 0 ? 4 : 8); }
int tma_box_h(int shape) { return kTmaTY[shape] + 4; }
int tma_tile_w(int shape) { return kTmaTX[shape]; }
int tma_ghost_cols(int precision) { return precision == 0 ? 4 : 8; }   // 16 bytes of columns
int tma_ghost_mode(const DevParams& P, int shape, int precision) {
    const int tx = tma_tile_w(shape), ty = kTmaTY[shape], gw = tma_ghost_cols(precision);
    // TMA ghost boxes: ghost-column boxes (gw columns = 16 bytes) on 16-byte boundaries, at least
    // two tiles per axis (an edge tile is never both left and right, top and bottom), edge tiles at
    // least gw columns and 2 rows wide, and room for the gw ghost columns past nx in the padded rows
    if (P.nx % gw == 0 && P.nx > tx && P.ny > ty && P.ny % ty != 1 && P.Ws >= P.nx + kGX + gw) return 1;
    return precision == 0 ? 2 : 0;   // direct stores of the images (FP32), else the refresh kernel
}
int tma_tile_h(int shape) { return kTmaTY[shape]; }

cudaError_t launch_fused(const DevParams& P, int precision, const StateBufs& B, const double* sums_cur,
                         double* sums_next, int first, cudaStream_t s, const TmaMaps* maps, bool* ghosts_written) {
    using Sh = FusedShape<kTY>;
    const int tiles_x = (P.nx + TX - 1) / TX, tiles_y = (P.ny + kTY - 1) / kTY;
    cudaError_t e = cudaSuccess;
    if (ghosts_written) *ghosts_written = false;
    if (maps && maps->ok && B.pull_f && B.pull_g && tma_eligible(P, precision)) {
        const int tx = kTmaTX[maps->shape], ty = kTmaTY[maps->shape];
        const int txs = (P.nx + tx - 1) / tx, tys = (P.ny + ty - 1) / ty;
        const int ctas = maps->sms < maps->items ? maps->sms : maps->items;
        if (ghosts_written) *ghosts_written = maps->ghosts != 0;
#define GB300_TMA(TXV, TYV, ST, WET)                                                                           \
        {                                                                                                      \
            using SH = TmaShape<TXV, TYV, ST>;                                                                 \
            e = cudaFuncSetAttribute(k_fused_tma<TXV, TYV, ST, WET>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                     (int)SH::kSmem);                                                          \
            if (e != cudaSuccess) return e;                                                                    \
            k_fused_tma<TXV, TYV, ST, WET><<<ctas, SH::kThreads, SH::kSmem, s>>>(                              \
                maps->m14[B.src_index], maps->m6[B.src_index], maps->mout[B.src_index ^ 1],                    \
                maps->mout_top[B.src_index ^ 1], maps->mgcol[B.src_index ^ 1], maps->mgcol_top[B.src_index ^ 1], \
                maps->mgrow[B.src_index ^ 1], maps->mgrow_right[B.src_index ^ 1], maps->mgcor[B.src_index ^ 1], \
                maps->ghosts, P, (const ST*)B.src, (ST*)B.dst, sums_cur, B.partial, B.counter,                  \
                sums_next, B.phis,                                                                             \
                B.flag, first, maps->zchunk, txs, tys, maps->items);                                           \
        }
        // the wetting wall's solid plane is a separate instantiation (FP32 storage only), so that
        // the kernel without it carries no trace of it
#define GB300_TMA_CASE(I, X, Y)                                                                                \
        case I:                                                                                                \
            if (precision == 0 && P.wet) GB300_TMA(X, Y, float, true)                                          \
            else if (precision == 0) GB300_TMA(X, Y, float, false)                                             \
            else if (precision == 1) GB300_TMA(X, Y, __nv_bfloat16, false)                                     \
            else GB300_TMA(X, Y, __half, false)                                                                \
            break;
        switch (maps->shape) {
            GB300_TMA_SHAPES(GB300_TMA_CASE)
        default: return cudaErrorInvalidValue;
        }
#undef GB300_TMA_CASE
#undef GB300_TMA
        return cudaGetLastError();
    }
    const int zc = zchunk_generic(P, tiles_x * tiles_y);
    dim3 grid(tiles_x, tiles_y, (P.nz + zc - 1) / zc);
    dim3 block(Sh::kThreads);
#define GB300_FUSED(S, QT)                                                                                      \
    {                                                                                                          \
        using ShQ = FusedShape<kTY, QT>;                                                                       \
        e = cudaFuncSetAttribute(k_fused<S, kTY, QT>, cudaFuncAttributeMaxDynamicSharedMemorySize,              \
                                 (int)ShQ::kSmemBytes);                                                        \
        if (e != cudaSuccess) return e;                                                                        \
        k_fused<S, kTY, QT><<<grid, block, ShQ::kSmemBytes, s>>>(P, (const S*)B.src, (S*)B.dst, B.pull_f,        \
                                                                B.pull_g, sums_cur, B.partial, B.counter,      \
                                                                sums_next, B.phis, B.flag, first, zc);         \
    }
    if (P.qt == 19) {   // the D3Q19 temperature lattice: FP32 storage only
        if (precision != 0) return cudaErrorInvalidValue;
        GB300_FUSED(float, 19)
    } else {
        switch (precision) {
        case 0: GB300_FUSED(float, 7) break;
        case 1: GB300_FUSED(__nv_bfloat16, 7) break;
        case 2: GB300_FUSED(__half, 7) break;
        default: return cudaErrorInvalidValue;
        }
    }
#undef GB300_FUSED
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

int batch_tile_rows(int ty) { return ty == 4 ? 4 : kTY; }

int batch_ctas_per_sm(int precision, int ty) {
    int n = 0;
#define GB300_OCC(S, TYV)                                                                                      \
    {                                                                                                          \
        using Sh = FusedShape<TYV>;                                                                            \
        if (cudaFuncSetAttribute(k_fused_batch<S, TYV>, cudaFuncAttributeMaxDynamicSharedMemorySize,            \
                                 (int)Sh::kSmemBytes) != cudaSuccess ||                                        \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused_batch<S, TYV>, Sh::kThreads,             \
                                                          Sh::kSmemBytes) != cudaSuccess)                      \
            n = 0;                                                                                             \
    }
#define GB300_OCC_TY(S) { if (ty == 4) GB300_OCC(S, 4) else GB300_OCC(S, kTY) }
    switch (precision) {
    case 0: GB300_OCC_TY(float) break;
    case 1: GB300_OCC_TY(__nv_bfloat16) break;
    case 2: GB300_OCC_TY(__half) break;
    }
#undef GB300_OCC_TY
#undef GB300_OCC
    cudaGetLastError();
    return n;
}

cudaError_t launch_fused_batch(const DevParams& P, int precision, int ty, const BatchInst* insts,
                               const BatchItem* items, int n_items, int n_inst, const StateBufs& B,
                               const double* sums_cur, double* sums_next, int first, int ctas, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
#define GB300_BATCH(S, TYV)                                                                                    \
    {                                                                                                          \
        using Sh = FusedShape<TYV>;                                                                            \
        e = cudaFuncSetAttribute(k_fused_batch<S, TYV>, cudaFuncAttributeMaxDynamicSharedMemorySize,            \
                                 (int)Sh::kSmemBytes);                                                         \
        if (e != cudaSuccess) return e;                                                                        \
        k_fused_batch<S, TYV><<<ctas, Sh::kThreads, Sh::kSmemBytes, s>>>(                                      \
            P, insts, items, n_items, n_inst, (const S*)B.src, (S*)B.dst, B.pull_f, B.pull_g, sums_cur,        \
            B.partial, B.counter, sums_next, B.phis, B.flag, first);                                           \
    }
#define GB300_BATCH_TY(S) { if (ty == 4) GB300_BATCH(S, 4) else GB300_BATCH(S, kTY) }
    switch (precision) {
    case 0: GB300_BATCH_TY(float) break;
    case 1: GB300_BATCH_TY(__nv_bfloat16) break;
    case 2: GB300_BATCH_TY(__half) break;
    default: return cudaErrorInvalidValue;
    }
#undef GB300_BATCH_TY
#undef GB300_BATCH
    return cudaGetLastError();
}

}  // namespace gb300lbm
