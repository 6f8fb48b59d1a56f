// Fused z-marching variant of the lattice update: one kernel per time step.
//
// A CTA owns a 32 x TY tile of (x, y) columns and marches through a chunk of z-planes.  For
// every plane it
//   phase A: pulls the 26 populations of each tile node and of the one-node halo ring around
//            the tile, forms rho = sum f (Eq. 10), T = sum g (Eq. 20) and psi (Eq. 8 with the
//            Peng-Robinson EOS, Eq. 49), and keeps (psi, rho) in a 3-plane shared-memory ring;
//            the tile's own populations are parked in shared memory for phase B;
//   phase B: collides the previous plane: interaction force (Eq. 7) and grad rho from the ring,
//            buoyancy, D3Q19 MRT collision (Eqs. 3-6, 9, 10), div u (Eq. 48), grad T (Eq. 45),
//            phi_s (Eq. 18), source Q (Eq. 23) and the D3Q7 MRT collision (Eqs. 38-43), and
//            stores f*, g+ and phi_s.
// psi and rho never go to HBM: the halo ring is recomputed from the populations (26 extra
// population reads per halo node, mostly L2 hits because neighbouring CTAs march through the
// same planes at the same time).  rho_ave for the buoyancy force is the deterministic FP64
// mean of this step's rho, used by the next step.
#include "lbm_launch.h"

namespace gb300lbm {

namespace {

constexpr int TX = 32;

template <int TY> struct FusedShape {
    static constexpr int kInterior = TX * TY;
    static constexpr int kHaloNodes = 2 * (TX + 2) + 2 * TY;
    static constexpr int kHaloThreads = ((kHaloNodes + 31) / 32) * 32;
    static constexpr int kThreads = kInterior + kHaloThreads;
    static constexpr int kRingW = TX + 2, kRingH = TY + 2;
    static constexpr int kRingPlane = kRingW * kRingH;
    // shared memory: two population stages of the tile (float) + the (psi, rho) ring
    static constexpr size_t kStageFloats = 26 * kInterior;
    static constexpr size_t kSmemBytes = 2 * kStageFloats * sizeof(float) + 3 * kRingPlane * sizeof(float2);
};

// coordinate of the node whose (psi, rho) fills a ring slot at coordinate c (may be -1 or n):
// wrap for periodic (f) faces, mirror (= clamp for one layer) for walls and outflow faces.
__device__ __forceinline__ int map_coord(int c, int n, int bc_lo, int bc_hi) {
    if (c < 0) return f_wraps(bc_lo) ? c + n : 0;
    if (c >= n) return f_wraps(bc_hi) ? c - n : n - 1;
    return c;
}

template <typename S, int TY>
__global__ void __launch_bounds__(FusedShape<TY>::kThreads, 2)
k_fused(DevParams P, const S* __restrict__ fs, const S* __restrict__ gs, S* __restrict__ fd,
        S* __restrict__ gd, int pull_f, int pull_g, const double* __restrict__ sums_cur, double2* partial,
        unsigned* counter, double* sums_next, float* __restrict__ phis, int* flag, int first, int zchunk) {
    using Sh = FusedShape<TY>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* stage = reinterpret_cast<float*>(smem_raw);                       // [2][26][TY][32]
    float2* ring = reinterpret_cast<float2*>(stage + 2 * Sh::kStageFloats);  // [3][TY+2][34]

    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(P.nz, z0 + zchunk);

    // ring slot handled by this thread in phase A
    int lx = -1, ly = -1;
    const bool interior = tid < Sh::kInterior;
    if (interior) {
        lx = (tid & 31) + 1;
        ly = (tid >> 5) + 1;
    } else {
        int h = tid - Sh::kInterior;
        if (h < TX + 2) { lx = h; ly = 0; }
        else if (h < 2 * (TX + 2)) { lx = h - (TX + 2); ly = TY + 1; }
        else if (h < Sh::kHaloNodes) { int k = h - 2 * (TX + 2); lx = (k & 1) ? TX + 1 : 0; ly = 1 + (k >> 1); }
    }
    const int gx = x0 + lx - 1, gy = y0 + ly - 1;
    // slots outside [-1, n] are never read by any stencil
    const bool slot_used = lx >= 0 && gx >= -1 && gx <= P.nx && gy >= -1 && gy <= P.ny;
    const int mx = slot_used ? map_coord(gx, P.nx, P.bc[0], P.bc[1]) : 0;
    const int my = slot_used ? map_coord(gy, P.ny, P.bc[2], P.bc[3]) : 0;
    // this thread's own node takes part in phase B
    const bool owner = interior && gx < P.nx && gy < P.ny;
    const int slot = ly * Sh::kRingW + lx;

    double r_acc = 0.0, t_acc = 0.0;
    int bad = 0;
    const float rho_ave = (float)(sums_cur[0] / (double)P.N);

    // ---------------------------------------------------------------- phase A for plane zp
    auto phase_a = [&](int zp) {
        if (!slot_used) return;
        const bool in_chunk = zp >= z0 && zp < z1;
        const int mz = map_coord(zp, P.nz, P.bc[4], P.bc[5]);
        const int i = node_of(P, mx, my, mz);
        Nbr n = make_nbr(P, mx, my, mz);
        float f[19], g[7];
        load_f<S>(P, fs, pull_f, i, mx, my, mz, n, f);
        load_g<S>(P, gs, pull_g, i, mx, my, mz, n, g);
        float rho = 0.f, T = 0.f;
#pragma unroll
        for (int a = 0; a < 19; ++a) rho += f[a];
#pragma unroll
        for (int a = 0; a < 7; ++a) T += g[a];
        float psi2 = psi_squared(P, rho, T);
        ring[((zp + 3) % 3) * Sh::kRingPlane + slot] = make_float2(sqrtf(psi2), rho);
        if (owner && in_chunk) {
            float* st = stage + ((zp - z0) & 1) * Sh::kStageFloats + tid;
#pragma unroll
            for (int a = 0; a < 19; ++a) st[a * Sh::kInterior] = f[a];
#pragma unroll
            for (int a = 0; a < 7; ++a) st[(19 + a) * Sh::kInterior] = g[a];
            r_acc += (double)rho;
            t_acc += (double)T;
            bad |= !(psi2 > 0.f) || !isfinite(rho) || !isfinite(T);
        }
    };

    // ---------------------------------------------------------------- phase B for plane z
    auto phase_b = [&](int z) {
        if (!owner) return;
        const int x = gx, y = gy;
        const int i = node_of(P, x, y, z);
        const float* st = stage + ((z - z0) & 1) * Sh::kStageFloats + tid;
        float f[19], g[7];
#pragma unroll
        for (int a = 0; a < 19; ++a) f[a] = st[a * Sh::kInterior];
#pragma unroll
        for (int a = 0; a < 7; ++a) g[a] = st[(19 + a) * Sh::kInterior];
        float rho = 0.f, T = 0.f;
#pragma unroll
        for (int a = 0; a < 19; ++a) rho += f[a];
#pragma unroll
        for (int a = 0; a < 7; ++a) T += g[a];
        const float2* rm = ring + ((z + 2) % 3) * Sh::kRingPlane;   // plane z - 1
        const float2* r0 = ring + (z % 3) * Sh::kRingPlane;
        const float2* rp = ring + ((z + 1) % 3) * Sh::kRingPlane;   // plane z + 1
        const float2 me = r0[slot];
        float Fx = 0.f, Fy = 0.f, Fz = 0.f, grx = 0.f, gry = 0.f, grz = 0.f;
        const int W = Sh::kRingW;
#define GB300_NB(PL, DX, DY, DZ, WGT)                                      \
        {                                                                  \
            float2 q = PL[slot + (DY) * W + (DX)];                         \
            if (DX) { Fx += (DX * WGT) * q.x; grx += (DX * WGT) * q.y; }   \
            if (DY) { Fy += (DY * WGT) * q.x; gry += (DY * WGT) * q.y; }   \
            if (DZ) { Fz += (DZ * WGT) * q.x; grz += (DZ * WGT) * q.y; }   \
        }
        const float w1 = 1.f / 6.f, w2 = 1.f / 12.f;
        GB300_NB(r0, 1, 0, 0, w1) GB300_NB(r0, -1, 0, 0, w1) GB300_NB(r0, 0, 1, 0, w1) GB300_NB(r0, 0, -1, 0, w1)
        GB300_NB(rp, 0, 0, 1, w1) GB300_NB(rm, 0, 0, -1, w1)
        GB300_NB(r0, 1, 1, 0, w2) GB300_NB(r0, -1, -1, 0, w2) GB300_NB(r0, 1, -1, 0, w2) GB300_NB(r0, -1, 1, 0, w2)
        GB300_NB(rp, 1, 0, 1, w2) GB300_NB(rm, -1, 0, -1, w2) GB300_NB(rm, 1, 0, -1, w2) GB300_NB(rp, -1, 0, 1, w2)
        GB300_NB(rp, 0, 1, 1, w2) GB300_NB(rm, 0, -1, -1, w2) GB300_NB(rm, 0, 1, -1, w2) GB300_NB(rp, 0, -1, 1, w2)
#undef GB300_NB
        float Fmx = me.x * Fx, Fmy = me.x * Fy, Fmz = me.x * Fz;
        float db = rho - rho_ave;
        float Fm2 = Fmx * Fmx + Fmy * Fmy + Fmz * Fmz;
        NodeOut o = collide_f(P, f, Fmx + db * P.gx, Fmy + db * P.gy, Fmz + db * P.gz, Fm2, me.x * me.x);
        if (!P.flow_off) {
#pragma unroll
            for (int a = 0; a < 19; ++a) Codec<S>::store(fd + (size_t)a * P.N + i, f[a], P.shift_f[a]);
        }
        float ph = collide_g(P, g, rho, T, o, grx, gry, grz, phis[i], first);
        if (!P.thermal_off) {
#pragma unroll
            for (int a = 0; a < 7; ++a) Codec<S>::store(gd + (size_t)a * P.N + i, g[a], P.shift_g[a]);
        }
        phis[i] = ph;
    };

    phase_a(z0 - 1);
    phase_a(z0);
    __syncthreads();
    for (int z = z0; z < z1; ++z) {
        phase_a(z + 1);
        __syncthreads();
        phase_b(z);
        __syncthreads();
    }

    if (__syncthreads_or(bad) && tid == 0) atomicOr(flag, 1);
    // deterministic FP64 sums of this step's rho and T (rho_ave of the next step)
    {
        __shared__ double sa[Sh::kThreads / 32], sb[Sh::kThreads / 32];
        __shared__ int is_last;
        double a = r_acc, b = t_acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        if ((tid & 31) == 0) { sa[tid >> 5] = a; sb[tid >> 5] = b; }
        __syncthreads();
        const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
        const int nblocks = gridDim.x * gridDim.y * gridDim.z;
        if (tid == 0) {
            double ta = 0.0, tb = 0.0;
            for (int w = 0; w < Sh::kThreads / 32; ++w) { ta += sa[w]; tb += sb[w]; }
            partial[bid] = make_double2(ta, tb);
            __threadfence();
            is_last = atomicAdd(counter, 1u) == (unsigned)(nblocks - 1);
        }
        __syncthreads();
        if (is_last) {
            __threadfence();
            double ta = 0.0, tb = 0.0;
            for (int k = tid; k < nblocks; k += Sh::kThreads) {
                double2 p = __ldcg(partial + k);
                ta += p.x;
                tb += p.y;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ta += __shfl_down_sync(0xffffffffu, ta, o);
                tb += __shfl_down_sync(0xffffffffu, tb, o);
            }
            __syncthreads();
            if ((tid & 31) == 0) { sa[tid >> 5] = ta; sb[tid >> 5] = tb; }
            __syncthreads();
            if (tid == 0) {
                double ra = 0.0, rb = 0.0;
                for (int w = 0; w < Sh::kThreads / 32; ++w) { ra += sa[w]; rb += sb[w]; }
                sums_next[0] = ra;
                sums_next[1] = rb;
                *counter = 0u;
            }
        }
    }
}

constexpr int kTY = 8;

int zchunk_for(const DevParams& P, int tiles) {
    // enough CTAs for about four waves of two CTAs per SM on 152 SMs, chunks of >= 8 planes
    const int target = 152 * 2 * 4;
    int chunks = (target + tiles - 1) / tiles;
    int zc = (P.nz + chunks - 1) / chunks;
    if (zc < 8) zc = 8;
    if (zc > P.nz) zc = P.nz;
    return zc;
}

}  // namespace

bool fused_supported(const DevParams& P) {
    // the grid's CTA count must fit the partial-sum buffer of the reductions
    int tiles = ((P.nx + TX - 1) / TX) * ((P.ny + kTY - 1) / kTY);
    int zc = zchunk_for(P, tiles);
    long long blocks = (long long)tiles * ((P.nz + zc - 1) / zc);
    return blocks <= (long long)max_partials(P);
}

cudaError_t launch_fused(const DevParams& P, int precision, const StateBufs& B, const double* sums_cur,
                         double* sums_next, int first, cudaStream_t s) {
    using Sh = FusedShape<kTY>;
    int tiles_x = (P.nx + TX - 1) / TX, tiles_y = (P.ny + kTY - 1) / kTY;
    int zc = zchunk_for(P, tiles_x * tiles_y);
    dim3 grid(tiles_x, tiles_y, (P.nz + zc - 1) / zc);
    dim3 block(Sh::kThreads);
    cudaError_t e = cudaSuccess;
#define GB300_FUSED(S)                                                                                     \
    {                                                                                                     \
        e = cudaFuncSetAttribute(k_fused<S, kTY>, cudaFuncAttributeMaxDynamicSharedMemorySize,            \
                                 (int)Sh::kSmemBytes);                                                    \
        if (e != cudaSuccess) return e;                                                                   \
        k_fused<S, kTY><<<grid, block, Sh::kSmemBytes, s>>>(P, (const S*)B.fsrc, (const S*)B.gsrc,       \
                                                            (S*)B.fdst, (S*)B.gdst, B.pull_f, B.pull_g,   \
                                                            sums_cur, B.partial, B.counter, sums_next,    \
                                                            B.phis, B.flag, first, zc);                   \
    }
    switch (precision) {
    case 0: GB300_FUSED(float) break;
    case 1: GB300_FUSED(__nv_bfloat16) break;
    case 2: GB300_FUSED(__half) break;
    default: return cudaErrorInvalidValue;
    }
#undef GB300_FUSED
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace gb300lbm
