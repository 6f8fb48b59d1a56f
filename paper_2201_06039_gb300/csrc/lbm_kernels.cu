// Two-pass kernels of the lattice update, initialisation, moments and deterministic
// FP64 reductions.  See lbm_device.cuh for the per-node arithmetic.
#include "lbm_launch.h"

namespace gb300lbm {

constexpr int TPB_X = 32, TPB_Y = 8, TPB = TPB_X * TPB_Y;
constexpr int SUM_BLOCKS_MAX = 1184;   // 8 x 148-152 SMs worth of blocks for field sums

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic two-value FP64 sum over the grid: each block writes its partial, the last
// block to finish (atomic ticket) adds the partials in index order and resets the ticket.
// The result depends only on the grid shape, never on block scheduling.
template <int NT>
__device__ void grid_sum2(double a, double b, double2* partial, unsigned* counter, double* out) {
    __shared__ double sa[NT / 32], sb[NT / 32];
    __shared__ int is_last;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int nblocks = gridDim.x * gridDim.y * gridDim.z;
    a = warp_sum(a);
    b = warp_sum(b);
    if ((tid & 31) == 0) { sa[tid >> 5] = a; sb[tid >> 5] = b; }
    __syncthreads();
    if (tid == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < NT / 32; ++w) { ta += sa[w]; tb += sb[w]; }
        partial[bid] = make_double2(ta, tb);
        __threadfence();
        unsigned ticket = atomicAdd(counter, 1u);
        is_last = (ticket == (unsigned)(nblocks - 1));
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double ta = 0.0, tb = 0.0;
    for (int k = tid; k < nblocks; k += NT) {
        double2 p = __ldcg(partial + k);
        ta += p.x;
        tb += p.y;
    }
    ta = warp_sum(ta);
    tb = warp_sum(tb);
    __syncthreads();
    if ((tid & 31) == 0) { sa[tid >> 5] = ta; sb[tid >> 5] = tb; }
    __syncthreads();
    if (tid == 0) {
        double ra = 0.0, rb = 0.0;
        for (int w = 0; w < NT / 32; ++w) { ra += sa[w]; rb += sb[w]; }
        out[0] = ra;
        out[1] = rb;
        *counter = 0u;
    }
}

// ---------------------------------------------------------------- init
template <typename S, int QT>
__global__ void __launch_bounds__(TPB) k_init(DevParams P, S* __restrict__ pops, const float* __restrict__ rho,
                                             const float* __restrict__ T, const float* __restrict__ u) {
    int x = blockIdx.x * TPB_X + threadIdx.x, y = blockIdx.y * TPB_Y + threadIdx.y, z = blockIdx.z;
    if (x >= P.nx || y >= P.ny) return;
    int d = node_of(P, x, y, z);
    float r = rho[d], t = T[d];
    float ux = 0.f, uy = 0.f, uz = 0.f;
    if (u) { ux = u[d]; uy = u[P.N + d]; uz = u[2 * P.N + d]; }
    float fe[19], ge[QT];
    feq(r, ux, uy, uz, fe);
    Therm<QT>::equilibrium(P, t, ge);
    Therm<QT>::template store<S>(P, pops, sidx(P, x, y, z), fe, ge);
}

// ---------------------------------------------------------------- psi / EOS pass (S1-S2)
template <typename S, int QT>
__global__ void __launch_bounds__(TPB) k_psi(DevParams P, const S* __restrict__ fs, int pull_f, int pull_g, float2* __restrict__ psirho,
                                            double2* partial, unsigned* counter, double* sums, int* flag) {
    int x = blockIdx.x * TPB_X + threadIdx.x, y = blockIdx.y * TPB_Y + threadIdx.y, z = blockIdx.z;
    double ra = 0.0, ta = 0.0;
    int bad = 0;
    if (x < P.nx && y < P.ny) {
        int i = sidx(P, x, y, z);
        Nbr n = make_nbr(P, x, y, z);
        float f[19], g[QT];
        load_f<S>(P, fs, pull_f, i, x, y, z, n, f);
        Therm<QT>::template load<S>(P, fs, pull_g, i, x, y, z, n, g);
        float rho = sum19(f), T = Therm<QT>::sum(g);
        float psi2 = psi_squared(P, rho, T);
        bad = !(psi2 > 0.f) || !isfinite(rho) || !isfinite(T);
        psirho[bidx(P, node_of(P, x, y, z), P.N)] = make_float2(psi_of(psi2), rho);
        ra = rho;
        ta = T;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0 && threadIdx.y == 0) atomicOr(flag, 1);
    if (sums) grid_sum2<TPB>(ra, ta, partial, counter, sums);
}

// ---------------------------------------------------------------- neighbourhood terms (S3-S4)
// F_m = -G psi(x) sum w psi(x+e) e (Eq. 7, G = -1) and grad rho = sum w rho(x+e) e.
struct Stencil {
    float2 x, y, z;   // (F component, grad rho component) per axis
};

// one neighbour's (psi, rho) added to each axis pair with one paired FP32 fma, in the order and
// the rounding of the fused kernels' ring stencil
template <int A>
__device__ __forceinline__ void stencil_term(const DevParams& P, const float2* __restrict__ pr, int x, int y,
                                             int z, const Nbr& n, Stencil& s) {
    constexpr int ex = ex19(A), ey = ey19(A), ez = ez19(A);
    constexpr float w = (ex * ex + ey * ey + ez * ez) == 1 ? (1.f / 6.f) : (1.f / 12.f);
    int j = (int)bidx(P, node_of(P, nb_c(ex, x, n.xm, n.xp), nb_c(ey, y, n.ym, n.yp), nb_c(ez, z, n.zm, n.zp)), P.N);
    float2 q;
    if (ez < 0 && z == 0 && P.wet)   // solid layer below a wetting -z wall: virtual (psi, rho)
        q = wall_entry(P, nb_c(ex, x, n.xm, n.xp), nb_c(ey, y, n.ym, n.yp));
    else
        q = __ldg(pr + j);
    if (ex) s.x = __ffma2_rn(make_float2(ex * w, ex * w), q, s.x);
    if (ey) s.y = __ffma2_rn(make_float2(ey * w, ey * w), q, s.y);
    if (ez) s.z = __ffma2_rn(make_float2(ez * w, ez * w), q, s.z);
}

__device__ __forceinline__ Stencil stencil(const DevParams& P, const float2* __restrict__ pr, int x, int y,
                                           int z, const Nbr& n) {
    Stencil s = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    stencil_term<1>(P, pr, x, y, z, n, s); stencil_term<2>(P, pr, x, y, z, n, s);
    stencil_term<3>(P, pr, x, y, z, n, s); stencil_term<4>(P, pr, x, y, z, n, s);
    stencil_term<5>(P, pr, x, y, z, n, s); stencil_term<6>(P, pr, x, y, z, n, s);
    stencil_term<7>(P, pr, x, y, z, n, s); stencil_term<8>(P, pr, x, y, z, n, s);
    stencil_term<9>(P, pr, x, y, z, n, s); stencil_term<10>(P, pr, x, y, z, n, s);
    stencil_term<11>(P, pr, x, y, z, n, s); stencil_term<12>(P, pr, x, y, z, n, s);
    stencil_term<13>(P, pr, x, y, z, n, s); stencil_term<14>(P, pr, x, y, z, n, s);
    stencil_term<15>(P, pr, x, y, z, n, s); stencil_term<16>(P, pr, x, y, z, n, s);
    stencil_term<17>(P, pr, x, y, z, n, s); stencil_term<18>(P, pr, x, y, z, n, s);
    return s;
}

// ---------------------------------------------------------------- velocity pass
// u = (sum e f + F/2) / rho (Eq. 10, total force F) of every node, for the finite-difference
// div u of the collide pass (divu_mode 1); same arithmetic as the collision's u.
template <typename S>
__global__ void __launch_bounds__(TPB) k_velocity(DevParams P, const S* __restrict__ fs, int pull_f,
                                                 const float2* __restrict__ psirho,
                                                 const double* __restrict__ sums_cur, float4* __restrict__ vel) {
    int x = blockIdx.x * TPB_X + threadIdx.x, y = blockIdx.y * TPB_Y + threadIdx.y, z = blockIdx.z;
    if (x >= P.nx || y >= P.ny) return;
    int i = sidx(P, x, y, z), d = (int)bidx(P, node_of(P, x, y, z), P.N);
    Nbr n = make_nbr(P, x, y, z);
    float f[19];
    load_f<S>(P, fs, pull_f, i, x, y, z, n, f);
    float rho = sum19(f);
    float jx = (f[1] - f[2]) + (f[7] - f[8]) + (f[9] - f[10]) + (f[11] - f[12]) + (f[13] - f[14]);
    float jy = (f[3] - f[4]) + (f[7] - f[8]) - (f[9] - f[10]) + (f[15] - f[16]) + (f[17] - f[18]);
    float jz = (f[5] - f[6]) + (f[11] - f[12]) - (f[13] - f[14]) + (f[15] - f[16]) - (f[17] - f[18]);
    float2 me = __ldg(psirho + d);
    Stencil st = stencil(P, psirho, x, y, z, n);
    const Forces F = total_force(P, me.x, st.x.x, st.y.x, st.z.x, rho - buoyancy_ref(P, sums_cur[0], P.inv_N));
    const float inv_rho = __fdividef(1.f, rho);
    vel[d] = make_float4((jx + 0.5f * F.Fx) * inv_rho, (jy + 0.5f * F.Fy) * inv_rho, (jz + 0.5f * F.Fz) * inv_rho, 0.f);
}

// Does the gradient stencil of (x, y, z) reach past a wall or outflow face?  There div u stays
// Eq. 48 in divu_mode 1.
__device__ __forceinline__ bool next_to_solid(const DevParams& P, int x, int y, int z) {
    return (x == 0 && !f_wraps(P.bc[0])) || (x == P.nx - 1 && !f_wraps(P.bc[1])) ||
           (y == 0 && !f_wraps(P.bc[2])) || (y == P.ny - 1 && !f_wraps(P.bc[3])) ||
           (z == 0 && !f_wraps(P.bc[4])) || (z == P.nz - 1 && !f_wraps(P.bc[5]));
}

// isotropic finite-difference divergence: sum_a W_a e_a . u(x + e_a), W = 1/6 (faces), 1/12 (edges)
template <int A>
__device__ __forceinline__ void fd_term(const DevParams& P, const float4* __restrict__ vel, int x, int y, int z,
                                        const Nbr& n, float& acc) {
    constexpr int ex = ex19(A), ey = ey19(A), ez = ez19(A);
    constexpr float w = (ex * ex + ey * ey + ez * ez) == 1 ? (1.f / 6.f) : (1.f / 12.f);
    const float4 q = __ldg(vel + node_of(P, nb_c(ex, x, n.xm, n.xp), nb_c(ey, y, n.ym, n.yp), nb_c(ez, z, n.zm, n.zp)));
    if (ex) acc = __fmaf_rn(ex * w, q.x, acc);
    if (ey) acc = __fmaf_rn(ey * w, q.y, acc);
    if (ez) acc = __fmaf_rn(ez * w, q.z, acc);
}
__device__ __forceinline__ float fd_divergence(const DevParams& P, const float4* __restrict__ vel, int x, int y,
                                               int z, const Nbr& n) {
    float acc = 0.f;
    fd_term<1>(P, vel, x, y, z, n, acc); fd_term<2>(P, vel, x, y, z, n, acc);
    fd_term<3>(P, vel, x, y, z, n, acc); fd_term<4>(P, vel, x, y, z, n, acc);
    fd_term<5>(P, vel, x, y, z, n, acc); fd_term<6>(P, vel, x, y, z, n, acc);
    fd_term<7>(P, vel, x, y, z, n, acc); fd_term<8>(P, vel, x, y, z, n, acc);
    fd_term<9>(P, vel, x, y, z, n, acc); fd_term<10>(P, vel, x, y, z, n, acc);
    fd_term<11>(P, vel, x, y, z, n, acc); fd_term<12>(P, vel, x, y, z, n, acc);
    fd_term<13>(P, vel, x, y, z, n, acc); fd_term<14>(P, vel, x, y, z, n, acc);
    fd_term<15>(P, vel, x, y, z, n, acc); fd_term<16>(P, vel, x, y, z, n, acc);
    fd_term<17>(P, vel, x, y, z, n, acc); fd_term<18>(P, vel, x, y, z, n, acc);
    return acc;
}

// ---------------------------------------------------------------- stream-collide pass (S3-S12)
template <typename S, int QT>
__global__ void __launch_bounds__(TPB) k_collide(DevParams P, const S* __restrict__ fs, S* __restrict__ fd,
                                                int pull_f, int pull_g,
                                                const float2* __restrict__ psirho, const double* __restrict__ sums_cur,
                                                float* __restrict__ phis, int first, const float4* __restrict__ vel) {
    int x = blockIdx.x * TPB_X + threadIdx.x, y = blockIdx.y * TPB_Y + threadIdx.y, z = blockIdx.z;
    if (x >= P.nx || y >= P.ny) return;
    int i = sidx(P, x, y, z), d = (int)bidx(P, node_of(P, x, y, z), P.N);
    Nbr n = make_nbr(P, x, y, z);
    float f[19], g[QT];
    load_f<S>(P, fs, pull_f, i, x, y, z, n, f);
    Therm<QT>::template load<S>(P, fs, pull_g, i, x, y, z, n, g);
    float rho = sum19(f), T = Therm<QT>::sum(g);
    float2 me = __ldg(psirho + d);
    Stencil st = stencil(P, psirho, x, y, z, n);
    float rho_ave = buoyancy_ref(P, sums_cur[0], P.inv_N);
    const Forces F = total_force(P, me.x, st.x.x, st.y.x, st.z.x, rho - rho_ave);
    NodeOut o = collide_f(P, f, rho, F.Fx, F.Fy, F.Fz, F.Fm2, me.x * me.x);
    if (vel && !next_to_solid(P, x, y, z)) o.divu = fd_divergence(P, vel, x, y, z, n);   // divu_mode 1
    float ph = Therm<QT>::collide(P, g, rho, T, o, st.x.y, st.y.y, st.z.y, phis[d], first);
    // frozen fields keep their stored values (no streaming, no collision)
    if (P.flow_off) {
#pragma unroll
        for (int a = 0; a < 19; ++a) f[a] = Codec<S>::load(fs + (size_t)fslot(a) * P.Ns + i, P.shift_f[a]);
    }
    if (P.thermal_off) Therm<QT>::template stored<S>(P, fs, i, g);
    Therm<QT>::template store<S>(P, fd, i, f, g);
    phis[d] = ph;
}

// ---------------------------------------------------------------- moments (lbm_get_moments)
template <typename S, int QT>
__global__ void __launch_bounds__(TPB) k_moments(DevParams P, const S* __restrict__ fs, int pull_f, int pull_g, const float2* __restrict__ psirho,
                                                const double* __restrict__ sums_cur, float* __restrict__ orho,
                                                float* __restrict__ oux, float* __restrict__ ouy,
                                                float* __restrict__ ouz, float* __restrict__ oT) {
    int x = blockIdx.x * TPB_X + threadIdx.x, y = blockIdx.y * TPB_Y + threadIdx.y, z = blockIdx.z;
    if (x >= P.nx || y >= P.ny) return;
    int i = sidx(P, x, y, z);
    Nbr n = make_nbr(P, x, y, z);
    float f[19], g[QT];
    load_f<S>(P, fs, pull_f, i, x, y, z, n, f);
    Therm<QT>::template load<S>(P, fs, pull_g, i, x, y, z, n, g);
    float rho = sum19(f), T = Therm<QT>::sum(g);
    i = node_of(P, x, y, z);
    float jx = (f[1] - f[2]) + (f[7] - f[8]) + (f[9] - f[10]) + (f[11] - f[12]) + (f[13] - f[14]);
    float jy = (f[3] - f[4]) + (f[7] - f[8]) - (f[9] - f[10]) + (f[15] - f[16]) + (f[17] - f[18]);
    float jz = (f[5] - f[6]) + (f[11] - f[12]) - (f[13] - f[14]) + (f[15] - f[16]) - (f[17] - f[18]);
    float2 me = __ldg(psirho + i);
    Stencil st = stencil(P, psirho, x, y, z, n);
    float rho_ave = buoyancy_ref(P, sums_cur[0], P.inv_N);
    float db = rho - rho_ave;
    float Fx = me.x * st.x.x + db * P.gx, Fy = me.x * st.y.x + db * P.gy, Fz = me.x * st.z.x + db * P.gz;
    float inv = 1.f / rho;
    bool fz = P.flow_off != 0;
    if (orho) orho[i] = rho;
    if (oux) oux[i] = fz ? 0.f : (jx + 0.5f * Fx) * inv;
    if (ouy) ouy[i] = fz ? 0.f : (jy + 0.5f * Fy) * inv;
    if (ouz) ouz[i] = fz ? 0.f : (jz + 0.5f * Fz) * inv;
    if (oT) oT[i] = T;
}

// ---------------------------------------------------------------- field sum
__global__ void __launch_bounds__(256) k_sum_field(const float* __restrict__ a, int n, double2* partial,
                                                   unsigned* counter, double* out) {
    double acc = 0.0;
    for (int i = blockIdx.x * 256 + threadIdx.x; i < n; i += gridDim.x * 256) acc += (double)a[i];
    grid_sum2<256>(acc, 0.0, partial, counter, out);
}

// ---------------------------------------------------------------- launchers
static dim3 grid_of(const DevParams& P) {
    return dim3((P.nx + TPB_X - 1) / TPB_X, (P.ny + TPB_Y - 1) / TPB_Y, P.nz);
}

int reduce_blocks_psi(const DevParams& P) {   // also bounds the fused kernels' blocks / items
    dim3 g = grid_of(P);
    return (int)(g.x * g.y * g.z);
}

int max_partials(const DevParams& P) {
    int a = reduce_blocks_psi(P);
    return a > SUM_BLOCKS_MAX ? a : SUM_BLOCKS_MAX;
}

#define GB300_DISPATCH(prec, CALL)                                          \
    switch (prec) {                                                          \
    case 0: { using S = float; CALL; break; }                                \
    case 1: { using S = __nv_bfloat16; CALL; break; }                        \
    case 2: { using S = __half; CALL; break; }                               \
    default: return cudaErrorInvalidValue;                                   \
    }
// storage type and temperature lattice (QT = 19 with FP32 storage only)
#define GB300_DISPATCH_QT(P, prec, CALL)                                     \
    if ((P).qt == 19) {                                                      \
        if (prec != 0) return cudaErrorInvalidValue;                         \
        using S = float;                                                     \
        constexpr int QT = 19;                                               \
        CALL;                                                                \
    } else {                                                                 \
        constexpr int QT = 7;                                                \
        GB300_DISPATCH(prec, CALL)                                           \
    }

cudaError_t launch_init(const DevParams& P, int precision, void* pops, const float* rho, const float* T,
                        const float* u, cudaStream_t s) {
    dim3 blk(TPB_X, TPB_Y);
    GB300_DISPATCH_QT(P, precision, (k_init<S, QT><<<grid_of(P), blk, 0, s>>>(P, (S*)pops, rho, T, u)));
    return cudaGetLastError();
}

cudaError_t launch_psi(const DevParams& P, int precision, const StateBufs& B, double* sums, cudaStream_t s) {
    dim3 blk(TPB_X, TPB_Y);
    GB300_DISPATCH_QT(P, precision, (k_psi<S, QT><<<grid_of(P), blk, 0, s>>>(P, (const S*)B.src, B.pull_f, B.pull_g, B.psirho,
                                                                    B.partial, B.counter, sums, B.flag)));
    return cudaGetLastError();
}

cudaError_t launch_collide(const DevParams& P, int precision, const StateBufs& B, const double* sums_cur,
                           int first, cudaStream_t s) {
    dim3 blk(TPB_X, TPB_Y);
    GB300_DISPATCH_QT(P, precision, (k_collide<S, QT><<<grid_of(P), blk, 0, s>>>(P, (const S*)B.src, (S*)B.dst, B.pull_f,
                                                                        B.pull_g, B.psirho, sums_cur, B.phis, first,
                                                                        B.vel)));
    return cudaGetLastError();
}

// (psi, rho) of the virtual-density solid layer below the -z wall, one entry per (x, y).  For
// scheme 1 the mean density of the solid node's fluid neighbours, (x, y, 0) with weight 1/6 and
// its four in-plane neighbours with 1/12 each (sum of weights 1/2), comes from the populations
// this step pulls, summed as the psi pass sums them.
template <typename S>
__global__ void __launch_bounds__(128) k_wall_table(DevParams P, const S* __restrict__ fs, int pull_f,
                                                    float2* __restrict__ tab) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    float rho_ave = 0.f;
    if (P.wet_scheme == 1) {
        const Nbr n = make_nbr(P, x, y, 0);
        auto rho_at = [&](int xx, int yy) {
            const Nbr m = make_nbr(P, xx, yy, 0);
            float f[19];
            load_f<S>(P, fs, pull_f, sidx(P, xx, yy, 0), xx, yy, 0, m, f);
            return sum19(f);
        };
        const float rc = rho_at(x, y);
        const float r4 = __fadd_rn(__fadd_rn(rho_at(n.xm, y), rho_at(n.xp, y)), __fadd_rn(rho_at(x, n.ym), rho_at(x, n.yp)));
        rho_ave = __fadd_rn(__fmul_rn(rc, 1.f / 3.f), __fmul_rn(r4, 1.f / 6.f));
    }
    tab[(size_t)y * P.nx + x] = wall_psirho(P, x, y, rho_ave);
}

// Wettability map of a scheme-1 wall from the rest / patch parameters (phi, drho)
__global__ void k_wall_params(DevParams P, float2* par) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const bool in = wall_in_patch(P, x, y);
    par[(size_t)y * P.nx + x] = in ? make_float2(P.wet_phi_p, P.wet_drho_p) : make_float2(P.wet_phi, P.wet_drho);
}

// A user map (phi, drho as two planes of nx * ny) checked and interleaved: bad != 0 if any value
// is out of range (phi <= 0, drho < 0, non-finite), in which case nothing is written (a first
// pass only checks).
__global__ void k_wall_map(DevParams P, const float* __restrict__ phi, const float* __restrict__ drho,
                           float2* par, int* bad, int write) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const size_t i = (size_t)y * P.nx + x;
    const float a = phi[i], b = drho[i];
    if (!write) {
        if (!(a > 0.f) || !(b >= 0.f) || !isfinite(a) || !isfinite(b)) atomicOr(bad, 1);
    } else {
        par[i] = make_float2(a, b);
    }
}

cudaError_t launch_wall_params(const DevParams& P, float2* par, cudaStream_t s) {
    k_wall_params<<<dim3((P.nx + 127) / 128, P.ny), 128, 0, s>>>(P, par);
    return cudaGetLastError();
}

cudaError_t launch_wall_map(const DevParams& P, const float* phi, const float* drho, float2* par, int* bad,
                            int write, cudaStream_t s) {
    k_wall_map<<<dim3((P.nx + 127) / 128, P.ny), 128, 0, s>>>(P, phi, drho, par, bad, write);
    return cudaGetLastError();
}

cudaError_t launch_wall_table(const DevParams& P, int precision, const void* fs, int pull_f, float2* tab,
                              cudaStream_t s) {
    const dim3 grid((P.nx + 127) / 128, P.ny);
    GB300_DISPATCH(precision, (k_wall_table<S><<<grid, 128, 0, s>>>(P, (const S*)fs, pull_f, tab)));
    return cudaGetLastError();
}

cudaError_t launch_velocity(const DevParams& P, int precision, const StateBufs& B, const double* sums_cur,
                            cudaStream_t s) {
    dim3 blk(TPB_X, TPB_Y);
    GB300_DISPATCH(precision, (k_velocity<S><<<grid_of(P), blk, 0, s>>>(P, (const S*)B.src, B.pull_f, B.psirho,
                                                                         sums_cur, B.vel)));
    return cudaGetLastError();
}

cudaError_t launch_moments(const DevParams& P, int precision, const StateBufs& B, const double* sums_cur,
                           float* rho, float* ux, float* uy, float* uz, float* T, cudaStream_t s) {
    dim3 blk(TPB_X, TPB_Y);
    GB300_DISPATCH_QT(P, precision, (k_moments<S, QT><<<grid_of(P), blk, 0, s>>>(P, (const S*)B.src, B.pull_f, B.pull_g,
                                                                        B.psirho, sums_cur, rho, ux, uy, uz, T)));
    return cudaGetLastError();
}

cudaError_t launch_sum_field(const float* a, int n, double2* partial, unsigned* counter, double* out,
                             cudaStream_t s) {
    int blocks = (n + 255) / 256;
    if (blocks > SUM_BLOCKS_MAX) blocks = SUM_BLOCKS_MAX;
    if (blocks < 1) blocks = 1;
    k_sum_field<<<blocks, 256, 0, s>>>(a, n, partial, counter, out);
    return cudaGetLastError();
}

}  // namespace gb300lbm
