// Device building blocks of the GB300 lattice update: parameters, population codecs,
// boundary-aware pull, Peng-Robinson psi, D3Q19 MRT collision with the forcing of
// Eq. 9, local div u (Eq. 48) and grad T (Eq. 45), phase-change source (Eq. 18, 23) and
// the D3Q7 MRT temperature collision (Eqs. 38-43).
//
// Everything here is FP32 arithmetic; reciprocals and square roots use the hardware approximations
// (__fdividef, rsqrtf: within 2 ulp), shared by every kernel variant.  The D3Q19 transform uses the raw polynomial
// moments of Eq. 5's order (1, e, |e|^2, 2ex^2-ey^2-ez^2, ey^2-ez^2, exey, exez, eyez,
// ex^2ey, exey^2, ex^2ez, exez^2, ey^2ez, eyez^2, ex^2ey^2, ex^2ez^2, ey^2ez^2) and its
// closed-form inverse, unrolled by hand (no 19x19 matrix product).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gb300lbm {

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_OUTFLOW = 2, BC_THERMAL_ONLY = 3 };

// D3Q19 velocities in the order of Eq. 2 and D3Q7 velocities of Eq. 21.
__host__ __device__ constexpr int ex19(int a) {
    return (a == 1 || a == 7 || a == 9 || a == 11 || a == 13) ? 1
         : (a == 2 || a == 8 || a == 10 || a == 12 || a == 14) ? -1 : 0;
}
__host__ __device__ constexpr int ey19(int a) {
    return (a == 3 || a == 7 || a == 10 || a == 15 || a == 17) ? 1
         : (a == 4 || a == 8 || a == 9 || a == 16 || a == 18) ? -1 : 0;
}
__host__ __device__ constexpr int ez19(int a) {
    return (a == 5 || a == 11 || a == 14 || a == 15 || a == 18) ? 1
         : (a == 6 || a == 12 || a == 13 || a == 16 || a == 17) ? -1 : 0;
}
__host__ __device__ constexpr int opp(int a) { return a == 0 ? 0 : ((a & 1) ? a + 1 : a - 1); }
__host__ __device__ constexpr int ex7(int a) { return a == 1 ? 1 : a == 2 ? -1 : 0; }
__host__ __device__ constexpr int ey7(int a) { return a == 3 ? 1 : a == 4 ? -1 : 0; }
__host__ __device__ constexpr int ez7(int a) { return a == 5 ? 1 : a == 6 ? -1 : 0; }

// Storage slots of the populations, grouped by e_z so that one tensor copy per group fetches a
// plane: slots 0..13 have e_z = 0 (f0-4, f7-10, g0-4), 14..19 e_z = +1 (f5, f11, f14, f15, f18,
// g5), 20..25 e_z = -1 (f6, f12, f13, f16, f17, g6).
__host__ __device__ constexpr int fslot(int a) {
    return a <= 4 ? a : a == 5 ? 14 : a == 6 ? 20 : a <= 10 ? a - 2 : a == 11 ? 15 : a == 12 ? 21
         : a == 13 ? 22 : a == 14 ? 16 : a == 15 ? 17 : a == 16 ? 23 : a == 17 ? 24 : 18;
}
__host__ __device__ constexpr int gslot(int a) { return a <= 4 ? 9 + a : a == 5 ? 19 : 25; }
constexpr int kSlots = 26;
// Temperature LB on the D3Q19 lattice (thermal_q 19): g_0..g_6 share the D3Q7 velocities and slots,
// g_7..g_18 take 12 more slots after them.
__host__ __device__ constexpr int gslot19(int a) { return a <= 6 ? gslot(a) : kSlots + (a - 7); }
__host__ __device__ constexpr int slots_of(int qt) { return qt == 19 ? kSlots + 12 : kSlots; }
constexpr int kGX = 8, kGY = 2;   // storage offsets: 8 columns (2 ghosts; rows stay 32-byte aligned), 2 rows

// Lattice constants and model parameters, converted once on the host.
struct DevParams {
    int nx, ny, nz;
    int N;                    // nx*ny*nz (< 2^31): dense fields (phi_s history, psi, user fields)
    int plane;                // nx*ny
    // population storage, rows of slots: node (x, y, z) at i = (x + kGX) + Rs (y + kGY) + splane z,
    // slot s at i + s Ns with Ns = Ws, so the slots of one row follow each other (Rs = slots x Ws,
    // splane = Rs Hs).  Ws: padded row width, Hs: padded rows; Nidx bounds the node index i.
    // Columns x = -2, -1, nx, nx+1 and rows y = -2, -1, ny, ny+1 are ghost copies of the periodic
    // images (kept current by every kernel that writes populations, only on f-periodic axes).
    int Ws, Hs, Rs, splane, Ns, Nidx;
    int bc[6];
    float T_wall[6];
    float hot_dT, hot_inv2s2, hot_cx, hot_cy;
    float a, b, R, Tc, kappa; // PR EOS (Eq. 49), kappa = 0.37464 + 1.54226 w - 0.26992 w^2
    float inv_Tc;
    double inv_N;             // 1 / (nx ny nz) for the domain mean of rho
    float sigma6;             // 6 sigma / (tau_e - 0.5)   (Eq. 9, S_4)
    float Le, Lv, Lq, Lpi;    // 1/tau of Eq. 6
    float inv_tau_e, half_Le; // 1/tau_e, (1 - 1/(2 tau_e)) of Eq. 48
    float cV, d, csT2, w0, w1;
    float inv_cV, inv_csT2, R_over_cV;
    float Gq, Gpi;            // 1/varsigma_q, 1/varsigma_pi (Eq. 43)
    int lambda_mode;
    float chi_or_lambda;
    float gx, gy, gz;
    float rho_buoy;           // > 0: fixed reference density of the buoyancy force, else rho_ave
    int flow_off, thermal_off;
    int test_stall;           // timeout-path test: the TMA producer waits on a barrier nothing completes
    int thermal_bgk;          // 1: BGK D3Q7 collision (n4..n6 relaxed at 1/varsigma_T too)
    int divu_mode;            // 1: finite-difference div u away from solid faces (two-pass kernels)
    int wet;                  // 1: virtual-density solid layer below the -z wall (wetting)
    float wet_rho, wet_rho_patch, wet_half, wet_cx, wet_cy;
    int wet_scheme;           // 0: fixed virtual densities; 1: phi rho_ave - drho from the fluid layer
    float wet_phi, wet_drho, wet_phi_p, wet_drho_p;
    const float2* wall_par;   // scheme 1: (phi, drho) per (x, y), nx * ny, x fastest
    const float2* wall_tab;   // (psi, rho) of that layer per (x, y), nx * ny, x fastest (wet only)
    float shift_f[19];        // storage shift w_a rho_ref (16-bit storage only, else 0)
    float shift_g[7];         // storage shift w_a T_ref
    int* check_flag;          // the context's flag word (bounds-checked builds record violations here)
    int qt;                   // temperature lattice: 7 (D3Q7 MRT) or 19 (Eq. 19 BGK on D3Q19)
};

// Debug builds (-DLBM_BOUNDS_CHECK): every population and field index of the update, and the
// shared-memory offsets of the fused kernels, is checked before use.  An index outside its buffer
// raises bit 4 of the context's flag word and the access goes to element 0 instead, so nothing
// out of range is ever touched; lbm_step then reports LBM_EBOUNDS.  Release builds compile the
// checks away.
__device__ __forceinline__ long long bidx(const DevParams& P, long long i, long long n) {
#ifdef LBM_BOUNDS_CHECK
    if (i < 0 || i >= n) {
        atomicOr(P.check_flag, 4);
        return 0;
    }
#endif
    return i;
}
// the same for a thread's base offset v that later accesses reach as v + [lo, hi]
__device__ __forceinline__ int bbase(const DevParams& P, int v, int lo, int hi, int n) {
#ifdef LBM_BOUNDS_CHECK
    if (v + lo < 0 || v + hi >= n) {
        atomicOr(P.check_flag, 4);
        return -lo;
    }
#endif
    return v;
}

// reference density of the buoyancy force F_b = (rho - rho_b) g: fixed, or the domain mean of the
// previous step (Sec. IV.C) from its FP64 sum
__device__ __forceinline__ float buoyancy_ref(const DevParams& P, double rho_sum, double inv_N) {
    return P.rho_buoy > 0.f ? P.rho_buoy : (float)(rho_sum * inv_N);
}

// ---------------------------------------------------------------- population storage
// Populations are stored structure-of-arrays: pop[a * N + node].
template <typename S> struct Codec;
template <> struct Codec<float> {
    static __device__ __forceinline__ float load(const float* p, float) { return __ldg(p); }
    static __device__ __forceinline__ void store(float* p, float v, float) { *p = v; }
};
template <> struct Codec<__nv_bfloat16> {
    static __device__ __forceinline__ float load(const __nv_bfloat16* p, float s) {
        return __bfloat162float(__ldg(p)) + s;
    }
    static __device__ __forceinline__ void store(__nv_bfloat16* p, float v, float s) {
        *p = __float2bfloat16_rn(v - s);
    }
};
template <> struct Codec<__half> {
    static __device__ __forceinline__ float load(const __half* p, float s) {
        return __half2float(__ldg(p)) + s;
    }
    static __device__ __forceinline__ void store(__half* p, float v, float s) {
        *p = __float2half_rn(v - s);
    }
};

// ---------------------------------------------------------------- neighbourhood of a node
// For each axis: coordinate of the node at -1 / +1 after periodic wrap, or clamped onto the
// node itself at a non-periodic face (that clamp is both the outflow extrapolation source
// of the f pull and the mirror image of the psi / grad-rho stencil).  Bit masks mark
// faces crossed by a pull: fbb (f halfway bounce-back, Eq. 50) and gabb (g anti-bounce-back,
// Eq. 51).  Bit 2k   : the -1 neighbour along axis k lies behind face 2k.
//          Bit 2k+1 : the +1 neighbour along axis k lies behind face 2k+1.
struct Nbr {
    int xm, xp, ym, yp, zm, zp;   // coordinates
    unsigned fbb, gabb;
};

__host__ __device__ inline bool f_wraps(int bc) { return bc == BC_PERIODIC || bc == BC_THERMAL_ONLY; }

__device__ __forceinline__ void axis_nbr(int c, int n, int bc_lo, int bc_hi, int bit,
                                         int& cm, int& cp, unsigned& fbb, unsigned& gabb) {
    cm = c - 1;
    cp = c + 1;
    if (c == 0) {
        cm = f_wraps(bc_lo) ? n - 1 : 0;
        if (bc_lo == BC_WALL) fbb |= 1u << bit;
        if (bc_lo != BC_PERIODIC) gabb |= 1u << bit;
    }
    if (c == n - 1) {
        cp = f_wraps(bc_hi) ? 0 : n - 1;
        if (bc_hi == BC_WALL) fbb |= 2u << bit;
        if (bc_hi != BC_PERIODIC) gabb |= 2u << bit;
    }
}

__device__ __forceinline__ Nbr make_nbr(const DevParams& P, int x, int y, int z) {
    Nbr n;
    n.fbb = 0;
    n.gabb = 0;
    axis_nbr(x, P.nx, P.bc[0], P.bc[1], 0, n.xm, n.xp, n.fbb, n.gabb);
    axis_nbr(y, P.ny, P.bc[2], P.bc[3], 2, n.ym, n.yp, n.fbb, n.gabb);
    axis_nbr(z, P.nz, P.bc[4], P.bc[5], 4, n.zm, n.zp, n.fbb, n.gabb);
    return n;
}

// dense node index (fields) and storage index (populations)
__device__ __forceinline__ int node_of(const DevParams& P, int x, int y, int z) {
    return x + P.nx * (y + P.ny * z);
}
__device__ __forceinline__ int sidx(const DevParams& P, int x, int y, int z) {
    return (x + kGX) + P.Rs * (y + kGY) + P.splane * z;
}

// Source coordinate of the pull along one axis for velocity component e (x - e).
__device__ __forceinline__ int src_c(int e, int c, int cm, int cp) { return e > 0 ? cm : (e < 0 ? cp : c); }
// Neighbour coordinate of the stencil along one axis (x + e).
__device__ __forceinline__ int nb_c(int e, int c, int cm, int cp) { return e > 0 ? cp : (e < 0 ? cm : c); }

// Does the pull of velocity a cross a wall face (Eq. 50)?
template <int A> __device__ __forceinline__ bool crosses(unsigned mask) {
    constexpr int ex = ex19(A), ey = ey19(A), ez = ez19(A);
    constexpr unsigned m = (ex > 0 ? 1u : 0u) | (ex < 0 ? 2u : 0u) | (ey > 0 ? 4u : 0u) |
                           (ey < 0 ? 8u : 0u) | (ez > 0 ? 16u : 0u) | (ez < 0 ? 32u : 0u);
    return (mask & m) != 0u;
}

__device__ __forceinline__ float wall_T(const DevParams& P, int face, int x, int y) {
    float T = P.T_wall[face];
    if (face == 4 && P.hot_dT != 0.f) {
        float dx = (float)x - P.hot_cx, dy = (float)y - P.hot_cy;
        T += P.hot_dT * expf(-__fmaf_rn(dy, dy, __fmul_rn(dx, dx)) * P.hot_inv2s2);
    }
    return T;
}

template <typename S, int A>
__device__ __forceinline__ float pull_f_one(const DevParams& P, const S* __restrict__ src, int i,
                                            int x, int y, int z, const Nbr& n) {
    constexpr int ex = ex19(A), ey = ey19(A), ez = ez19(A);
    if (A != 0 && crosses<A>(n.fbb))   // Eq. 50: f_a(x_b, t+1) = f*_{abar}(x_b, t)
        return Codec<S>::load(src + (size_t)fslot(opp(A)) * P.Ns + bidx(P, i, P.Nidx), P.shift_f[opp(A)]);
    int s = sidx(P, src_c(ex, x, n.xm, n.xp), src_c(ey, y, n.ym, n.yp), src_c(ez, z, n.zm, n.zp));
    return Codec<S>::load(src + (size_t)fslot(A) * P.Ns + bidx(P, s, P.Nidx), P.shift_f[A]);
}

// Node at least one node away from every face: every pull source is i - (ex + nx ey + nx ny ez).
__device__ __forceinline__ bool deep_interior(const DevParams& P, int x, int y, int z) {
    return (unsigned)(x - 1) < (unsigned)(P.nx - 2) && (unsigned)(y - 1) < (unsigned)(P.ny - 2) &&
           (unsigned)(z - 1) < (unsigned)(P.nz - 2);
}

template <typename S, int A>
__device__ __forceinline__ float pull_f_fast(const DevParams& P, const S* __restrict__ src, int i) {
    constexpr int ex = ex19(A), ey = ey19(A), ez = ez19(A);
    return Codec<S>::load(src + (size_t)fslot(A) * P.Ns + bidx(P, i - ex - ey * P.Rs - ez * P.splane, P.Nidx),
                          P.shift_f[A]);
}

// Pull of all 19 f (pull != 0) or direct read of the node's own values (fresh state).
template <typename S>
__device__ __forceinline__ void load_f(const DevParams& P, const S* __restrict__ src, int pull, int i,
                                       int x, int y, int z, const Nbr& n, float f[19]) {
    if (pull && deep_interior(P, x, y, z)) {
#define GB300_PULL(A) f[A] = pull_f_fast<S, A>(P, src, i);
        GB300_PULL(0) GB300_PULL(1) GB300_PULL(2) GB300_PULL(3) GB300_PULL(4) GB300_PULL(5)
        GB300_PULL(6) GB300_PULL(7) GB300_PULL(8) GB300_PULL(9) GB300_PULL(10) GB300_PULL(11)
        GB300_PULL(12) GB300_PULL(13) GB300_PULL(14) GB300_PULL(15) GB300_PULL(16) GB300_PULL(17)
        GB300_PULL(18)
#undef GB300_PULL
    } else if (pull) {
#define GB300_PULL(A) f[A] = pull_f_one<S, A>(P, src, i, x, y, z, n);
        GB300_PULL(0) GB300_PULL(1) GB300_PULL(2) GB300_PULL(3) GB300_PULL(4) GB300_PULL(5)
        GB300_PULL(6) GB300_PULL(7) GB300_PULL(8) GB300_PULL(9) GB300_PULL(10) GB300_PULL(11)
        GB300_PULL(12) GB300_PULL(13) GB300_PULL(14) GB300_PULL(15) GB300_PULL(16) GB300_PULL(17)
        GB300_PULL(18)
#undef GB300_PULL
    } else {
#pragma unroll
        for (int a = 0; a < 19; ++a) f[a] = Codec<S>::load(src + (size_t)fslot(a) * P.Ns + bidx(P, i, P.Nidx), P.shift_f[a]);
    }
}

template <typename S, int A>
__device__ __forceinline__ float pull_g_one(const DevParams& P, const S* __restrict__ src, int i,
                                            int x, int y, int z, const Nbr& n) {
    constexpr int ex = ex7(A), ey = ey7(A), ez = ez7(A);
    constexpr int face = ex > 0 ? 0 : ex < 0 ? 1 : ey > 0 ? 2 : ey < 0 ? 3 : ez > 0 ? 4 : 5;
    if (A != 0 && (n.gabb & (1u << face))) {
        // Eq. 51: g_a(x_b, t+1) = -g+_{abar}(x_b, t) + 2 w_abar T_w   (w_abar = w_a on D3Q7)
        float gp = Codec<S>::load(src + (size_t)gslot(opp(A)) * P.Ns + bidx(P, i, P.Nidx), P.shift_g[opp(A)]);
        return -gp + 2.f * P.w1 * wall_T(P, face, x, y);
    }
    int s = sidx(P, src_c(ex, x, n.xm, n.xp), src_c(ey, y, n.ym, n.yp), src_c(ez, z, n.zm, n.zp));
    return Codec<S>::load(src + (size_t)gslot(A) * P.Ns + bidx(P, s, P.Nidx), P.shift_g[A]);
}

template <typename S>
__device__ __forceinline__ void load_g(const DevParams& P, const S* __restrict__ src, int pull, int i,
                                       int x, int y, int z, const Nbr& n, float g[7]) {
    if (pull && deep_interior(P, x, y, z)) {
        g[0] = Codec<S>::load(src + (size_t)gslot(0) * P.Ns + bidx(P, i, P.Nidx), P.shift_g[0]);
        g[1] = Codec<S>::load(src + (size_t)gslot(1) * P.Ns + bidx(P, i - 1, P.Nidx), P.shift_g[1]);
        g[2] = Codec<S>::load(src + (size_t)gslot(2) * P.Ns + bidx(P, i + 1, P.Nidx), P.shift_g[2]);
        g[3] = Codec<S>::load(src + (size_t)gslot(3) * P.Ns + bidx(P, i - P.Rs, P.Nidx), P.shift_g[3]);
        g[4] = Codec<S>::load(src + (size_t)gslot(4) * P.Ns + bidx(P, i + P.Rs, P.Nidx), P.shift_g[4]);
        g[5] = Codec<S>::load(src + (size_t)gslot(5) * P.Ns + bidx(P, i - P.splane, P.Nidx), P.shift_g[5]);
        g[6] = Codec<S>::load(src + (size_t)gslot(6) * P.Ns + bidx(P, i + P.splane, P.Nidx), P.shift_g[6]);
    } else if (pull) {
        g[0] = pull_g_one<S, 0>(P, src, i, x, y, z, n);
        g[1] = pull_g_one<S, 1>(P, src, i, x, y, z, n);
        g[2] = pull_g_one<S, 2>(P, src, i, x, y, z, n);
        g[3] = pull_g_one<S, 3>(P, src, i, x, y, z, n);
        g[4] = pull_g_one<S, 4>(P, src, i, x, y, z, n);
        g[5] = pull_g_one<S, 5>(P, src, i, x, y, z, n);
        g[6] = pull_g_one<S, 6>(P, src, i, x, y, z, n);
    } else {
#pragma unroll
        for (int a = 0; a < 7; ++a) g[a] = Codec<S>::load(src + (size_t)gslot(a) * P.Ns + bidx(P, i, P.Nidx), P.shift_g[a]);
    }
}

// Store the 26 post-collision populations at storage index i, walking the slots in order.
template <typename S>
__device__ __forceinline__ void store_slots(const DevParams& P, S* __restrict__ dst, int i, const float f[19],
                                            const float g[7]) {
    S* q = dst + bidx(P, i, P.Nidx);
#define GB300_ST(V, SH) { Codec<S>::store(q, V, SH); q += P.Ns; }
    GB300_ST(f[0], P.shift_f[0]) GB300_ST(f[1], P.shift_f[1]) GB300_ST(f[2], P.shift_f[2])
    GB300_ST(f[3], P.shift_f[3]) GB300_ST(f[4], P.shift_f[4]) GB300_ST(f[7], P.shift_f[7])
    GB300_ST(f[8], P.shift_f[8]) GB300_ST(f[9], P.shift_f[9]) GB300_ST(f[10], P.shift_f[10])
    GB300_ST(g[0], P.shift_g[0]) GB300_ST(g[1], P.shift_g[1]) GB300_ST(g[2], P.shift_g[2])
    GB300_ST(g[3], P.shift_g[3]) GB300_ST(g[4], P.shift_g[4])
    GB300_ST(f[5], P.shift_f[5]) GB300_ST(f[11], P.shift_f[11]) GB300_ST(f[14], P.shift_f[14])
    GB300_ST(f[15], P.shift_f[15]) GB300_ST(f[18], P.shift_f[18]) GB300_ST(g[5], P.shift_g[5])
    GB300_ST(f[6], P.shift_f[6]) GB300_ST(f[12], P.shift_f[12]) GB300_ST(f[13], P.shift_f[13])
    GB300_ST(f[16], P.shift_f[16]) GB300_ST(f[17], P.shift_f[17]) Codec<S>::store(q, g[6], P.shift_g[6]);
#undef GB300_ST
}

// Store the 26 post-collision populations of node (x, y, z) at storage index i.  Ghost cells are
// not touched here: the TMA path refreshes them with a separate kernel after every step.
template <typename S>
__device__ __forceinline__ void store_node(const DevParams& P, S* __restrict__ dst, int i, int, int, int,
                                           const float f[19], const float g[7]) {
    store_slots<S>(P, dst, i, f, g);
}

// rho = sum f and T = sum g in one fixed pairwise order (every kernel uses these, so all variants
// agree bit for bit; the tree also shortens the dependency chain)
__device__ __forceinline__ float sum19(const float f[19]) {
    float a = (f[1] + f[2]) + (f[3] + f[4]), b = (f[5] + f[6]) + (f[7] + f[8]);
    float c = (f[9] + f[10]) + (f[11] + f[12]), d = (f[13] + f[14]) + (f[15] + f[16]);
    float e = (f[17] + f[18]) + f[0];
    return ((a + b) + (c + d)) + e;
}
__device__ __forceinline__ float sum7(const float g[7]) {
    return ((g[1] + g[2]) + (g[3] + g[4])) + ((g[5] + g[6]) + g[0]);
}

// ---------------------------------------------------------------- thermodynamics
// Rounding.  Where two or more products are summed, the sum is written with explicit
// __fmaf_rn / __fmul_rn: left as plain arithmetic, the compiler may fuse either product into the
// add and chooses differently in different kernels, so kernels that share these functions would
// no longer round alike (a sum with one product has one fusion and is left to the compiler).
//
// Peng-Robinson pressure (Eq. 49) and psi^2 = 2 (p_EOS - rho cs^2) / (G c^2) with G = -1 (Eq. 8).
__device__ __forceinline__ float psi_of(float psi2) { return psi2 * rsqrtf(psi2); }   // sqrt; NaN if <= 0
__device__ __forceinline__ float psi_squared(const DevParams& P, float rho, float T) {
    const float tr = T * P.inv_Tc;
    float s = 1.f + P.kappa * (1.f - tr * rsqrtf(tr));   // sqrt(T / Tc)
    float theta = s * s;
    float brho = P.b * rho;
    float d1 = 1.f - brho, d2 = 1.f + 2.f * brho - brho * brho;
    float inv = __fdividef(1.f, d1 * d2);   // one reciprocal for both denominators
    float p = __fmaf_rn(-(P.a * theta * rho * rho), d1 * inv, __fmul_rn(rho * P.R * T, d2 * inv));
    return 2.f * (rho * (1.f / 3.f) - p);
}

// Is (x, y) of the -z wall inside the square patch |x - nx/2| < h, |y - ny/2| < h?
__device__ __forceinline__ bool wall_in_patch(const DevParams& P, int x, int y) {
    const float dx = (float)x - P.wet_cx, dy = (float)y - P.wet_cy;
    return fabsf(dx) < P.wet_half && fabsf(dy) < P.wet_half;
}

// (psi, rho) of the solid node below (x, y) of the -z wall when it carries a virtual density
// (wetting), psi from Eqs. 8, 49 at the wall temperature T_w(x, y).  Scheme 0: rho_w outside the
// square patch, the patch value inside.  Scheme 1: phi rho_ave - drho with the node's (phi, drho)
// from the wettability map P.wall_par, floored at rho_ave / 10; rho_ave is the weighted mean
// density of the node's five fluid neighbours.  k_wall_table evaluates it into P.wall_tab (once
// per context for scheme 0, at the start of every step for scheme 1), which the stencils read
// (wall_entry).
__device__ __forceinline__ float2 wall_psirho(const DevParams& P, int x, int y, float rho_ave) {
    float rw;
    if (P.wet_scheme == 1) {
        const float2 pd = P.wall_par[(size_t)y * P.nx + x];
        rw = fmaxf(__fsub_rn(__fmul_rn(pd.x, rho_ave), pd.y), __fmul_rn(0.1f, rho_ave));
    } else {
        rw = wall_in_patch(P, x, y) ? P.wet_rho_patch : P.wet_rho;
    }
    return make_float2(psi_of(psi_squared(P, rw, wall_T(P, 4, x, y))), rw);
}

__device__ __forceinline__ float2 wall_entry(const DevParams& P, int x, int y) {
    return __ldg(P.wall_tab + bidx(P, (long long)y * P.nx + x, (long long)P.nx * P.ny));
}

// f = M^-1 m from the pair sums / differences of the raw moments: a* = f_+ + f_-, b* = f_+ - f_-
// of the three axis pairs, and the 12 edge populations from m7..m18.  f_0 = rho - sum f_1..18.
__device__ __forceinline__ void back_transform(float rho, float ax, float bx, float ay, float by, float az,
                                               float bz, float m7, float m8, float m9, float m10, float m11,
                                               float m12, float m13, float m14, float m15, float m16,
                                               float m17, float m18, float f[19]) {
    f[1] = 0.5f * (ax + bx); f[2] = 0.5f * (ax - bx);
    f[3] = 0.5f * (ay + by); f[4] = 0.5f * (ay - by);
    f[5] = 0.5f * (az + bz); f[6] = 0.5f * (az - bz);
    f[7] = 0.25f * (m16 + m7 + m10 + m11);
    f[8] = 0.25f * (m16 + m7 - m10 - m11);
    f[9] = 0.25f * (m16 - m7 - m10 + m11);
    f[10] = 0.25f * (m16 - m7 + m10 - m11);
    f[11] = 0.25f * (m17 + m8 + m12 + m13);
    f[12] = 0.25f * (m17 + m8 - m12 - m13);
    f[13] = 0.25f * (m17 - m8 - m12 + m13);
    f[14] = 0.25f * (m17 - m8 + m12 - m13);
    f[15] = 0.25f * (m18 + m9 + m14 + m15);
    f[16] = 0.25f * (m18 + m9 - m14 - m15);
    f[17] = 0.25f * (m18 - m9 - m14 + m15);
    f[18] = 0.25f * (m18 - m9 + m14 - m15);
    float s = ((f[1] + f[2]) + (f[3] + f[4]) + (f[5] + f[6])) +
              (((f[7] + f[8]) + (f[9] + f[10])) + ((f[11] + f[12]) + (f[13] + f[14])) +
               ((f[15] + f[16]) + (f[17] + f[18])));
    f[0] = rho - s;
}

// ---------------------------------------------------------------- D3Q19 MRT collision
// One moment of Eq. 3: m* = m - L (m - m_eq) + (1 - L/2) S = m + (-L (m - m_eq) + h S), with every
// rounding step explicit.  Written as plain arithmetic the sum of two products leaves the compiler
// free to fuse either product into the add, and it chose differently in different kernels.
__device__ __forceinline__ float relax(float m, float eq, float S, float L, float h) {
    return __fadd_rn(m, __fmaf_rn(-L, __fsub_rn(m, eq), __fmul_rn(h, S)));
}

struct NodeOut {
    float ux, uy, uz, divu, inv_rho;
};

// Interaction force F_m = -G psi sum_a w_a psi(x + e_a) e_a (Eq. 7, G = -1) from the stencil sums
// (sx, sy, sz), |F_m|^2, and the total force F = F_m + (rho - rho_ave) g (buoyancy).
struct Forces {
    float Fx, Fy, Fz, Fm2;
};
__device__ __forceinline__ Forces total_force(const DevParams& P, float psi, float sx, float sy, float sz, float db) {
    const float mx = __fmul_rn(psi, sx), my = __fmul_rn(psi, sy), mz = __fmul_rn(psi, sz);
    Forces F;
    F.Fm2 = __fmaf_rn(mz, mz, __fmaf_rn(my, my, __fmul_rn(mx, mx)));
    F.Fx = __fmaf_rn(db, P.gx, mx);
    F.Fy = __fmaf_rn(db, P.gy, my);
    F.Fz = __fmaf_rn(db, P.gz, mz);
    return F;
}

// In: post-streaming f with rho = sum19(f), total force F, interaction force Fm, psi^2.
// Out: f* in place.
// Eq. 10 velocity, Eq. 5 equilibrium moments, Eq. 9 forcing, Eq. 6 rates, Eq. 3 relaxation,
// Eq. 4 back-transform, Eq. 48 divergence.
__device__ __forceinline__ NodeOut collide_f(const DevParams& P, float f[19], float rho, float Fx, float Fy,
                                             float Fz, float Fm2, float psi2) {
    const float cs2 = 1.f / 3.f;
    float jx = (f[1] - f[2]) + (f[7] - f[8]) + (f[9] - f[10]) + (f[11] - f[12]) + (f[13] - f[14]);
    float jy = (f[3] - f[4]) + (f[7] - f[8]) - (f[9] - f[10]) + (f[15] - f[16]) + (f[17] - f[18]);
    float jz = (f[5] - f[6]) + (f[11] - f[12]) - (f[13] - f[14]) + (f[15] - f[16]) - (f[17] - f[18]);
    float inv_rho = __fdividef(1.f, rho);
    float ux = (jx + 0.5f * Fx) * inv_rho, uy = (jy + 0.5f * Fy) * inv_rho, uz = (jz + 0.5f * Fz) * inv_rho;

    // raw moments (rows of M)
    float s7 = f[7] + f[8], s9 = f[9] + f[10], s11 = f[11] + f[12], s13 = f[13] + f[14];
    float s15 = f[15] + f[16], s17 = f[17] + f[18];
    float m16 = s7 + s9, m17 = s11 + s13, m18 = s15 + s17;
    float xx = f[1] + f[2] + m16 + m17;
    float yy = f[3] + f[4] + m16 + m18;
    float zz = f[5] + f[6] + m17 + m18;
    float m4 = xx + yy + zz;
    float m5 = 2.f * xx - yy - zz;
    float m6 = yy - zz;
    float m7 = s7 - s9, m8 = s11 - s13, m9 = s15 - s17;
    float d7 = f[7] - f[8], d9 = f[9] - f[10], d11 = f[11] - f[12], d13 = f[13] - f[14];
    float d15 = f[15] - f[16], d17 = f[17] - f[18];
    float m10 = d7 - d9, m11 = d7 + d9, m12 = d11 - d13, m13 = d11 + d13, m14 = d15 - d17, m15 = d15 + d17;

    // equilibrium moments (Eq. 5)
    float ux2 = __fmul_rn(ux, ux), uy2 = __fmul_rn(uy, uy), uz2 = __fmul_rn(uz, uz), u2 = ux2 + uy2 + uz2;
    float phi = __fmul_rn(rho * (cs2 * cs2), 1.f - 1.5f * u2);
    float e4 = rho + rho * u2;
    float e5 = rho * (2.f * ux2 - uy2 - uz2), e6 = rho * (uy2 - uz2);
    float e7 = rho * ux * uy, e8 = rho * ux * uz, e9 = rho * uy * uz;
    float e10 = rho * uy * (cs2 + ux2), e11 = rho * ux * (cs2 + uy2);
    float e12 = rho * uz * (cs2 + ux2), e13 = rho * ux * (cs2 + uz2);
    float e14 = rho * uz * (cs2 + uy2), e15 = rho * uy * (cs2 + uz2);
    float e16 = phi + rho * cs2 * (ux2 + uy2), e17 = phi + rho * cs2 * (ux2 + uz2);
    float e18 = phi + rho * cs2 * (uy2 + uz2);

    // forcing moments (Eq. 9)
    float Fu_x = __fmul_rn(Fx, ux), Fu_y = __fmul_rn(Fy, uy), Fu_z = __fmul_rn(Fz, uz);
    float S4 = __fmaf_rn(P.sigma6, __fdividef(Fm2, psi2), 2.f * (Fu_x + Fu_y + Fu_z));
    float S5 = 2.f * (2.f * Fu_x - Fu_y - Fu_z), S6 = 2.f * (Fu_y - Fu_z);
    float S7 = __fmaf_rn(Fy, ux, __fmul_rn(Fx, uy)), S8 = __fmaf_rn(Fz, ux, __fmul_rn(Fx, uz));
    float S9 = __fmaf_rn(Fz, uy, __fmul_rn(Fy, uz));
    float S10 = cs2 * Fy, S11 = cs2 * Fx, S12 = cs2 * Fz, S13 = cs2 * Fx, S14 = cs2 * Fz, S15 = cs2 * Fy;
    float S16 = 2.f * cs2 * (Fu_x + Fu_y), S17 = 2.f * cs2 * (Fu_x + Fu_z), S18 = 2.f * cs2 * (Fu_y + Fu_z);

    NodeOut o;
    o.ux = ux; o.uy = uy; o.uz = uz;
    o.inv_rho = inv_rho;
    // Eq. 48 (pre-collision m_4, force-corrected u, full S_4, total F)
    o.divu = (__fmaf_rn(P.half_Le, S4, __fmul_rn(-(m4 - e4), P.inv_tau_e)) - 2.f * (Fu_x + Fu_y + Fu_z)) *
             (1.5f * inv_rho);

    // relaxation (Eq. 3): m* = m - L (m - meq) + (1 - L/2) S
    const float Le = P.Le, Lv = P.Lv, Lq = P.Lq, Lp = P.Lpi;
    float r1 = jx + Fx, r2 = jy + Fy, r3 = jz + Fz;   // rates 1: m* = rho u + F/2 = j + F
    const float he = 1.f - 0.5f * Le, hv = 1.f - 0.5f * Lv, hq = 1.f - 0.5f * Lq, hp = 1.f - 0.5f * Lp;
    m4 = relax(m4, e4, S4, Le, he);
    m5 = relax(m5, e5, S5, Lv, hv);
    m6 = relax(m6, e6, S6, Lv, hv);
    m7 = relax(m7, e7, S7, Lv, hv);
    m8 = relax(m8, e8, S8, Lv, hv);
    m9 = relax(m9, e9, S9, Lv, hv);
    m10 = relax(m10, e10, S10, Lq, hq);
    m11 = relax(m11, e11, S11, Lq, hq);
    m12 = relax(m12, e12, S12, Lq, hq);
    m13 = relax(m13, e13, S13, Lq, hq);
    m14 = relax(m14, e14, S14, Lq, hq);
    m15 = relax(m15, e15, S15, Lq, hq);
    m16 = relax(m16, e16, S16, Lp, hp);
    m17 = relax(m17, e17, S17, Lp, hp);
    m18 = relax(m18, e18, S18, Lp, hp);

    // back-transform f* = M^-1 m* (closed form of the raw-moment inverse).  The rest population
    // is formed last as rho - sum of the others, so that FP32 rounding (e.g. of the 1/3 factor)
    // cannot drift the mass: m_0* = rho exactly as Eq. 3 demands.
    float X = __fmul_rn(m4 + m5, 1.f / 3.f);
    float Y = 0.5f * (m4 - X + m6);
    float Z = 0.5f * (m4 - X - m6);
    float ax = X - m16 - m17, bx = r1 - m11 - m13;
    float ay = Y - m16 - m18, by = r2 - m10 - m15;
    float az = Z - m17 - m18, bz = r3 - m12 - m14;
    back_transform(rho, ax, bx, ay, by, az, bz, m7, m8, m9, m10, m11, m12, m13, m14, m15, m16, m17, m18, f);
    return o;
}

// Equilibrium populations f = M^-1 m_eq(rho, u) (Eq. 5) for the initial state.
__device__ __forceinline__ void feq(float rho, float ux, float uy, float uz, float f[19]) {
    const float cs2 = 1.f / 3.f;
    float ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz, u2 = ux2 + uy2 + uz2;
    float phi = rho * (cs2 * cs2) * (1.f - 1.5f * u2);
    float m4 = rho + rho * u2, m5 = rho * (2.f * ux2 - uy2 - uz2), m6 = rho * (uy2 - uz2);
    float m7 = rho * ux * uy, m8 = rho * ux * uz, m9 = rho * uy * uz;
    float m10 = rho * uy * (cs2 + ux2), m11 = rho * ux * (cs2 + uy2);
    float m12 = rho * uz * (cs2 + ux2), m13 = rho * ux * (cs2 + uz2);
    float m14 = rho * uz * (cs2 + uy2), m15 = rho * uy * (cs2 + uz2);
    float m16 = phi + rho * cs2 * (ux2 + uy2), m17 = phi + rho * cs2 * (ux2 + uz2);
    float m18 = phi + rho * cs2 * (uy2 + uz2);
    float X = (m4 + m5) * (1.f / 3.f);
    float Y = 0.5f * (m4 - X + m6);
    float Z = 0.5f * (m4 - X - m6);
    float ax = X - m16 - m17, bx = rho * ux - m11 - m13;
    float ay = Y - m16 - m18, by = rho * uy - m10 - m15;
    float az = Z - m17 - m18, bz = rho * uz - m12 - m14;
    back_transform(rho, ax, bx, ay, by, az, bz, m7, m8, m9, m10, m11, m12, m13, m14, m15, m16, m17, m18, f);
}

// ---------------------------------------------------------------- D3Q7 MRT temperature LB
// n = N g (Eq. 38); grad T from the first moments (Eq. 45); phi_s (Eq. 18); Q (Eqs. 23-24);
// n* = n - Gamma (n - n_eq) with n_eq = (T, 0, 0, 0, 3 cs_T^2 T, 0, 0) (Eqs. 39, 42, 43);
// g+ = N^-1 n* + Q (Eqs. 40-41).  g is replaced by g+ in place; returns phi_s.
__device__ __forceinline__ float collide_g(const DevParams& P, float g[7], float rho, float T,
                                           const NodeOut& o, float grx, float gry, float grz,
                                           float phis_prev, int first) {
    float n1 = g[1] - g[2], n2 = g[3] - g[4], n3 = g[5] - g[6];
    float n4 = g[1] + g[2] + g[3] + g[4] + g[5] + g[6];
    float n5 = g[1] + g[2] - g[3] - g[4];
    float n6 = g[1] + g[2] - g[5] - g[6];
    const float inv_rho = o.inv_rho;
    float chi = P.lambda_mode ? P.chi_or_lambda * inv_rho * P.inv_cV : P.chi_or_lambda;
    float vsT = chi * P.inv_csT2 + 0.5f;             // chi = (varsigma_T - 1/2) cs_T^2
    float inv_vsT = __fdividef(1.f, vsT);
    float k = -inv_vsT * P.inv_csT2;                 // Eq. 45
    float gTx = k * n1, gTy = k * n2, gTz = k * n3;
    float phis;
    if (!P.flow_off) {
        phis = __fmaf_rn(chi * grz * inv_rho - o.uz, gTz,
                         __fmaf_rn(chi * gry * inv_rho - o.uy, gTy, __fmul_rn(chi * grx * inv_rho - o.ux, gTx)));
        // T/(rho cV) (dp/dT)_rho div u with (dp/dT)_rho ~ rho R / (1 - b rho)
        phis -= __fdividef(T * P.R_over_cV, 1.f - P.b * rho) * o.divu;
    } else {
        // frozen flow: a static fluid (u = 0, div u = 0); the conduction term of Eq. 18 remains
        phis = __fmaf_rn(chi * grz * inv_rho, gTz, __fmaf_rn(chi * gry * inv_rho, gTy, __fmul_rn(chi * grx * inv_rho, gTx)));
    }
    float C = first ? phis : phis_prev;
    float qs = __fmaf_rn(-0.5f, C, __fmul_rn(1.5f, phis));   // Q_a = w_a (3/2 phi_s(t) - 1/2 phi_s(t-1))
    float om = 1.f - inv_vsT;
    n1 = __fmul_rn(n1, om); n2 = __fmul_rn(n2, om); n3 = __fmul_rn(n3, om);
    // n4* = n4 - Gq (n4 - d T) with 3 cs_T^2 T = d T; explicit rounding as in relax().  The BGK
    // variant relaxes n4..n6 at the rate of n1..n3, 1/varsigma_T.
    const float Gq = P.thermal_bgk ? inv_vsT : P.Gq, Gpi = P.thermal_bgk ? inv_vsT : P.Gpi;
    n4 = __fsub_rn(n4, __fmul_rn(Gq, __fsub_rn(n4, __fmul_rn(P.d, T))));
    n5 = __fmul_rn(n5, 1.f - Gpi);
    n6 = __fmul_rn(n6, 1.f - Gpi);
    // g* = N^-1 n* (Eq. 41); g*_0 = T - sum g*_1..6 keeps sum g* = T free of rounding drift
    // (n_0* = T; a rounded 1/6 factor would otherwise bias it); then g+ = g* + Q (Eq. 40).
    const float s6 = 1.f / 6.f;
    float n456 = n4 + n5 + n6;
    float h1 = __fmul_rn(s6, n456 + 3.f * n1), h2 = __fmul_rn(s6, n456 - 3.f * n1);
    float n4_5 = n4 - 2.f * n5 + n6;
    float h3 = __fmul_rn(s6, n4_5 + 3.f * n2), h4 = __fmul_rn(s6, n4_5 - 3.f * n2);
    float n4_6 = n4 + n5 - 2.f * n6;
    float h5 = __fmul_rn(s6, n4_6 + 3.f * n3), h6 = __fmul_rn(s6, n4_6 - 3.f * n3);
    float h0 = T - ((h1 + h2) + (h3 + h4) + (h5 + h6));
    float q0 = P.w0 * qs, q1 = P.w1 * qs;
    g[0] = h0 + q0;
    g[1] = h1 + q1; g[2] = h2 + q1; g[3] = h3 + q1;
    g[4] = h4 + q1; g[5] = h5 + q1; g[6] = h6 + q1;
    return phis;
}

// ---------------------------------------------------------------- D3Q19 temperature LB
// The BGK equation of Eq. 19 on the D3Q19 lattice: g_eq = w_a T with the standard weights,
// cs_T^2 = 1/3, chi = (tau_g - 1/2) cs_T^2; grad T = -sum e_a g_a / (tau_g cs_T^2) from the
// pre-collision first moment (the D3Q19 form of Eq. 45: sum e g_eq = 0 and sum e Q = 0).
__host__ __device__ constexpr float w19(int a) { return a == 0 ? 1.f / 3.f : a <= 6 ? 1.f / 18.f : 1.f / 36.f; }

// Pull of g_a on the D3Q19 velocities: g_a(x, t+1) = g+_a(x - e_a, t), or, where x - e_a lies
// behind a face that is not periodic for g, Eq. 51 at the node itself:
// g_a(x, t+1) = -g+_abar(x, t) + 2 w_a T_w (the face of the highest axis crossed gives T_w).
template <typename S, int A>
__device__ __forceinline__ float pull_g19_one(const DevParams& P, const S* __restrict__ src, int i, int x, int y,
                                              int z, const Nbr& n) {
    constexpr int ex = ex19(A), ey = ey19(A), ez = ez19(A);
    // faces crossed by the source x - e_a: ex > 0 -> -x (bit 0), ex < 0 -> +x (bit 1), etc.
    const bool cx = ex > 0 ? (n.gabb & 1u) : ex < 0 ? (n.gabb & 2u) : 0u;
    const bool cy = ey > 0 ? (n.gabb & 4u) : ey < 0 ? (n.gabb & 8u) : 0u;
    const bool cz = ez > 0 ? (n.gabb & 16u) : ez < 0 ? (n.gabb & 32u) : 0u;
    if (A != 0 && (cx || cy || cz)) {
        const int face = cz ? (ez > 0 ? 4 : 5) : cy ? (ey > 0 ? 2 : 3) : (ex > 0 ? 0 : 1);
        const float gp = Codec<S>::load(src + (size_t)gslot19(opp(A)) * P.Ns + bidx(P, i, P.Nidx), 0.f);
        return -gp + 2.f * w19(A) * wall_T(P, face, x, y);
    }
    const int s = sidx(P, src_c(ex, x, n.xm, n.xp), src_c(ey, y, n.ym, n.yp), src_c(ez, z, n.zm, n.zp));
    return Codec<S>::load(src + (size_t)gslot19(A) * P.Ns + bidx(P, s, P.Nidx), 0.f);
}

template <typename S>
__device__ __forceinline__ void load_g19(const DevParams& P, const S* __restrict__ src, int pull, int i, int x,
                                         int y, int z, const Nbr& n, float g[19]) {
    if (pull) {
#define GB300_PULL(A) g[A] = pull_g19_one<S, A>(P, src, i, x, y, z, n);
        GB300_PULL(0) GB300_PULL(1) GB300_PULL(2) GB300_PULL(3) GB300_PULL(4) GB300_PULL(5)
        GB300_PULL(6) GB300_PULL(7) GB300_PULL(8) GB300_PULL(9) GB300_PULL(10) GB300_PULL(11)
        GB300_PULL(12) GB300_PULL(13) GB300_PULL(14) GB300_PULL(15) GB300_PULL(16) GB300_PULL(17)
        GB300_PULL(18)
#undef GB300_PULL
    } else {
#pragma unroll
        for (int a = 0; a < 19; ++a) g[a] = Codec<S>::load(src + (size_t)gslot19(a) * P.Ns + bidx(P, i, P.Nidx), 0.f);
    }
}

// the 19 f and 19 g of a node at storage index i (FP32 storage only)
template <typename S>
__device__ __forceinline__ void store_slots19(const DevParams& P, S* __restrict__ dst, int i, const float f[19],
                                              const float g[19]) {
    S* q = dst + bidx(P, i, P.Nidx);
#pragma unroll
    for (int a = 0; a < 19; ++a) Codec<S>::store(q + (size_t)fslot(a) * P.Ns, f[a], 0.f);
#pragma unroll
    for (int a = 0; a < 19; ++a) Codec<S>::store(q + (size_t)gslot19(a) * P.Ns, g[a], 0.f);
}

// In: post-streaming g (19), rho, T = sum g, the flow quantities o, grad rho, phi_s(t-1).
// Out: g+ = g - (g - w T) / tau_g + Q (Eq. 19, Eq. 23) in place; returns phi_s (Eq. 18).
__device__ __forceinline__ float collide_g19(const DevParams& P, float g[19], float rho, float T,
                                             const NodeOut& o, float grx, float gry, float grz,
                                             float phis_prev, int first) {
    const float jx = ((g[1] - g[2]) + (g[7] - g[8])) + ((g[9] - g[10]) + (g[11] - g[12])) + (g[13] - g[14]);
    const float jy = ((g[3] - g[4]) + (g[7] - g[8])) + ((g[10] - g[9]) + (g[15] - g[16])) + (g[17] - g[18]);
    const float jz = ((g[5] - g[6]) + (g[11] - g[12])) + ((g[14] - g[13]) + (g[15] - g[16])) + (g[18] - g[17]);
    const float inv_rho = o.inv_rho;
    const float chi = P.lambda_mode ? P.chi_or_lambda * inv_rho * P.inv_cV : P.chi_or_lambda;
    const float tau = __fmaf_rn(3.f, chi, 0.5f);             // chi = (tau_g - 1/2) / 3
    const float inv_tau = __fdividef(1.f, tau);
    const float k = -3.f * inv_tau;                          // -1 / (tau_g cs_T^2)
    const float gTx = k * jx, gTy = k * jy, gTz = k * jz;
    float phis;
    if (!P.flow_off) {
        phis = __fmaf_rn(chi * grz * inv_rho - o.uz, gTz,
                         __fmaf_rn(chi * gry * inv_rho - o.uy, gTy, __fmul_rn(chi * grx * inv_rho - o.ux, gTx)));
        phis -= __fdividef(T * P.R_over_cV, 1.f - P.b * rho) * o.divu;
    } else {
        phis = __fmaf_rn(chi * grz * inv_rho, gTz, __fmaf_rn(chi * gry * inv_rho, gTy, __fmul_rn(chi * grx * inv_rho, gTx)));
    }
    const float C = first ? phis : phis_prev;
    const float qs = __fmaf_rn(-0.5f, C, __fmul_rn(1.5f, phis));
    // g+_a = g_a - (g_a - w_a T) / tau + w_a qs for a >= 1; g+_0 = T + qs - sum of the others, so
    // that sum g+ = T + qs holds free of rounding drift
    float s = 0.f;
#pragma unroll
    for (int a = 1; a < 19; ++a) {
        const float wa = w19(a);
        g[a] = __fmaf_rn(wa, qs, __fmaf_rn(-inv_tau, __fsub_rn(g[a], __fmul_rn(wa, T)), g[a]));
        s += g[a];
    }
    g[0] = (T + qs) - s;
    return phis;
}

// ---------------------------------------------------------------- thermal lattice traits
// The generic and two-pass kernels take the temperature lattice as a template parameter: QT = 7
// (D3Q7 MRT, Eqs. 38-43) or 19 (Eq. 19 BGK on D3Q19, FP32 storage).
template <int QT> struct Therm;
template <> struct Therm<7> {
    static constexpr int Q = 7;
    template <typename S>
    static __device__ __forceinline__ void load(const DevParams& P, const S* src, int pull, int i, int x, int y, int z,
                                                const Nbr& n, float g[7]) {
        load_g<S>(P, src, pull, i, x, y, z, n, g);
    }
    static __device__ __forceinline__ float sum(const float g[7]) { return sum7(g); }
    static __device__ __forceinline__ float collide(const DevParams& P, float g[7], float rho, float T,
                                                    const NodeOut& o, float grx, float gry, float grz,
                                                    float phis_prev, int first) {
        return collide_g(P, g, rho, T, o, grx, gry, grz, phis_prev, first);
    }
    template <typename S>
    static __device__ __forceinline__ void store(const DevParams& P, S* dst, int i, const float f[19],
                                                 const float g[7]) {
        store_slots<S>(P, dst, i, f, g);
    }
    static __device__ __forceinline__ void equilibrium(const DevParams& P, float T, float g[7]) {
        g[0] = P.w0 * T;
#pragma unroll
        for (int a = 1; a < 7; ++a) g[a] = P.w1 * T;
    }
    template <typename S>
    static __device__ __forceinline__ void stored(const DevParams& P, const S* src, int i, float g[7]) {
#pragma unroll
        for (int a = 0; a < 7; ++a) g[a] = Codec<S>::load(src + (size_t)gslot(a) * P.Ns + bidx(P, i, P.Nidx), P.shift_g[a]);
    }
};
template <> struct Therm<19> {
    static constexpr int Q = 19;
    template <typename S>
    static __device__ __forceinline__ void load(const DevParams& P, const S* src, int pull, int i, int x, int y, int z,
                                                const Nbr& n, float g[19]) {
        load_g19<S>(P, src, pull, i, x, y, z, n, g);
    }
    static __device__ __forceinline__ float sum(const float g[19]) { return sum19(g); }
    static __device__ __forceinline__ float collide(const DevParams& P, float g[19], float rho, float T,
                                                    const NodeOut& o, float grx, float gry, float grz,
                                                    float phis_prev, int first) {
        return collide_g19(P, g, rho, T, o, grx, gry, grz, phis_prev, first);
    }
    template <typename S>
    static __device__ __forceinline__ void store(const DevParams& P, S* dst, int i, const float f[19],
                                                 const float g[19]) {
        store_slots19<S>(P, dst, i, f, g);
    }
    static __device__ __forceinline__ void equilibrium(const DevParams&, float T, float g[19]) {
#pragma unroll
        for (int a = 0; a < 19; ++a) g[a] = w19(a) * T;
    }
    template <typename S>
    static __device__ __forceinline__ void stored(const DevParams& P, const S* src, int i, float g[19]) {
#pragma unroll
        for (int a = 0; a < 19; ++a) g[a] = Codec<S>::load(src + (size_t)gslot19(a) * P.Ns + bidx(P, i, P.Nidx), 0.f);
    }
};

}  // namespace gb300lbm
