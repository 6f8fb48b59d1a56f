/*
 * FP64 CPU oracle of the improved 3D thermal pseudopotential LB model
 * (Li, Yu & Luo, "Improved three-dimensional thermal multiphase lattice Boltzmann
 * model for liquid-vapor phase change").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the package smoke check and the CPU
 * baseline leg of bench.py load this library.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * It is the algorithm written out plainly, one node at a time, in the paper's order:
 *   1. rho = sum f, T = sum g                                  (Eq. 10, Eq. 20)
 *   2. psi = sqrt(2 (p_EOS - rho cs^2) / (G c^2)), G = -1      (Eq. 8, Peng-Robinson Eq. 49)
 *   3. F_m = -G psi(x) sum_a w(|e_a|^2) psi(x + e_a) e_a       (Eq. 7)
 *      F_b = (rho - rho_b) g, rho_b = rho_ave or a fixed value  (Sec. IV.C buoyancy)
 *   4. u = (sum e f + F/2) / rho                               (Eq. 10)
 *   5. m = M f, m* = m - Lambda (m - m_eq) + (I - Lambda/2) S  (Eqs. 3, 5, 6, 9)
 *      f* = M^-1 m*                                            (Eq. 4)
 *   6. div u from the m_4 non-equilibrium                      (Eq. 48)
 *   7. n = N g, grad T = -(n_1..3 - 0) / (varsigma_T cs_T^2)    (Eqs. 38, 45)
 *   8. phi_s = (chi grad(rho cV)/(rho cV) - u).grad T
 *              - T/(rho cV) (dp/dT)_rho div u                  (Eq. 18, (dp/dT) ~ rho R/(1-b rho))
 *   9. Q = w (3/2 phi_s(t) - 1/2 phi_s(t-1))                   (Eqs. 23-24, C = w phi_s)
 *  10. n* = n - Gamma (n - n_eq), g+ = N^-1 n* + Q             (Eqs. 39-43)
 *  11. streaming (push, Eq. 4) with halfway bounce-back (Eq. 50) for f and
 *      anti-bounce-back (Eq. 51) for g at wall faces.
 *
 * M is not printed in the paper; its rows are the raw polynomial velocity moments
 * that the equilibrium moments of Eq. 5 and the force moments of Eq. 9 imply, in the
 * order of Eq. 5.  M^-1 is obtained by a generic Gauss-Jordan elimination.  N and
 * N^-1 are the printed matrices of Eqs. 38 and 41.
 *
 * Readings where the paper is silent (the same readings bind the CUDA path):
 *  - c = dt = dx = 1, cs^2 = 1/3, G = -1.
 *  - Tc = 0.0778 a / (0.45724 b R) (the paper's rounded PR constants, Eq. 49 text).
 *  - Eq. 48 is used at every node; Eq. 45 with the local varsigma_T.
 *  - Q at the first step uses C(t-1) := C(t).
 *  - rho_ave used at step t is the FP64 mean of rho at step t-1 (at step 0 the
 *    initial mean).
 *  - Solid / outflow neighbours of the psi and grad-rho stencils take the value of
 *    their fluid mirror image across the face (neutral wetting), unless the -z wall
 *    carries a virtual density (wall_virtual): a fixed one per region (scheme 0), or the
 *    improved virtual-density scheme Sec. III.C names, rho_w = phi rho_ave - drho from the
 *    solid node's fluid neighbours with (phi, drho) from a per-node wettability map
 *    (scheme 1; floored at rho_ave / 10, our addition).
 *  - Options outside the default path: BGK D3Q7 collision (thermal_bgk), isotropic
 *    finite-difference div u away from solid faces (divu_mode 1), and the temperature LB on the
 *    D3Q19 lattice (thermal_q 19): the BGK equation of Eq. 19 with the D3Q19 weights and
 *    cs_T^2 = 1/3 (Sec. III.B), chi = (tau_g - 1/2) cs_T^2, grad T = -sum e g / (tau_g cs_T^2)
 *    (the first moment, as Eq. 45 for D3Q7), the same source Q = w (3/2 phi_s - 1/2 phi_s(t-1)).
 *  - Outflow face: f unknowns copied from the layer inside (zero gradient), g by
 *    Eq. 51 with T fixed at the face temperature.
 *  - Bottom-face hot spot: T_w(x,y) = T_wall[-z] + dT exp(-((x-nx/2)^2+(y-ny/2)^2)/(2 s^2)).
 *
 * Storage is node-major: f[node*19 + a], g[node*7 + a], node = x + nx (y + ny z).
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Arithmetic precision of the state and of every per-node operation.  The oracle is FP64;
 * building with -DORC_REAL=float gives the same algorithm in FP32, which the tests use only to
 * measure the rounding floor of FP32 arithmetic on a case (matrices, parameters, the rho_ave
 * mean and the API stay FP64). */
#ifndef ORC_REAL
#define ORC_REAL double
#endif
typedef ORC_REAL real;

#define Q19 19
#define Q7 7
#define QMAX 19   /* populations of the thermal lattice at most (D3Q19) */

enum { ORC_PERIODIC = 0, ORC_WALL = 1, ORC_OUTFLOW = 2, ORC_THERMAL_ONLY = 3 };

typedef struct {
    int nx, ny, nz;
    int bc[6];               /* faces -x,+x,-y,+y,-z,+z */
    double T_wall[6];
    double hot_dT, hot_sigma;
    double a, b, R, acentric;
    double sigma;            /* thermodynamic-consistency constant of Eq. 9 */
    double tau_e, tau_v, tau_q, tau_pi;
    double cV, d, varsigma_q, varsigma_pi;
    int lambda_mode;         /* 0: constant chi, 1: constant lambda */
    double chi_or_lambda;
    double g[3];
    int flow_off;            /* f frozen: a static fluid (u = 0, div u = 0; Eq. 18 keeps its conduction term) */
    int thermal_off;         /* g frozen (isothermal) */
    double rho_buoy;         /* > 0: fixed reference density of the buoyancy force, else rho_ave */
    int thermal_bgk;         /* 1: single-relaxation-time (BGK) D3Q7 collision: every non-conserved
                                moment relaxes at 1/varsigma_T, in place of the free rates of Eq. 43 */
    int divu_mode;           /* 0: div u by Eq. 48 at every node; 1: isotropic finite differences of
                                u, with Eq. 48 only at nodes whose stencil reaches a wall or
                                outflow face (the traditional treatment Sec. III.C describes) */
    double wall_rho;         /* > 0: wetting -z wall: virtual density of the solid layer below it in
                                the psi and grad-rho stencils (psi at the wall temperature) */
    double wall_rho_patch, wall_patch_half;   /* virtual density inside the square
                                |x - nx/2| < half, |y - ny/2| < half; half 0: none */
    int wall_scheme;         /* 1: virtual density phi rho_ave - drho (floored at rho_ave / 10) from
                                the fluid neighbours of each solid node, every step */
    double wall_phi, wall_drho, wall_phi_patch, wall_drho_patch;
    int thermal_q;           /* thermal lattice: 7 (default; 0 means 7) or 19 (Eq. 19 BGK on D3Q19) */
} orc_params;

typedef struct {
    orc_params p;
    long N;
    real *f, *g, *fn, *gn;
    real *fs, *gp;         /* post-collision f*, g+ */
    real *rho, *T, *psi;
    real *phis_prev, *phis;
    real *divu, *gradT, *gradrho, *Fm;   /* diagnostics of the last step */
    real *uvec;                          /* u of every node (finite-difference div u) */
    real *wphi, *wdrho;                  /* wall scheme 1: phi and drho per (x, y) of the -z wall */
    int first;
    double rho_ave;        /* value the next step uses (FP64 mean) */
    real M[Q19 * Q19], Minv[Q19 * Q19];
    int qt;                /* populations of the thermal lattice (7 or 19) */
    int ok;
} orc_state;

/* D3Q19 velocities in the order of Eq. 2 */
static const int EX[Q19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int EY[Q19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int EZ[Q19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
/* D3Q7 velocities (Eq. 21) */
static const int TX[Q7] = {0, 1, -1, 0, 0, 0, 0};
static const int TY[Q7] = {0, 0, 0, 1, -1, 0, 0};
static const int TZ[Q7] = {0, 0, 0, 0, 0, 1, -1};

/* N and N^-1 as printed (Eqs. 38, 41) */
static const real NMAT[Q7][Q7] = {
    {1, 1, 1, 1, 1, 1, 1},
    {0, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 1, -1, 0, 0},
    {0, 0, 0, 0, 0, 1, -1},
    {0, 1, 1, 1, 1, 1, 1},
    {0, 1, 1, -1, -1, 0, 0},
    {0, 1, 1, 0, 0, -1, -1}};
static const real NINV6[Q7][Q7] = {   /* times 1/6 */
    {6, 0, 0, 0, -6, 0, 0},
    {0, 3, 0, 0, 1, 1, 1},
    {0, -3, 0, 0, 1, 1, 1},
    {0, 0, 3, 0, 1, -2, 1},
    {0, 0, -3, 0, 1, -2, 1},
    {0, 0, 0, 3, 1, 1, -2},
    {0, 0, 0, -3, 1, 1, -2}};

static const real CS2 = 1.0 / 3.0;
static const real G_INT = -1.0;   /* interaction strength G of Eqs. 7-8 */

/* ---------------------------------------------------------------- matrices */

/* Row k of M evaluated at velocity (x,y,z): the polynomial whose moment is m_k. */
static double m_row(int k, double x, double y, double z) {
    switch (k) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return x * x + y * y + z * z;
    case 5: return 2 * x * x - y * y - z * z;
    case 6: return y * y - z * z;
    case 7: return x * y;
    case 8: return x * z;
    case 9: return y * z;
    case 10: return x * x * y;
    case 11: return x * y * y;
    case 12: return x * x * z;
    case 13: return x * z * z;
    case 14: return y * y * z;
    case 15: return y * z * z;
    case 16: return x * x * y * y;
    case 17: return x * x * z * z;
    case 18: return y * y * z * z;
    }
    return 0.0;
}

void orc_matrix_M(double* M) {
    for (int k = 0; k < Q19; ++k)
        for (int a = 0; a < Q19; ++a) M[k * Q19 + a] = m_row(k, EX[a], EY[a], EZ[a]);
}

/* generic Gauss-Jordan inverse with partial pivoting; returns 0 on success */
int orc_invert(int n, const double* A, double* Ainv) {
    double* w = (double*)malloc(sizeof(double) * n * 2 * n);
    if (!w) return -1;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < 2 * n; ++j)
            w[i * 2 * n + j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(w[r * 2 * n + c]) > fabs(w[piv * 2 * n + c])) piv = r;
        if (fabs(w[piv * 2 * n + c]) < 1e-300) { free(w); return -2; }
        if (piv != c)
            for (int j = 0; j < 2 * n; ++j) {
                double t = w[c * 2 * n + j]; w[c * 2 * n + j] = w[piv * 2 * n + j]; w[piv * 2 * n + j] = t;
            }
        double inv = 1.0 / w[c * 2 * n + c];
        for (int j = 0; j < 2 * n; ++j) w[c * 2 * n + j] *= inv;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double fct = w[r * 2 * n + c];
            if (fct == 0.0) continue;
            for (int j = 0; j < 2 * n; ++j) w[r * 2 * n + j] -= fct * w[c * 2 * n + j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Ainv[i * n + j] = w[i * 2 * n + n + j];
    free(w);
    return 0;
}

void orc_matrix_N(double* N) {
    for (int i = 0; i < Q7; ++i) for (int j = 0; j < Q7; ++j) N[i * Q7 + j] = NMAT[i][j];
}
void orc_matrix_Ninv(double* Ni) {
    for (int i = 0; i < Q7; ++i) for (int j = 0; j < Q7; ++j) Ni[i * Q7 + j] = NINV6[i][j] / 6.0;
}
void orc_velocities19(int* e) { for (int a = 0; a < Q19; ++a) { e[3*a] = EX[a]; e[3*a+1] = EY[a]; e[3*a+2] = EZ[a]; } }

/* ---------------------------------------------------------------- thermodynamics */

/* Peng-Robinson constants: a = 0.45724 R^2 Tc^2/pc and b = 0.0778 R Tc/pc (Eq. 49 text) */
double orc_Tc(const orc_params* p) { return 0.0778 * p->a / (0.45724 * p->b * p->R); }

static real p_eos(const orc_params* p, real rho, real T) {
    real Tc = (real)orc_Tc(p);
    real om = p->acentric;
    real kap = 0.37464 + 1.54226 * om - 0.26992 * om * om;
    real s = 1.0 + kap * (1.0 - sqrt(T / Tc));
    real theta = s * s;                                        /* vartheta(T) */
    return rho * p->R * T / (1.0 - p->b * rho)
         - p->a * theta * rho * rho / (1.0 + 2.0 * p->b * rho - p->b * p->b * rho * rho);
}

double orc_p_eos(const orc_params* p, double rho, double T) { return (double)p_eos(p, (real)rho, (real)T); }

/* (dp/dT)_rho as the paper approximates it in Sec. IV.A */
static real dpdT(const orc_params* p, real rho) { return rho * p->R / (1.0 - p->b * rho); }

/* ---------------------------------------------------------------- collision pieces */

static void m_equilibrium(real rho, const real u[3], real meq[Q19]) {  /* Eq. 5 */
    real ux = u[0], uy = u[1], uz = u[2];
    real u2 = ux * ux + uy * uy + uz * uz;
    real phi = rho * CS2 * CS2 * (1.0 - 1.5 * u2);
    meq[0] = rho;
    meq[1] = rho * ux; meq[2] = rho * uy; meq[3] = rho * uz;
    meq[4] = rho + rho * u2;
    meq[5] = rho * (2 * ux * ux - uy * uy - uz * uz);
    meq[6] = rho * (uy * uy - uz * uz);
    meq[7] = rho * ux * uy; meq[8] = rho * ux * uz; meq[9] = rho * uy * uz;
    meq[10] = rho * CS2 * uy + rho * ux * ux * uy;
    meq[11] = rho * CS2 * ux + rho * uy * uy * ux;
    meq[12] = rho * CS2 * uz + rho * ux * ux * uz;
    meq[13] = rho * CS2 * ux + rho * uz * uz * ux;
    meq[14] = rho * CS2 * uz + rho * uy * uy * uz;
    meq[15] = rho * CS2 * uy + rho * uz * uz * uy;
    meq[16] = phi + rho * CS2 * (ux * ux + uy * uy);
    meq[17] = phi + rho * CS2 * (ux * ux + uz * uz);
    meq[18] = phi + rho * CS2 * (uy * uy + uz * uz);
}

static void force_moments(const orc_params* p, const real F[3], const real u[3],
                          const real Fm[3], real psi2, real S[Q19]) {   /* Eq. 9 */
    real Fx = F[0], Fy = F[1], Fz = F[2], ux = u[0], uy = u[1], uz = u[2];
    real Fm2 = Fm[0] * Fm[0] + Fm[1] * Fm[1] + Fm[2] * Fm[2];
    S[0] = 0.0;
    S[1] = Fx; S[2] = Fy; S[3] = Fz;
    S[4] = 2.0 * (Fx * ux + Fy * uy + Fz * uz) + 6.0 * p->sigma * Fm2 / (psi2 * (p->tau_e - 0.5));
    S[5] = 2.0 * (2 * Fx * ux - Fy * uy - Fz * uz);
    S[6] = 2.0 * (Fy * uy - Fz * uz);
    S[7] = Fx * uy + Fy * ux; S[8] = Fx * uz + Fz * ux; S[9] = Fy * uz + Fz * uy;
    S[10] = CS2 * Fy; S[11] = CS2 * Fx; S[12] = CS2 * Fz;
    S[13] = CS2 * Fx; S[14] = CS2 * Fz; S[15] = CS2 * Fy;
    S[16] = 2 * CS2 * (ux * Fx + uy * Fy);
    S[17] = 2 * CS2 * (ux * Fx + uz * Fz);
    S[18] = 2 * CS2 * (uy * Fy + uz * Fz);
}

static void relaxation_rates(const orc_params* p, real L[Q19]) {   /* Eq. 6 */
    for (int k = 0; k < 4; ++k) L[k] = 1.0;
    L[4] = 1.0 / p->tau_e;
    for (int k = 5; k < 10; ++k) L[k] = 1.0 / p->tau_v;
    for (int k = 10; k < 16; ++k) L[k] = 1.0 / p->tau_q;
    for (int k = 16; k < 19; ++k) L[k] = 1.0 / p->tau_pi;
}

/*
 * MRT collision of one node in moment space (Eq. 3) and back-transform (Eq. 4).
 * Inputs: f (post-streaming), total force F, interaction force Fm, psi^2.
 * Outputs: f*, and (optionally) u, m4 - m4eq, S4 for Eq. 48.
 */
static void collide_f(const orc_state* s, const real f[Q19], const real F[3],
                      const real Fm[3], real psi2, real fstar[Q19],
                      real u_out[3], real* rho_out, real* m4neq, real* S4) {
    const orc_params* p = &s->p;
    real rho = 0.0, j[3] = {0, 0, 0};
    for (int a = 0; a < Q19; ++a) {
        rho += f[a];
        j[0] += EX[a] * f[a]; j[1] += EY[a] * f[a]; j[2] += EZ[a] * f[a];
    }
    real u[3];
    for (int i = 0; i < 3; ++i) u[i] = (j[i] + 0.5 * F[i]) / rho;       /* Eq. 10 */
    real m[Q19], meq[Q19], S[Q19], L[Q19], ms[Q19];
    for (int k = 0; k < Q19; ++k) {
        real acc = 0.0;
        for (int a = 0; a < Q19; ++a) acc += s->M[k * Q19 + a] * f[a];
        m[k] = acc;
    }
    m_equilibrium(rho, u, meq);
    force_moments(p, F, u, Fm, psi2, S);
    relaxation_rates(p, L);
    for (int k = 0; k < Q19; ++k) ms[k] = m[k] - L[k] * (m[k] - meq[k]) + (1.0 - 0.5 * L[k]) * S[k];
    for (int a = 0; a < Q19; ++a) {
        real acc = 0.0;
        for (int k = 0; k < Q19; ++k) acc += s->Minv[a * Q19 + k] * ms[k];
        fstar[a] = acc;
    }
    if (u_out) { u_out[0] = u[0]; u_out[1] = u[1]; u_out[2] = u[2]; }
    if (rho_out) *rho_out = rho;
    if (m4neq) *m4neq = m[4] - meq[4];
    if (S4) *S4 = S[4];
}

/* ---------------------------------------------------------------- lattice helpers */

static long node_index(const orc_params* p, int x, int y, int z) {
    return (long)x + (long)p->nx * ((long)y + (long)p->ny * (long)z);
}

/* Neighbour x+e of the psi / grad-rho stencil: wrap periodic axes, mirror at walls. */
static long stencil_neighbour(const orc_params* p, int x, int y, int z, int ex, int ey, int ez) {
    int c[3] = {x + ex, y + ey, z + ez};
    int n[3] = {p->nx, p->ny, p->nz};
    for (int k = 0; k < 3; ++k) {
        if (c[k] >= 0 && c[k] < n[k]) continue;
        int face = 2 * k + (c[k] < 0 ? 0 : 1);
        int bc = p->bc[face];
        if (bc == ORC_PERIODIC || bc == ORC_THERMAL_ONLY) c[k] = (c[k] + n[k]) % n[k];
        else c[k] = c[k] < 0 ? -1 - c[k] : 2 * n[k] - 1 - c[k];   /* mirror image */
    }
    return node_index(p, c[0], c[1], c[2]);
}

/* 1 if a stencil neighbour of (x, y, z) lies beyond a wall or outflow face */
static int next_to_solid(const orc_params* p, int x, int y, int z) {
    int c[3] = {x, y, z}, n[3] = {p->nx, p->ny, p->nz};
    for (int k = 0; k < 3; ++k) {
        if (c[k] == 0 && !(p->bc[2 * k] == ORC_PERIODIC || p->bc[2 * k] == ORC_THERMAL_ONLY)) return 1;
        if (c[k] == n[k] - 1 && !(p->bc[2 * k + 1] == ORC_PERIODIC || p->bc[2 * k + 1] == ORC_THERMAL_ONLY)) return 1;
    }
    return 0;
}

/* Isotropic finite-difference divergence with the weights of the gradient stencil of Sec. III.C:
   div u (x) = (1/cs^2) sum_a w_a e_a . u(x + e_a) = sum_a W_a e_a . u(x + e_a), W = 1/6 on the
   faces (w = 1/18), 1/12 on the edges (w = 1/36); u holds 3 values per node. */
static real fd_divergence(const orc_params* p, const real* u, int x, int y, int z) {
    real acc = 0.0;
    for (int a = 1; a < Q19; ++a) {
        int e2 = EX[a] * EX[a] + EY[a] * EY[a] + EZ[a] * EZ[a];
        real w = e2 == 1 ? 1.0 / 6.0 : 1.0 / 12.0;
        long j = stencil_neighbour(p, x, y, z, EX[a], EY[a], EZ[a]);
        acc += w * (EX[a] * u[3 * j] + EY[a] * u[3 * j + 1] + EZ[a] * u[3 * j + 2]);
    }
    return acc;
}

static real wall_T(const orc_params* p, int face, int x, int y) {
    real T = p->T_wall[face];
    if (face == 4 && p->hot_dT != 0.0) {
        real dx = x - 0.5 * p->nx, dy = y - 0.5 * p->ny;
        T += p->hot_dT * exp(-(dx * dx + dy * dy) / (2.0 * p->hot_sigma * p->hot_sigma));
    }
    return T;
}

static int opposite19(int a) { return a == 0 ? 0 : ((a & 1) ? a + 1 : a - 1); }
static int opposite7(int a) { return a == 0 ? 0 : ((a & 1) ? a + 1 : a - 1); }

/* weights and velocities of the thermal lattice: D3Q7 (w_0 = 1 - d, w_1..6 = d/6, Eq. 21) or
   D3Q19 (the standard weights 1/3, 1/18, 1/36; Sec. III.B) */
static void thermal_weights(const orc_state* s, real w[QMAX]) {
    if (s->qt == 19) {
        for (int a = 0; a < Q19; ++a) {
            int e2 = EX[a] * EX[a] + EY[a] * EY[a] + EZ[a] * EZ[a];
            w[a] = e2 == 0 ? 1.0 / 3.0 : (e2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        }
    } else {
        w[0] = 1.0 - s->p.d;
        for (int a = 1; a < Q7; ++a) w[a] = s->p.d / 6.0;
    }
}
static void thermal_velocity(const orc_state* s, int a, int e[3]) {
    if (s->qt == 19) { e[0] = EX[a]; e[1] = EY[a]; e[2] = EZ[a]; }
    else { e[0] = TX[a]; e[1] = TY[a]; e[2] = TZ[a]; }
}

/* ---------------------------------------------------------------- API */

/* M and its inverse in FP64, then stored in the state's precision */
static int fill_matrices(orc_state* s) {
    double M[Q19 * Q19], Mi[Q19 * Q19];
    orc_matrix_M(M);
    if (orc_invert(Q19, M, Mi) != 0) return -1;
    for (int k = 0; k < Q19 * Q19; ++k) { s->M[k] = (real)M[k]; s->Minv[k] = (real)Mi[k]; }
    return 0;
}

orc_state* orc_create(const orc_params* p) {
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return NULL;
    orc_state* s = (orc_state*)calloc(1, sizeof(orc_state));
    if (!s) return NULL;
    s->p = *p;
    s->N = (long)p->nx * p->ny * p->nz;
    long N = s->N;
    s->f = (real*)malloc(sizeof(real) * N * Q19);
    s->fn = (real*)malloc(sizeof(real) * N * Q19);
    s->fs = (real*)malloc(sizeof(real) * N * Q19);
    if (p->thermal_q != 0 && p->thermal_q != 7 && p->thermal_q != 19) { free(s); return NULL; }
    s->qt = p->thermal_q == 19 ? 19 : 7;
    s->g = (real*)malloc(sizeof(real) * N * s->qt);
    s->gn = (real*)malloc(sizeof(real) * N * s->qt);
    s->gp = (real*)malloc(sizeof(real) * N * s->qt);
    s->rho = (real*)malloc(sizeof(real) * N);
    s->T = (real*)malloc(sizeof(real) * N);
    s->psi = (real*)malloc(sizeof(real) * N);
    s->phis_prev = (real*)malloc(sizeof(real) * N);
    s->phis = (real*)malloc(sizeof(real) * N);
    s->divu = (real*)malloc(sizeof(real) * N);
    s->uvec = (real*)malloc(sizeof(real) * N * 3);
    s->gradT = (real*)malloc(sizeof(real) * N * 3);
    s->gradrho = (real*)malloc(sizeof(real) * N * 3);
    s->Fm = (real*)malloc(sizeof(real) * N * 3);
    if (!s->f || !s->fn || !s->fs || !s->g || !s->gn || !s->gp || !s->rho || !s->T || !s->psi ||
        !s->phis_prev || !s->phis || !s->divu || !s->uvec || !s->gradT || !s->gradrho || !s->Fm) {
        return NULL;
    }
    if (fill_matrices(s)) return NULL;
    /* wettability map of a scheme-1 wall: the patch values inside the square around
       (nx/2, ny/2), the rest values elsewhere, until orc_set_wall_map replaces it */
    s->wphi = (real*)malloc(sizeof(real) * p->nx * p->ny);
    s->wdrho = (real*)malloc(sizeof(real) * p->nx * p->ny);
    if (!s->wphi || !s->wdrho) return NULL;
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            real dx = (real)x - 0.5 * p->nx, dy = (real)y - 0.5 * p->ny, h = p->wall_patch_half;
            int in = h > 0.0 && fabs(dx) < h && fabs(dy) < h;
            s->wphi[y * p->nx + x] = in ? p->wall_phi_patch : p->wall_phi;
            s->wdrho[y * p->nx + x] = in ? p->wall_drho_patch : p->wall_drho;
        }
    s->first = 1;
    s->ok = 1;
    return s;
}

/* replace the wettability map (nx * ny values each, x fastest); -1 and no change if a phi <= 0,
   a drho < 0 or a value is not finite */
int orc_set_wall_map(orc_state* s, const double* phi, const double* drho) {
    long M = (long)s->p.nx * s->p.ny;
    for (long i = 0; i < M; ++i)
        if (!(phi[i] > 0.0) || !(drho[i] >= 0.0) || !isfinite(phi[i]) || !isfinite(drho[i])) return -1;
    for (long i = 0; i < M; ++i) {
        s->wphi[i] = (real)phi[i];
        s->wdrho[i] = (real)drho[i];
    }
    return 0;
}

void orc_destroy(orc_state* s) {
    if (!s) return;
    free(s->f); free(s->fn); free(s->fs); free(s->g); free(s->gn); free(s->gp);
    free(s->rho); free(s->T); free(s->psi); free(s->phis_prev); free(s->phis);
    free(s->divu); free(s->uvec); free(s->gradT); free(s->gradrho); free(s->Fm);
    free(s->wphi); free(s->wdrho);
    free(s);
}

/* f = M^-1 m_eq(rho, u0), g = w T (w_0 = 1-d, w_1..6 = d/6, Sec. III.B) */
int orc_init(orc_state* s, const double* rho, const double* T, const double* u) {
    real wT[QMAX];
    thermal_weights(s, wT);
    double sum = 0.0;
    for (long i = 0; i < s->N; ++i) {
        real uu[3] = {0, 0, 0};
        if (u) { uu[0] = u[i]; uu[1] = u[s->N + i]; uu[2] = u[2 * s->N + i]; }
        real meq[Q19];
        m_equilibrium((real)rho[i], uu, meq);
        for (int a = 0; a < Q19; ++a) {
            real acc = 0.0;
            for (int k = 0; k < Q19; ++k) acc += s->Minv[a * Q19 + k] * meq[k];
            s->f[i * Q19 + a] = acc;
        }
        for (int a = 0; a < s->qt; ++a) s->g[i * s->qt + a] = wT[a] * (real)T[i];
        sum += (double)(real)rho[i];
    }
    s->rho_ave = sum / (real)s->N;
    s->first = 1;
    return 0;
}

/* rho, T, psi of every node from the current (post-streaming) populations */
static int macroscopic(orc_state* s) {
    const orc_params* p = &s->p;
    long N = s->N;
    int bad = 0;
#pragma omp parallel for reduction(| : bad) schedule(static)
    for (long i = 0; i < N; ++i) {
        real r = 0.0, t = 0.0;
        for (int a = 0; a < Q19; ++a) r += s->f[i * Q19 + a];
        for (int a = 0; a < s->qt; ++a) t += s->g[i * s->qt + a];
        s->rho[i] = r;
        s->T[i] = t;
        real arg = 2.0 * (p_eos(p, r, t) - r * CS2) / (G_INT * 1.0);   /* Eq. 8, c = 1 */
        if (!(arg > 0.0) || !isfinite(r) || !isfinite(t)) bad = 1;
        s->psi[i] = sqrt(arg);
    }
    return bad;
}

/* psi and rho of the solid node (x, y, -1) below a wetting -z wall, psi from Eqs. 8, 49 at
   T_w(x, y).  Scheme 0: the fixed virtual density (the patch value inside the square around
   (nx/2, ny/2)).  Scheme 1 (the improved virtual-density scheme named in Sec. III.C), with the
   node's (phi, drho) from the wettability map:
   rho_w = phi rho_ave - drho, rho_ave = sum_a w_a rho(x_s + e_a) s(x_s + e_a) / sum_a w_a s(x_s + e_a)
   over the velocity set, s = 1 on fluid nodes and 0 on solid ones; floored at rho_ave / 10 so that
   psi_w stays real. */
static void wall_virtual(const orc_state* s, int x, int y, real* psi, real* rho) {
    const orc_params* p = &s->p;
    real dx = (real)x - 0.5 * p->nx, dy = (real)y - 0.5 * p->ny;
    real h = p->wall_patch_half;
    int in = h > 0.0 && fabs(dx) < h && fabs(dy) < h;
    real rw;
    if (p->wall_scheme == 1) {
        real num = 0.0, den = 0.0;
        for (int a = 1; a < Q19; ++a) {
            if (EZ[a] != 1) continue;   /* the other neighbours of (x, y, -1) are solid */
            int e2 = EX[a] * EX[a] + EY[a] * EY[a] + EZ[a] * EZ[a];
            real w = e2 == 1 ? 1.0 / 6.0 : 1.0 / 12.0;
            long j = stencil_neighbour(p, x, y, -1, EX[a], EY[a], EZ[a]);
            num += w * s->rho[j];
            den += w;
        }
        real ra = num / den;
        real phi = s->wphi[y * p->nx + x], drho = s->wdrho[y * p->nx + x];
        rw = phi * ra - drho;
        if (rw < 0.1 * ra) rw = 0.1 * ra;
    } else {
        rw = in ? (real)p->wall_rho_patch : (real)p->wall_rho;
    }
    real Tw = wall_T(p, 4, x, y);
    *psi = sqrt(2.0 * (p_eos(p, rw, Tw) - rw * CS2) / (G_INT * 1.0));
    *rho = rw;
}

/* per-node force pieces: F_m (Eq. 7) and the isotropic gradient of rho (stencil of Sec. III.C) */
static void node_forces(const orc_state* s, int x, int y, int z, real Fm[3], real grho[3]) {
    const orc_params* p = &s->p;
    long i = node_index(p, x, y, z);
    const int wet = (p->wall_rho > 0.0 || p->wall_scheme == 1) && p->bc[4] == ORC_WALL;
    real acc[3] = {0, 0, 0}, gr[3] = {0, 0, 0};
    for (int a = 1; a < Q19; ++a) {
        int e2 = EX[a] * EX[a] + EY[a] * EY[a] + EZ[a] * EZ[a];
        real w = e2 == 1 ? 1.0 / 6.0 : 1.0 / 12.0;
        long j = stencil_neighbour(p, x, y, z, EX[a], EY[a], EZ[a]);
        real ps = s->psi[j], rh = s->rho[j];
        if (wet && z + EZ[a] < 0) {   /* solid layer below the wetting wall */
            long jj = stencil_neighbour(p, x, y, 0, EX[a], EY[a], 0);
            wall_virtual(s, (int)(jj % p->nx), (int)((jj / p->nx) % p->ny), &ps, &rh);
        }
        acc[0] += w * ps * EX[a]; acc[1] += w * ps * EY[a]; acc[2] += w * ps * EZ[a];
        gr[0] += w * rh * EX[a]; gr[1] += w * rh * EY[a]; gr[2] += w * rh * EZ[a];
    }
    for (int k = 0; k < 3; ++k) {
        Fm[k] = -G_INT * s->psi[i] * acc[k];
        grho[k] = gr[k];
    }
}

static void push_stream(orc_state* s) {
    const orc_params* p = &s->p;
    long N = s->N;
    int n[3] = {p->nx, p->ny, p->nz};
    const int qt = s->qt;
    real wT[QMAX];
    thermal_weights(s, wT);
    for (long i = 0; i < N * Q19; ++i) s->fn[i] = NAN;
    for (long i = 0; i < N * qt; ++i) s->gn[i] = NAN;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long i = node_index(p, x, y, z);
                int c0[3] = {x, y, z};
                if (!p->flow_off) {
                    for (int a = 0; a < Q19; ++a) {
                        int c[3] = {x + EX[a], y + EY[a], z + EZ[a]};
                        int wall = 0, out = 0;
                        for (int k = 0; k < 3; ++k) {
                            if (c[k] >= 0 && c[k] < n[k]) continue;
                            int bc = p->bc[2 * k + (c[k] < 0 ? 0 : 1)];
                            if (bc == ORC_PERIODIC || bc == ORC_THERMAL_ONLY) c[k] = (c[k] + n[k]) % n[k];
                            else if (bc == ORC_WALL) wall = 1;
                            else out = 1;
                        }
                        if (wall) s->fn[i * Q19 + opposite19(a)] = s->fs[i * Q19 + a];     /* Eq. 50 */
                        else if (!out) s->fn[node_index(p, c[0], c[1], c[2]) * Q19 + a] = s->fs[i * Q19 + a];
                        /* else: leaves through an outflow face */
                    }
                }
                if (!p->thermal_off) {
                    for (int a = 0; a < qt; ++a) {
                        int e[3];
                        thermal_velocity(s, a, e);
                        int c[3] = {x + e[0], y + e[1], z + e[2]};
                        int face = -1;
                        for (int k = 0; k < 3; ++k) {
                            if (c[k] >= 0 && c[k] < n[k]) continue;
                            int fc = 2 * k + (c[k] < 0 ? 0 : 1);
                            if (p->bc[fc] == ORC_PERIODIC) c[k] = (c[k] + n[k]) % n[k];
                            else face = fc;
                        }
                        if (face >= 0) {   /* Eq. 51, anti-bounce-back with the face temperature */
                            real Tw = wall_T(p, face, c0[0], c0[1]);
                            s->gn[i * qt + opposite7(a)] = -s->gp[i * qt + a] + 2.0 * wT[a] * Tw;
                        } else {
                            s->gn[node_index(p, c[0], c[1], c[2]) * qt + a] = s->gp[i * qt + a];
                        }
                    }
                }
            }
    /* outflow faces: unknown incoming f copied from the layer inside (zero normal gradient) */
    if (!p->flow_off) {
        for (int z = 0; z < p->nz; ++z)
            for (int y = 0; y < p->ny; ++y)
                for (int x = 0; x < p->nx; ++x) {
                    long i = node_index(p, x, y, z);
                    for (int a = 0; a < Q19; ++a) {
                        if (!isnan(s->fn[i * Q19 + a])) continue;
                        int c[3] = {x, y, z};
                        int src[3] = {x - EX[a], y - EY[a], z - EZ[a]};
                        for (int k = 0; k < 3; ++k) {
                            if (src[k] >= 0 && src[k] < n[k]) continue;
                            int bc = p->bc[2 * k + (src[k] < 0 ? 0 : 1)];
                            if (bc == ORC_OUTFLOW) c[k] += src[k] < 0 ? 1 : -1;
                        }
                        s->fn[i * Q19 + a] = s->fn[node_index(p, c[0], c[1], c[2]) * Q19 + a];
                    }
                }
    }
    if (p->flow_off) memcpy(s->fn, s->f, sizeof(real) * N * Q19);
    if (p->thermal_off) memcpy(s->gn, s->g, sizeof(real) * N * qt);
    real* t;
    t = s->f; s->f = s->fn; s->fn = t;
    t = s->g; s->g = s->gn; s->gn = t;
}

/* one time step; returns 0, or -5 when a non-finite value or psi^2 <= 0 appears */
static int step_once(orc_state* s) {
    const orc_params* p = &s->p;
    long N = s->N;
    if (macroscopic(s)) return -5;
    real rho_ave = p->rho_buoy > 0.0 ? (real)p->rho_buoy : (real)s->rho_ave;
    double sum = 0.0;
    for (long i = 0; i < N; ++i) sum += s->rho[i];
    const int qt = s->qt;
    real wT[QMAX];
    thermal_weights(s, wT);
    const real csT2 = qt == 19 ? 1.0 / 3.0 : p->d / 3.0;   /* cs_T^2 = d/3 (D3Q7), 1/3 (D3Q19) */
    real Gam_q = 1.0 / p->varsigma_q, Gam_pi = 1.0 / p->varsigma_pi;
    if (p->divu_mode == 1) {
        /* u of every node first (Eq. 10 with the total force), for the finite differences */
#pragma omp parallel for schedule(static)
        for (int z = 0; z < p->nz; ++z)
            for (int y = 0; y < p->ny; ++y)
                for (int x = 0; x < p->nx; ++x) {
                    long i = node_index(p, x, y, z);
                    real rho = s->rho[i], Fm[3], grho[3], j[3] = {0.0, 0.0, 0.0};
                    node_forces(s, x, y, z, Fm, grho);
                    for (int a = 0; a < Q19; ++a) {
                        j[0] += EX[a] * s->f[i * Q19 + a];
                        j[1] += EY[a] * s->f[i * Q19 + a];
                        j[2] += EZ[a] * s->f[i * Q19 + a];
                    }
                    for (int k = 0; k < 3; ++k)
                        s->uvec[3 * i + k] = (j[k] + 0.5 * (Fm[k] + (rho - rho_ave) * p->g[k])) / rho;
                }
    }
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long i = node_index(p, x, y, z);
                real rho = s->rho[i], T = s->T[i];
                real Fm[3], grho[3], F[3];
                node_forces(s, x, y, z, Fm, grho);
                for (int k = 0; k < 3; ++k) F[k] = Fm[k] + (rho - rho_ave) * p->g[k];
                real psi2 = s->psi[i] * s->psi[i];
                real u[3], rr, m4neq, S4;
                collide_f(s, &s->f[i * Q19], F, Fm, psi2, &s->fs[i * Q19], u, &rr, &m4neq, &S4);
                /* Eq. 48 */
                real Fu = F[0] * u[0] + F[1] * u[1] + F[2] * u[2];
                real divu = (-m4neq / p->tau_e + (1.0 - 0.5 / p->tau_e) * S4 - 2.0 * Fu) / (2.0 * rho * CS2);
                if (p->divu_mode == 1 && !next_to_solid(p, x, y, z)) divu = fd_divergence(p, s->uvec, x, y, z);
                real chi = p->lambda_mode ? p->chi_or_lambda / (rho * p->cV) : p->chi_or_lambda;
                real vsT = chi / csT2 + 0.5;     /* chi = (varsigma_T - 0.5) cs_T^2 dt (tau_g on D3Q19) */
                real gT[3];
                real nm[Q7];
                if (qt == 7) {
                    /* thermal moments, Eq. 38 */
                    for (int k = 0; k < Q7; ++k) {
                        real acc = 0.0;
                        for (int a = 0; a < Q7; ++a) acc += NMAT[k][a] * s->g[i * Q7 + a];
                        nm[k] = acc;
                    }
                    for (int k = 0; k < 3; ++k) gT[k] = -(nm[1 + k] - 0.0) / (vsT * csT2);   /* Eq. 45 */
                } else {
                    /* D3Q19: the first moment is all non-equilibrium (sum e g_eq = 0, sum e Q = 0) */
                    real j[3] = {0.0, 0.0, 0.0};
                    for (int a = 0; a < Q19; ++a) {
                        j[0] += EX[a] * s->g[i * Q19 + a];
                        j[1] += EY[a] * s->g[i * Q19 + a];
                        j[2] += EZ[a] * s->g[i * Q19 + a];
                    }
                    for (int k = 0; k < 3; ++k) gT[k] = -j[k] / (vsT * csT2);
                }
                /* Eq. 18 with cV constant: grad(rho cV)/(rho cV) = grad rho / rho.  A frozen flow is
                   a static fluid: u = 0 and div u = 0, and only the conduction term remains */
                if (p->flow_off) {
                    u[0] = u[1] = u[2] = 0.0;
                    divu = 0.0;
                }
                real phis = 0.0;
                for (int k = 0; k < 3; ++k) phis += (chi * grho[k] / rho - u[k]) * gT[k];
                phis -= T / (rho * p->cV) * dpdT(p, rho) * divu;
                real phis_old = s->first ? phis : s->phis_prev[i];
                if (qt == 7) {
                    /* Eq. 42 equilibrium moments and Eq. 43 rates */
                    real neq[Q7] = {T, 0.0, 0.0, 0.0, 3.0 * csT2 * T, 0.0, 0.0};
                    real Gm[Q7] = {1.0, 1.0 / vsT, 1.0 / vsT, 1.0 / vsT, Gam_q, Gam_pi, Gam_pi};
                    if (p->thermal_bgk) Gm[4] = Gm[5] = Gm[6] = 1.0 / vsT;   /* BGK: one rate */
                    real ns[Q7];
                    for (int k = 0; k < Q7; ++k) ns[k] = nm[k] - Gm[k] * (nm[k] - neq[k]);    /* Eq. 39 */
                    for (int a = 0; a < Q7; ++a) {
                        real acc = 0.0;
                        for (int k = 0; k < Q7; ++k) acc += NINV6[a][k] / 6.0 * ns[k];
                        real Qa = 1.5 * wT[a] * phis - 0.5 * wT[a] * phis_old;             /* Eq. 23 */
                        s->gp[i * Q7 + a] = acc + Qa;                                        /* Eq. 40 */
                    }
                } else {
                    /* Eq. 19 with g_eq = w T and tau_g = vsT */
                    for (int a = 0; a < Q19; ++a) {
                        real ga = s->g[i * Q19 + a];
                        real Qa = 1.5 * wT[a] * phis - 0.5 * wT[a] * phis_old;             /* Eq. 23 */
                        s->gp[i * Q19 + a] = ga - (ga - wT[a] * T) / vsT + Qa;
                    }
                }
                s->phis[i] = phis;
                s->divu[i] = divu;
                for (int k = 0; k < 3; ++k) {
                    s->gradT[3 * i + k] = gT[k];
                    s->gradrho[3 * i + k] = grho[k];
                    s->Fm[3 * i + k] = Fm[k];
                }
            }
    push_stream(s);
    real* t = s->phis_prev; s->phis_prev = s->phis; s->phis = t;
    s->first = 0;
    s->rho_ave = sum / (real)N;
    return 0;
}

int orc_step(orc_state* s, int nsteps) {
    for (int k = 0; k < nsteps; ++k) {
        int rc = step_once(s);
        if (rc) return rc;
    }
    return 0;
}

/* rho, u = (sum e f + F/2)/rho and T of the current state (F with the rho_ave the next step uses) */
int orc_moments(orc_state* s, double* rho_o, double* ux, double* uy, double* uz, double* T_o) {
    const orc_params* p = &s->p;
    if (macroscopic(s)) return -5;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long i = node_index(p, x, y, z);
                real Fm[3], grho[3];
                node_forces(s, x, y, z, Fm, grho);
                real rho = s->rho[i], j[3] = {0, 0, 0};
                for (int a = 0; a < Q19; ++a) {
                    j[0] += EX[a] * s->f[i * Q19 + a];
                    j[1] += EY[a] * s->f[i * Q19 + a];
                    j[2] += EZ[a] * s->f[i * Q19 + a];
                }
                real u[3];
                for (int k = 0; k < 3; ++k) {
                    real rb = p->rho_buoy > 0.0 ? (real)p->rho_buoy : (real)s->rho_ave;
                    real F = Fm[k] + (rho - rb) * (real)p->g[k];
                    u[k] = p->flow_off ? 0.0 : (j[k] + 0.5 * F) / rho;
                }
                if (rho_o) rho_o[i] = rho;
                if (ux) ux[i] = u[0];
                if (uy) uy[i] = u[1];
                if (uz) uz[i] = u[2];
                if (T_o) T_o[i] = s->T[i];
            }
    return 0;
}

/* ---------------------------------------------------------------- state access for tests */

static void to_double(double* dst, const real* src, long n) { for (long k = 0; k < n; ++k) dst[k] = (double)src[k]; }
static void to_real(real* dst, const double* src, long n) { for (long k = 0; k < n; ++k) dst[k] = (real)src[k]; }

/* f: 19 per node; g: 7 or 19 per node (the thermal lattice) */
void orc_get_pops(const orc_state* s, double* f, double* g) {
    if (f) to_double(f, s->f, s->N * Q19);
    if (g) to_double(g, s->g, s->N * s->qt);
}
void orc_set_pops(orc_state* s, const double* f, const double* g) {
    if (f) to_real(s->f, f, s->N * Q19);
    if (g) to_real(s->g, g, s->N * s->qt);
}
/* diagnostics of the last completed step (pre-streaming values at each node) */
void orc_get_diag(const orc_state* s, double* divu, double* gradT, double* gradrho,
                  double* Fm, double* phis, double* psi) {
    if (divu) to_double(divu, s->divu, s->N);
    if (gradT) to_double(gradT, s->gradT, s->N * 3);
    if (gradrho) to_double(gradrho, s->gradrho, s->N * 3);
    if (Fm) to_double(Fm, s->Fm, s->N * 3);
    if (phis) to_double(phis, s->phis_prev, s->N);
    if (psi) to_double(psi, s->psi, s->N);
}
double orc_get_rho_ave(const orc_state* s) { return s->rho_ave; }
void orc_set_rho_ave(orc_state* s, double v) { s->rho_ave = v; }

/* single-node MRT collision for direct checks of Eqs. 3-10 */
void orc_collide_node(const orc_params* p, const double* f, const double* F, const double* Fm,
                      double psi2, double* fstar, double* u) {
    orc_state tmp;
    memset(&tmp, 0, sizeof(tmp));
    tmp.p = *p;
    fill_matrices(&tmp);
    real fr[Q19], Fr[3], Fmr[3], fs[Q19], ur[3];
    to_real(fr, f, Q19); to_real(Fr, F, 3); to_real(Fmr, Fm, 3);
    collide_f(&tmp, fr, Fr, Fmr, (real)psi2, fs, ur, NULL, NULL, NULL);
    to_double(fstar, fs, Q19);
    to_double(u, ur, 3);
}

/* equilibrium populations M^-1 m_eq(rho, u) */
void orc_feq(double rho, const double* u, double* feq) {
    double M[Q19 * Q19], Mi[Q19 * Q19];
    real meq[Q19], ur[3];
    orc_matrix_M(M);
    orc_invert(Q19, M, Mi);
    to_real(ur, u, 3);
    m_equilibrium((real)rho, ur, meq);
    for (int a = 0; a < Q19; ++a) {
        double acc = 0.0;
        for (int k = 0; k < Q19; ++k) acc += Mi[a * Q19 + k] * (double)meq[k];
        feq[a] = acc;
    }
}

/* forcing populations G = M^-1 S (Eq. 9) */
void orc_force_pops(const orc_params* p, const double* F, const double* u, const double* Fm,
                    double psi2, double* G) {
    double M[Q19 * Q19], Mi[Q19 * Q19];
    real S[Q19], Fr[3], ur[3], Fmr[3];
    orc_matrix_M(M);
    orc_invert(Q19, M, Mi);
    to_real(Fr, F, 3); to_real(ur, u, 3); to_real(Fmr, Fm, 3);
    force_moments(p, Fr, ur, Fmr, (real)psi2, S);
    for (int a = 0; a < Q19; ++a) {
        double acc = 0.0;
        for (int k = 0; k < Q19; ++k) acc += Mi[a * Q19 + k] * (double)S[k];
        G[a] = acc;
    }
}

/* finite-difference divergence of a given field u (3 per node) at every node (test helper) */
void orc_fd_divergence(const orc_params* p, const double* u, double* out) {
    long N = (long)p->nx * p->ny * p->nz;
    real* ur = (real*)malloc(sizeof(real) * 3 * N);
    if (!ur) return;
    for (long k = 0; k < 3 * N; ++k) ur[k] = (real)u[k];
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) out[node_index(p, x, y, z)] = (double)fd_divergence(p, ur, x, y, z);
    free(ur);
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* threads of the following calls (n >= 1; no effect without OpenMP) */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
