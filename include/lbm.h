/*
 * C-ABI of the GB300 (sm_103a) implementation of the per-time-step lattice update of
 * the improved 3D thermal pseudopotential lattice Boltzmann model of
 * Li, Yu & Luo, "Improved three-dimensional thermal multiphase lattice Boltzmann
 * model for liquid-vapor phase change" (arXiv 2201.06039).
 *
 * One time step is: the D3Q19 MRT pseudopotential LB for density and velocity
 * (Sec. II, Eqs. 1-10) with the Peng-Robinson equation of state (Sec. IV.A, Eq. 49),
 * coupled to the D3Q7 MRT temperature LB (Sec. III.C, Eqs. 37-45) whose source
 * phi_s (Eq. 18, with the second-order time extrapolation of Eqs. 23-24) uses the
 * local div u of Eq. 48 and the local grad T of Eq. 45, with halfway bounce-back
 * (Eq. 50) and anti-bounce-back (Eq. 51) walls and the buoyancy force of Sec. IV.C.
 *
 * Units are lattice units: c = dx = dt = 1, cs^2 = 1/3, interaction strength G = -1.
 *
 * Conventions shared by every call
 *  - Fields are float32 arrays of nx*ny*nz values, node index x + nx*(y + ny*z)
 *    (x fastest).  A velocity field is three such planes (ux, uy, uz) back to back.
 *  - Field pointers may be host or device pointers (told apart with
 *    cudaPointerGetAttributes).  They are borrowed for the duration of the call only.
 *  - All device work is enqueued on the stream given in lbm_params.cuda_stream (the
 *    legacy default stream if NULL).  A context is used by one host thread at a time.
 *  - Every call returns an lbm_status; LBM_OK is 0, errors are negative.  After an
 *    error the context stays valid and can be re-initialised with lbm_init_fields.
 *  - The context owns all device memory it allocates; lbm_destroy frees it.  If
 *    lbm_params.workspace is non-NULL the state lives there instead (caller-owned,
 *    at least lbm_workspace_bytes() bytes, 256-byte aligned, device memory), and the
 *    library allocates nothing for the fields.
 */
#ifndef GB300_LBM_H
#define GB300_LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = -1,      /* invalid argument or parameter (message via lbm_last_error) */
    LBM_ENOMEM = -2,      /* device or host allocation failed */
    LBM_ECUDA = -3,       /* a CUDA runtime call failed */
    LBM_ESTATE = -4,      /* call out of order (e.g. lbm_step before lbm_init_fields) */
    LBM_ENONFINITE = -5,  /* a non-finite rho/T/psi, or psi^2 <= 0 (Eq. 8 domain) appeared */
    LBM_ETIMEOUT = -6,    /* a bounded device wait gave up */
    LBM_EBOUNDS = -7      /* bounds-checked builds only: a kernel index fell outside its buffer
                             (the access was skipped; the state is not to be trusted) */
} lbm_status;

/* Boundary type of one face of the box (faces ordered -x, +x, -y, +y, -z, +z). */
typedef enum {
    LBM_BC_PERIODIC = 0,      /* f and g wrap around */
    LBM_BC_WALL = 1,          /* f: halfway bounce-back, Eq. 50; g: anti-bounce-back, Eq. 51 */
    LBM_BC_OUTFLOW = 2,       /* f: zero normal gradient; g: Eq. 51 at T_wall of the face */
    LBM_BC_THERMAL_ONLY = 3   /* f periodic; g: Eq. 51 at T_wall of the face */
} lbm_bc;

typedef enum { LBM_FP32 = 0, LBM_BF16_SHIFTED = 1, LBM_FP16_SHIFTED = 2 } lbm_precision;

typedef enum {
    LBM_KERNEL_AUTO = 0,      /* fastest available variant */
    LBM_KERNEL_TWO_PASS = 1,  /* psi/EOS kernel, then the stream-collide kernel */
    LBM_KERNEL_FUSED = 2,     /* one z-marching kernel per step (halo recomputation) */
    LBM_KERNEL_FUSED_TMA = 3  /* reported by lbm_kernel_in_use: FUSED with TMA-fed pipeline (any
                                 storage precision; x and y faces periodic or thermal-only;
                                 nx, ny >= 4; flow and temperature both evolving) */
} lbm_kernel_variant;

typedef struct {
    int nx, ny, nz;               /* lattice size, each >= 1 */
    int bc[6];                    /* lbm_bc per face: -x, +x, -y, +y, -z, +z */
    double T_wall[6];             /* face temperatures of Eq. 51 (absolute, lattice units) */
    double hot_dT, hot_sigma;     /* -z face: T_w(x,y) = T_wall[4] + hot_dT exp(-r^2/(2 hot_sigma^2)),
                                     r measured from (nx/2, ny/2); hot_dT = 0 disables */
    double a, b, R, acentric;     /* Peng-Robinson EOS (Eq. 49); Tc = 0.0778 a / (0.45724 b R) */
    double sigma;                 /* thermodynamic-consistency constant of Eq. 9 */
    double tau_e, tau_v, tau_q, tau_pi;     /* relaxation times of Eq. 6 (each > 0.5) */
    double cV, d, varsigma_q, varsigma_pi;  /* cV of Eq. 18; D3Q7 d (w0 = 1-d, w1..6 = d/6);
                                               free rates of Eq. 43 */
    int lambda_mode;              /* 0: chi = chi_or_lambda constant; 1: lambda constant,
                                     chi = lambda / (rho cV) per node (Sec. IV.A) */
    double chi_or_lambda;         /* varsigma_T = chi / cs_T^2 + 1/2, cs_T^2 = d/3 */
    double g[3];                  /* gravity of the buoyancy force F_b = (rho - rho_b) g */
    double rho_buoy;              /* rho_b: > 0 fixes it; 0 takes the domain mean rho_ave of the
                                     previous step (Sec. IV.C) */
    int flow_off;                 /* 1: f frozen, a static fluid: u = 0 and div u = 0 in Eq. 18, which keeps its conduction term chi grad(rho cV).grad T/(rho cV) */
    int thermal_off;              /* 1: g frozen (isothermal phase) */
    int precision;                /* lbm_precision of the stored populations */
    double rho_ref, T_ref;        /* shifts of 16-bit storage: f - w rho_ref, g - w T_ref */
    int kernel;                   /* lbm_kernel_variant */
    int use_graph;                /* 1: lbm_step replays a captured CUDA graph of n steps */
    int use_tma;                  /* 1: FUSED uses the TMA-fed pipeline where the lattice allows it */
    int check_nonfinite;          /* 1: lbm_step synchronises and reports LBM_ENONFINITE */
    void* cuda_stream;            /* borrowed cudaStream_t, NULL = legacy default stream */
    void* workspace;              /* optional caller-owned device memory (see above) */
    size_t workspace_bytes;
    int test_stall;               /* test of the timeout path only (0 in normal use): in the next
                                     step of the TMA kernel the producer waits for its first stage
                                     to be released before loading it, which nothing can do, so
                                     the bounded waits give up and lbm_step reports LBM_ETIMEOUT;
                                     cleared once that step is enqueued (never graph-captured) */
    int thermal_bgk;              /* 1: single-relaxation-time (BGK) D3Q7 collision, every
                                     non-conserved moment relaxed at 1/varsigma_T, in place of
                                     the free rates varsigma_q, varsigma_pi of Eq. 43 (MRT) */
    int divu_mode;                /* 0: div u of Eq. 48 at every node (default); 1: isotropic
                                     finite differences of u (gradient weights of Sec. III.C) at
                                     nodes whose stencil stays inside the fluid, Eq. 48 next to
                                     wall and outflow faces.  Runs the two-pass kernels plus a
                                     velocity pass (kernel AUTO or TWO_PASS; FUSED is rejected) */
    double wall_rho;              /* wetting of the -z wall (LBM_BC_WALL): virtual density of the
                                     solid layer below it in the psi and grad-rho stencils (its psi
                                     from Eqs. 8, 49 at the wall temperature); 0 = neutral mirror
                                     (the solid node copies the fluid node above it) */
    double wall_rho_patch, wall_patch_half;   /* virtual density inside the square
                                     |x - nx/2| < half, |y - ny/2| < half of the -z wall (the
                                     hydrophobic region of the boiling test, Sec. IV.C; a side of
                                     55 nodes is half = 27.5); half 0 = no patch */
    int wall_scheme;              /* wetting of the -z wall: 0 = the fixed virtual densities above;
                                     1 = densities that follow the fluid (the improved virtual-density
                                     scheme the paper uses, Sec. III.C): every step the solid node
                                     below (x, y) takes rho_w = max(phi rho_ave - drho, rho_ave / 10),
                                     rho_ave the weighted mean (w = 1/6 face, 1/12 edge) of the
                                     densities of its five fluid neighbours in the layer z = 0;
                                     phi >= 1 makes the wall hydrophilic, drho > 0 hydrophobic.
                                     Needs a -z LBM_BC_WALL and wall_rho = wall_rho_patch = 0 */
    double wall_phi, wall_drho;               /* scheme 1: phi > 0 and drho >= 0 outside the patch */
    double wall_phi_patch, wall_drho_patch;   /* scheme 1: the same inside the patch */
    int    thermal_q;             /* temperature lattice: 7 (0 also means 7; D3Q7 MRT, Eqs. 37-43) or 19
                                     (the BGK equation of Eq. 19 on the D3Q19 lattice, its standard
                                     weights, cs_T^2 = 1/3, Sec. III.B; 38 population slots per node,
                                     generic and two-pass kernels, no batch) */
} lbm_params;

/* Fill *p with the workload-independent defaults of Sec. IV: tau_e = 1.25, tau_v = 0.8,
 * tau_q = tau_pi = 1, cV = 5, d = 0.95, varsigma_q = varsigma_pi = 1, a = 2/49, b = 2/21,
 * R = 1, acentric factor 0.344, all faces periodic, FP32 populations. */
void lbm_params_default(lbm_params* p);

/* Critical temperature and pressure of the Peng-Robinson EOS with the paper's rounded
 * constants (Sec. IV.A text after Eq. 49): Tc = 0.0778 a / (0.45724 b R), pc = 0.0778 R Tc / b. */
int lbm_eos_critical(const lbm_params* p, double* Tc, double* pc);

/* Device bytes the state of a lattice with parameters p needs. */
size_t lbm_workspace_bytes(const lbm_params* p);

/* Validate p (tau > 0.5, sizes >= 1, outflow faces need >= 2 nodes across, ...), allocate
 * the state and create a context.  Errors: LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA. */
int lbm_create(const lbm_params* p, lbm_ctx** out);

/* Set the initial state: f = M^-1 m_eq(rho, u) with the equilibrium moments of Eq. 5,
 * g = w T (Sec. III.B), phi_s history empty (the first step uses C(t-dt) := C(t) in Eq. 23),
 * rho_ave = mean of rho.  rho and T are required; u may be NULL (fluid at rest).
 * Errors: LBM_EINVAL (NULL rho/T), LBM_ECUDA. */
int lbm_init_fields(lbm_ctx* ctx, const float* rho, const float* T, const float* u);

/* Enqueue n >= 0 time steps (each: Eqs. 7-10, 3-6, 9, 48, 45, 18, 23, 39-43, streaming
 * of Eq. 4 with Eqs. 50-51).  Returns after enqueueing, unless check_nonfinite is set, in
 * which case it synchronises the stream and returns LBM_ENONFINITE if any node's rho, T
 * or psi became non-finite or psi^2 <= 0 during these steps, or LBM_ETIMEOUT if a bounded
 * pipeline wait of the TMA kernel gave up (the state of those steps is then not to be trusted;
 * re-initialise), or, in a library built with -DLBM_BOUNDS_CHECK (libgb300lbm_bounds.so), LBM_EBOUNDS
 * if a kernel index fell outside its buffer.
 * Errors: LBM_ESTATE (no init), LBM_EINVAL (n < 0), LBM_ECUDA, LBM_ENONFINITE, LBM_ETIMEOUT,
 * LBM_EBOUNDS. */
int lbm_step(lbm_ctx* ctx, int n);

/* Macroscopic fields of the current state: rho = sum f (Eq. 10), u = (sum e f + F/2)/rho
 * (Eq. 10, F = F_m of Eq. 7 + F_b with the rho_ave the next step uses), T = sum g (Eq. 20).
 * Any output pointer may be NULL.  Synchronises the stream before returning.
 * Errors: LBM_ESTATE, LBM_ECUDA. */
int lbm_get_moments(lbm_ctx* ctx, float* rho, float* ux, float* uy, float* uz, float* T);

/* FP64 totals of the current state, reduced deterministically on the device:
 * mass = sum rho, energy = sum T, and the rho_ave the next step uses.  Synchronises. */
int lbm_get_totals(lbm_ctx* ctx, double* mass, double* T_sum, double* rho_ave);

/* Number of steps taken since lbm_init_fields. */
long long lbm_steps_done(const lbm_ctx* ctx);

/* Checkpoint of the state (every population of the current buffer, the phi_s history of
 * Eqs. 23-24, the sums that give the next step's rho_ave, the step count), for resuming a run
 * later or in another context of the same lattice size and storage precision: the steps that
 * follow lbm_load_state are bit-identical to those the saving context would have taken.
 *   lbm_state_bytes  size of a checkpoint of this context (0 if ctx is NULL)
 *   lbm_save_state   writes it to buf (host memory, at least lbm_state_bytes bytes); synchronises
 *   lbm_load_state   reads it from buf (host memory); LBM_EINVAL if it was written for another
 *                    lattice size or precision, or is not a checkpoint; synchronises
 * Errors: LBM_EINVAL (NULL or short buffer, mismatch), LBM_ESTATE (save before init), LBM_ECUDA. */
size_t lbm_state_bytes(const lbm_ctx* ctx);
int lbm_save_state(lbm_ctx* ctx, void* buf, size_t bytes);
int lbm_load_state(lbm_ctx* ctx, const void* buf, size_t bytes);

/* Wettability map of a scheme-1 wetting wall (wall_scheme 1, Sec. III.C): phi and drho of the
 * solid node below every (x, y) of the -z wall, nx * ny floats each, x fastest, host or device
 * memory (copied; the caller keeps ownership).  lbm_create fills the map from wall_phi /
 * wall_drho and the patch values; this call replaces it for the steps that follow, e.g. to pin
 * a contact line by a step in wettability around a drop's footprint.  The map is a parameter,
 * not part of the state: checkpoints do not carry it.
 * Errors: LBM_EINVAL (NULL ctx or array, a phi <= 0, a drho < 0 or a non-finite value: the map is
 * then left unchanged), LBM_ESTATE (the context has no scheme-1 wall), LBM_ECUDA.  Synchronises. */
int lbm_set_wall_map(lbm_ctx* ctx, const float* phi, const float* drho);

/* Kernel variant the context runs (LBM_KERNEL_TWO_PASS, LBM_KERNEL_FUSED or
 * LBM_KERNEL_FUSED_TMA; AUTO resolved).  The first step after lbm_init_fields, and steps with a
 * frozen field, always run the generic fused kernel. */
int lbm_kernel_in_use(const lbm_ctx* ctx);

/* Tile plan of the TMA kernel (the default path on lattices with f-periodic x and y faces).  A
 * persistent CTA per SM marches tiles of tile_w x tile_h nodes up z; the lattice is cut into
 * items (tile, z-chunk of zchunk planes) taken round robin by the CTAs.  The plan is chosen at
 * lbm_create from a model of the kernel's cost; these calls report, pin or measure it.  Plans do
 * not change results: every plan computes the same state bit for bit.
 *   lbm_plan_shapes  number of tile shapes, and each one's tile_w / tile_h (arrays of max ints;
 *                    either may be NULL)
 *   lbm_get_plan     the plan in use: shape index, z-chunk, items, persistent CTAs (each
 *                    nullable); shape -1 if the context does not run the TMA kernel
 *   lbm_select_plan  pin a shape (-1: the model's choice) and a z-chunk (0: the model's choice
 *                    for that shape); drops the captured step graphs.  LBM_EINVAL if the plan
 *                    does not fit (the previous plan is kept), LBM_ESTATE if the context does not
 *                    run the TMA kernel
 *   lbm_autotune     time `steps` steps of every shape (with its three best modelled z-chunks
 *                    and with whole columns) on the current state, keep the fastest, restore the state
 *                    exactly; best_ms (nullable) receives its time per step.  Takes the pending
 *                    first step after lbm_init_fields first.  Needs free device memory for one
 *                    copy of the state (LBM_ENOMEM otherwise).  Synchronises.
 * No counterpart in the paper: this is the build's scheduling of the update (Secs. II-III). */
int lbm_plan_shapes(int* tile_w, int* tile_h, int max);
int lbm_get_plan(const lbm_ctx* ctx, int* shape, int* zchunk, int* items, int* ctas);
int lbm_select_plan(lbm_ctx* ctx, int shape, int zchunk);
int lbm_autotune(lbm_ctx* ctx, int steps, double* best_ms);

/* Enqueue n steps outside any graph and accumulate, per kernel kind, the device time
 * measured with CUDA events on the context's stream and the number of launches
 * (kernel_ms[0]: psi/EOS or fused kernel, [1]: stream-collide kernel, [2]: ghost-cell
 * refresh and the per-step table of a scheme-1 wetting wall).  Each launch is bracketed by a
 * CUDA event pair on the context's stream; the n steps are enqueued back to back and the events
 * read once at the end, so a launch starts as it would without the events.  Synchronises.  Used
 * for the roofline figures. */
int lbm_step_profiled(lbm_ctx* ctx, int n, double kernel_ms[3], int launches[3]);

/* Allocation-free FP64 sum of a device float field (the paper has no counterpart: this is a
 * service for callers that cannot allocate device memory, e.g. code running under a framework
 * whose memory pool forbids cudaMalloc outside its allocator, plug-ins with a fixed device-memory
 * budget, or latency-critical sections that must not allocate).
 *
 *   field     device (or managed) pointer of the current device to n float32 values, all inside
 *             one allocation (not modified)
 *   n         0 <= n <= LBM_NOALLOC_MAX_ELEMENTS
 *   sum_out   host pointer; receives the sum in FP64 (deterministic: fixed-order block partials
 *             added in index order)
 *   stream    cudaStream_t to run on (NULL = legacy default stream); the call synchronises it
 *
 * The working memory (1024 block partials, a ticket and the result, about 16 KB) is one
 * file-scope device array of the library, present on every GPU that loads the library until the
 * process exits; nothing is allocated per call.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress).  The call synchronises its stream and copies
 * the result to host memory, so it must not be made while its stream is being captured (it
 * returns LBM_ESTATE then, before any work).  Every call shares the array: calls that overlap on
 * the GPU (other streams, other host threads) race and must be serialised by the caller.
 * Errors (message via lbm_last_error): LBM_EINVAL (NULL pointers, n out of range, field not
 * device memory of the current device, or the n floats running past the end of field's
 * allocation: all checked before any launch), LBM_ESTATE (stream capture), LBM_ECUDA. */
#define LBM_NOALLOC_MAX_ELEMENTS (1LL << 31)
int lbm_field_sum_noalloc(const float* field, long long n, double* sum_out, void* stream);

/* ------------------------------------------------------------------ batched ensemble
 * Many independent lattices of uneven sizes advanced together (the same update as lbm_step on
 * each, Secs. II-IV): each time step is ONE persistent kernel launch over all instances, whose
 * CTAs draw (instance, tile column, z-chunk) work items from a table, largest instances first;
 * lbm_batch_step(n) replays the n launches as a captured CUDA graph.  Every plan computes the
 * states of single-lattice contexts bit for bit.
 *
 *   common   parameters shared by every instance (EOS, relaxation times, faces, gravity,
 *            precision, stream, use_graph, check_nonfinite); its nx, ny, nz and workspace
 *            fields are ignored (the batch allocates and owns its device memory)
 *   dims     3 * n_instances ints: (nx, ny, nz) of instance k at dims[3k .. 3k+2]
 *
 * Fields passed to lbm_batch_init_fields and returned by lbm_batch_get_moments are the
 * instances' fields (layout of a single lattice) concatenated in instance order; u is, per
 * instance, its three planes (ux, uy, uz) before the next instance's.  rho_ave of the
 * buoyancy force is each instance's own domain mean.
 * Errors as for the single-lattice calls; LBM_EINVAL names the offending instance. */
typedef struct lbm_batch lbm_batch;
int lbm_batch_create(const lbm_params* common, int n_instances, const int* dims, lbm_batch** out);
/* nodes of instance k (k < 0: of the whole batch) */
long long lbm_batch_nodes(const lbm_batch* b, int instance);
int lbm_batch_init_fields(lbm_batch* b, const float* rho, const float* T, const float* u);
int lbm_batch_step(lbm_batch* b, int n);
/* Time every candidate work plan (tile rows 4 or 8, columns split into 1, 2 or 4 z-chunks, and
 * the TMA mode) over `steps` steps of the current state, keep the fastest, and restore the state exactly
 * (the candidates' steps are undone).  Needs free device memory for one copy of the state.
 * best_ms (nullable) receives the chosen plan's time per step. */
int lbm_batch_autotune(lbm_batch* b, int steps, double* best_ms);
/* the plan in use: tile rows, z-chunks per column, work items, persistent CTAs (each nullable).
 * Tile rows 0 and z-chunks 0: the TMA mode (one TMA-kernel launch per instance, each with its
 * own tile shape and whole-column items, the launches fanned out over 48 streams that fork from
 * and join the batch's stream); items and CTAs are then the totals over the instances. */
int lbm_batch_plan(const lbm_batch* b, int* tile_rows, int* z_split, int* items, int* ctas);
/* Select a plan by its tile rows (4 or 8) and z-chunks per column (1, 2 or 4), or the TMA mode
 * (0, 0); LBM_EINVAL if there is no such plan, LBM_ESTATE if an instance cannot run the TMA
 * kernel.  lbm_batch_autotune times the TMA mode beside the batched-kernel plans. */
int lbm_batch_select_plan(lbm_batch* b, int tile_rows, int z_split);
int lbm_batch_get_moments(lbm_batch* b, float* rho, float* ux, float* uy, float* uz, float* T);
/* sums[2k] = sum of rho, sums[2k+1] = sum of T over instance k (FP64, host pointer) */
int lbm_batch_get_totals(lbm_batch* b, double* sums);
long long lbm_batch_steps_done(const lbm_batch* b);
/* Kernel launches that one step of the current plan enqueues once the state is streamed: 1 for
 * a persistent batched-kernel plan; in the TMA mode one per instance plus one ghost refresh for
 * each instance whose tiles do not write their own ghost cells.  LBM_EINVAL if b is NULL. */
int lbm_batch_launches_per_step(const lbm_batch* b);
void lbm_batch_destroy(lbm_batch* b);

/* Release everything the context owns.  NULL is ignored. */
void lbm_destroy(lbm_ctx* ctx);

/* Static description of a status code. */
const char* lbm_status_str(int status);

/* Message of the last error on this thread (empty string if none). */
const char* lbm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GB300_LBM_H */
