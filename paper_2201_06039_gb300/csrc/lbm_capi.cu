// Host implementation of the C-ABI declared in include/lbm.h.
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include <vector>

#include "../../include/lbm.h"
#include "lbm_host.h"
#include "lbm_launch.h"

using namespace gb300lbm;

namespace {
thread_local char g_err[512] = "";
}  // namespace

namespace gb300lbm {

int fail(int status, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return status;
}

#define CK(call)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));         \
    } while (0)

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

size_t pop_bytes(int precision) { return precision == LBM_FP32 ? 4 : 2; }

}  // namespace gb300lbm

namespace {

struct Layout {
    size_t pops[2], psirho, phis, sums, partial, counter, flag, vel, wall, wpar, wbad, total;
};

// Device memory of a context: two population buffers (rows of 26 or 38 slots: the padded,
// ghost-carrying storage of lbm_device.cuh), dense (psi, rho) and phi_s fields, FP64 sums.
Layout layout_of(const lbm_params* p, const DevParams& dp) {
    Layout L;
    size_t N = (size_t)dp.N, pb = pop_bytes(p->precision), off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    L.pops[0] = take(pop_elems(dp) * pb);
    L.pops[1] = take(pop_elems(dp) * pb);
    L.psirho = take(8 * N);
    L.phis = take(4 * N);
    L.sums = take(8 * sizeof(double));          // slots: [0..1] [2..3] rho_ave ping-pong, [4..5] totals
    L.partial = take(sizeof(double2) * (size_t)max_partials(dp));
    L.counter = take(sizeof(unsigned));
    L.flag = take(sizeof(int));
    L.vel = take(p->divu_mode == 1 ? 16 * N : 0);
    L.wall = take(dp.wet ? 8 * (size_t)dp.nx * dp.ny : 0);
    L.wpar = take(dp.wet && dp.wet_scheme == 1 ? 8 * (size_t)dp.nx * dp.ny : 0);
    L.wbad = take(dp.wet && dp.wet_scheme == 1 ? sizeof(int) : 0);
    L.total = off;
    return L;
}

const int kGraphCache = 8;

struct GraphEntry {
    int n, cur, slot;
    cudaGraphExec_t exec;
    unsigned long long last_use;
};

}  // namespace

struct lbm_ctx {
    lbm_params p;
    DevParams dp;
    cudaStream_t stream;        // caller's stream: every launch and graph replay goes here
    cudaStream_t capture;       // private non-blocking stream used only to record graphs
    cudaStream_t launch;        // stream enqueue_step launches on (== stream, or capture while recording)
    char* base;
    bool owns;
    Layout L;
    int cur, slot;              // population buffer holding the state; rho_ave slot of the next step
    bool fresh_f, fresh_g, first, initialised;
    long long steps;
    int variant;   // LBM_KERNEL_TWO_PASS or LBM_KERNEL_FUSED
    TmaMaps maps;
    int plan_shape, plan_zchunk;   // TMA plan pinned by lbm_select_plan (-1 / 0: automatic)
    GraphEntry graphs[kGraphCache];
    int n_graphs;
    unsigned long long use_clock;

    void* pbuf(int k) { return base + L.pops[k]; }
    double* sums(int k) { return (double*)(base + L.sums) + 2 * k; }
    StateBufs bufs() {
        StateBufs B;
        B.src = pbuf(cur);
        B.dst = pbuf(cur ^ 1);
        B.src_index = cur;
        B.pull_f = fresh_f ? 0 : 1;
        B.pull_g = fresh_g ? 0 : 1;
        B.psirho = (float2*)(base + L.psirho);
        B.phis = (float*)(base + L.phis);
        B.partial = (double2*)(base + L.partial);
        B.counter = (unsigned*)(base + L.counter);
        B.flag = (int*)(base + L.flag);
        B.vel = p.divu_mode == 1 ? (float4*)(base + L.vel) : nullptr;
        return B;
    }
};

namespace gb300lbm {

double critical_T(const lbm_params* p) { return 0.0778 * p->a / (0.45724 * p->b * p->R); }

int validate(const lbm_params* p) {
    if (!p) return fail(LBM_EINVAL, "params is NULL");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail(LBM_EINVAL, "lattice size must be >= 1");
    if (p->thermal_q != 0 && p->thermal_q != 7 && p->thermal_q != 19)
        return fail(LBM_EINVAL, "thermal_q must be 7 (D3Q7) or 19 (D3Q19), not %d", p->thermal_q);
    const int slots = slots_of(p->thermal_q == 19 ? 19 : 7);
    long long Ws = ((long long)p->nx + kGX + 2 + 7) / 8 * 8, Hs = (long long)p->ny + kGY + 2;
    if ((long long)slots * Ws * Hs * p->nz >= (1LL << 31))
        return fail(LBM_EINVAL, "lattice too large (%d x padded nodes must be < 2^31)", slots);
    int n[3] = {p->nx, p->ny, p->nz};
    for (int f = 0; f < 6; ++f) {
        if (p->bc[f] < 0 || p->bc[f] > 3) return fail(LBM_EINVAL, "bc[%d] = %d is not an lbm_bc", f, p->bc[f]);
        if (p->bc[f] == LBM_BC_OUTFLOW && n[f / 2] < 2) return fail(LBM_EINVAL, "outflow face needs >= 2 nodes");
    }
    for (int a = 0; a < 3; ++a) {
        bool plo = p->bc[2 * a] == LBM_BC_PERIODIC || p->bc[2 * a] == LBM_BC_THERMAL_ONLY;
        bool phi = p->bc[2 * a + 1] == LBM_BC_PERIODIC || p->bc[2 * a + 1] == LBM_BC_THERMAL_ONLY;
        if (plo != phi) return fail(LBM_EINVAL, "axis %d: f is periodic on one face only", a);
        if ((p->bc[2 * a] == LBM_BC_PERIODIC) != (p->bc[2 * a + 1] == LBM_BC_PERIODIC))
            return fail(LBM_EINVAL, "axis %d: g is periodic on one face only", a);
    }
    if (!(p->tau_e > 0.5 && p->tau_v > 0.5 && p->tau_q > 0.5 && p->tau_pi > 0.5))
        return fail(LBM_EINVAL, "relaxation times must exceed 1/2");
    if (!(p->varsigma_q > 0.5 && p->varsigma_pi > 0.5)) return fail(LBM_EINVAL, "varsigma_q, varsigma_pi must exceed 1/2");
    if (!(p->a > 0 && p->b > 0 && p->R > 0)) return fail(LBM_EINVAL, "EOS constants a, b, R must be positive");
    if (!(p->d > 0 && p->d < 1)) return fail(LBM_EINVAL, "D3Q7 d must lie in (0, 1)");
    if (!(p->cV > 0)) return fail(LBM_EINVAL, "cV must be positive");
    if (!(p->chi_or_lambda > 0)) return fail(LBM_EINVAL, "chi / lambda must be positive");
    if (p->precision < 0 || p->precision > 2) return fail(LBM_EINVAL, "unknown precision");
    if (p->kernel < 0 || p->kernel > 2) return fail(LBM_EINVAL, "unknown kernel variant");
    if (p->divu_mode < 0 || p->divu_mode > 1) return fail(LBM_EINVAL, "divu_mode must be 0 or 1");
    if (p->wall_scheme != 0 && p->wall_scheme != 1) return fail(LBM_EINVAL, "wall_scheme must be 0 or 1");
    if (p->wall_rho < 0.0 || (p->wall_rho > 0.0 && p->bc[4] != LBM_BC_WALL))
        return fail(LBM_EINVAL, "wall_rho > 0 needs a wall (LBM_BC_WALL) at the -z face");
    if (p->wall_patch_half < 0.0) return fail(LBM_EINVAL, "wall_patch_half must be >= 0");
    if (p->wall_scheme == 0 && p->wall_patch_half > 0.0 && !(p->wall_rho > 0.0 && p->wall_rho_patch > 0.0))
        return fail(LBM_EINVAL, "a wetting patch needs wall_rho > 0 and wall_rho_patch > 0");
    if (p->wall_scheme == 1) {
        if (p->bc[4] != LBM_BC_WALL) return fail(LBM_EINVAL, "wall_scheme 1 needs a wall (LBM_BC_WALL) at the -z face");
        if (p->wall_rho != 0.0 || p->wall_rho_patch != 0.0)
            return fail(LBM_EINVAL, "wall_scheme 1 takes wall_phi / wall_drho, not wall_rho");
        if (!(p->wall_phi > 0.0) || !(p->wall_drho >= 0.0))
            return fail(LBM_EINVAL, "wall_scheme 1 needs wall_phi > 0 and wall_drho >= 0");
        if (p->wall_patch_half > 0.0 && (!(p->wall_phi_patch > 0.0) || !(p->wall_drho_patch >= 0.0)))
            return fail(LBM_EINVAL, "a wetting patch needs wall_phi_patch > 0 and wall_drho_patch >= 0");
    }
    if (p->divu_mode == 1 && p->kernel == LBM_KERNEL_FUSED)
        return fail(LBM_EINVAL, "finite-difference div u runs on the two-pass kernels (kernel AUTO or TWO_PASS)");
    if (p->hot_dT != 0.0 && !(p->hot_sigma > 0)) return fail(LBM_EINVAL, "hot_sigma must be positive");
    if (p->thermal_q == 19) {
        if (p->precision != LBM_FP32) return fail(LBM_EINVAL, "the D3Q19 temperature lattice needs FP32 storage");
        if (p->thermal_bgk) return fail(LBM_EINVAL, "thermal_bgk selects the D3Q7 BGK collision; D3Q19 is BGK already");
        if (p->wall_scheme == 1 || p->wall_rho > 0.0)
            return fail(LBM_EINVAL, "the wetting wall runs with the D3Q7 temperature lattice only");
    }
    return LBM_OK;
}

DevParams make_dev(const lbm_params* p) {
    DevParams d;
    memset(&d, 0, sizeof(d));
    d.nx = p->nx; d.ny = p->ny; d.nz = p->nz;
    d.N = p->nx * p->ny * p->nz;
    d.plane = p->nx * p->ny;
    d.Ws = (p->nx + kGX + 2 + 7) / 8 * 8;   // ghost columns -2..-1 and nx..nx+1; 32-byte aligned rows
    d.Hs = p->ny + kGY + 2;
    const int slots = slots_of(p->thermal_q == 19 ? 19 : 7);
    d.Rs = slots * d.Ws;                    // the slots of a row follow each other
    d.splane = d.Rs * d.Hs;
    d.Ns = d.Ws;
    d.Nidx = d.splane * p->nz - (slots - 1) * d.Ws;
    for (int k = 0; k < 6; ++k) { d.bc[k] = p->bc[k]; d.T_wall[k] = (float)p->T_wall[k]; }
    d.hot_dT = (float)p->hot_dT;
    d.hot_inv2s2 = p->hot_dT != 0.0 ? (float)(1.0 / (2.0 * p->hot_sigma * p->hot_sigma)) : 0.f;
    d.hot_cx = 0.5f * (float)p->nx;
    d.hot_cy = 0.5f * (float)p->ny;
    d.a = (float)p->a; d.b = (float)p->b; d.R = (float)p->R;
    d.Tc = (float)critical_T(p);
    d.inv_Tc = (float)(1.0 / critical_T(p));
    d.inv_N = 1.0 / (double)d.N;
    double w = p->acentric;
    d.kappa = (float)(0.37464 + 1.54226 * w - 0.26992 * w * w);
    d.sigma6 = (float)(6.0 * p->sigma / (p->tau_e - 0.5));
    d.Le = (float)(1.0 / p->tau_e); d.Lv = (float)(1.0 / p->tau_v);
    d.Lq = (float)(1.0 / p->tau_q); d.Lpi = (float)(1.0 / p->tau_pi);
    d.inv_tau_e = (float)(1.0 / p->tau_e);
    d.half_Le = (float)(1.0 - 0.5 / p->tau_e);
    d.cV = (float)p->cV; d.d = (float)p->d; d.csT2 = (float)(p->d / 3.0);
    d.w0 = (float)(1.0 - p->d); d.w1 = (float)(p->d / 6.0);
    d.inv_cV = (float)(1.0 / p->cV); d.inv_csT2 = (float)(3.0 / p->d); d.R_over_cV = (float)(p->R / p->cV);
    d.Gq = (float)(1.0 / p->varsigma_q); d.Gpi = (float)(1.0 / p->varsigma_pi);
    d.lambda_mode = p->lambda_mode; d.chi_or_lambda = (float)p->chi_or_lambda;
    d.gx = (float)p->g[0]; d.gy = (float)p->g[1]; d.gz = (float)p->g[2];
    d.rho_buoy = p->rho_buoy > 0.0 ? (float)p->rho_buoy : 0.f;
    d.flow_off = p->flow_off; d.thermal_off = p->thermal_off;
    d.qt = p->thermal_q == 19 ? 19 : 7;
    d.test_stall = p->test_stall ? 1 : 0;
    d.thermal_bgk = p->thermal_bgk ? 1 : 0;
    d.divu_mode = p->divu_mode;
    d.wet = (p->wall_rho > 0.0 || p->wall_scheme == 1) && p->bc[4] == LBM_BC_WALL ? 1 : 0;
    d.wet_scheme = p->wall_scheme;
    d.wet_phi = (float)p->wall_phi;
    d.wet_drho = (float)p->wall_drho;
    d.wet_phi_p = (float)p->wall_phi_patch;
    d.wet_drho_p = (float)p->wall_drho_patch;
    d.wet_rho = (float)p->wall_rho;
    d.wet_rho_patch = (float)p->wall_rho_patch;
    d.wet_half = p->wall_patch_half > 0.0 ? (float)p->wall_patch_half : 0.f;
    d.wet_cx = 0.5f * (float)p->nx;
    d.wet_cy = 0.5f * (float)p->ny;
    if (p->precision != LBM_FP32) {
        for (int a = 0; a < 19; ++a) {
            int e2 = ex19(a) * ex19(a) + ey19(a) * ey19(a) + ez19(a) * ez19(a);
            double wa = e2 == 0 ? 1.0 / 3.0 : (e2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
            d.shift_f[a] = (float)(wa * p->rho_ref);
        }
        for (int a = 0; a < 7; ++a) d.shift_g[a] = (float)((a == 0 ? 1.0 - p->d : p->d / 6.0) * p->T_ref);
    }
    return d;
}

bool is_device_ptr(const void* ptr) {
    if (!ptr) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace gb300lbm

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Tensor maps of both population buffers for the TMA kernel: dims (Ws, Hs, nz, 26) of FP32,
// boxes (TX + 8, TY + 4, 1, 14) and (TX + 8, TY + 4, 1, 6) of the planned tile shape;
// out-of-range cells read as zero (never used).
bool make_tma_maps(lbm_ctx* c);

void drop_graphs(lbm_ctx* c) {
    for (int k = 0; k < c->n_graphs; ++k) cudaGraphExecDestroy(c->graphs[k].exec);
    c->n_graphs = 0;
}

// Device durations of the kernels of a run of steps: an event pair around each launch, recorded
// as the launches are enqueued (no synchronisation in between, so a launch follows the previous
// one as it would without the events), read after the run.
struct KernelTimer {
    std::vector<cudaEvent_t> ev;   // two per launch
    std::vector<int> kind;         // 0: psi/EOS or fused kernel, 1: stream-collide, 2: ghosts / wall table
    void begin(cudaStream_t s) {
        cudaEvent_t a = nullptr, b = nullptr;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        ev.push_back(a);
        ev.push_back(b);
        cudaEventRecord(a, s);
    }
    void end(int k, cudaStream_t s) {
        cudaEventRecord(ev.back(), s);
        kind.push_back(k);
    }
    // waits for the run, adds each launch's duration to kernel_ms[kind] and counts it
    cudaError_t collect(double* kernel_ms, int* launches) {
        cudaError_t r = ev.empty() ? cudaSuccess : cudaEventSynchronize(ev.back());
        for (size_t i = 0; i < kind.size() && r == cudaSuccess; ++i) {
            float ms = 0.f;
            r = cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
            kernel_ms[kind[i]] += ms;
            launches[kind[i]] += 1;
        }
        return r;
    }
    ~KernelTimer() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
};

// Enqueue one time step of the selected variant on the context's stream (each launch timed when
// a timer is given).
int enqueue_step(lbm_ctx* c, KernelTimer* timer = nullptr) {
    StateBufs B = c->bufs();
    cudaError_t e;
    bool ghosts_done = false;
    if (c->dp.wet && c->dp.wet_scheme == 1) {   // virtual densities of this step from the fluid layer z = 0
        if (timer) timer->begin(c->launch);
        e = launch_wall_table(c->dp, c->p.precision, B.src, B.pull_f, (float2*)(c->base + c->L.wall), c->launch);
        if (e != cudaSuccess) return fail(LBM_ECUDA, "wall table launch: %s", cudaGetErrorString(e));
        if (timer) timer->end(2, c->launch);
    }
    if (c->variant == LBM_KERNEL_FUSED) {
        if (timer) timer->begin(c->launch);
        e = launch_fused(c->dp, c->p.precision, B, c->sums(c->slot), c->sums(c->slot ^ 1), c->first ? 1 : 0,
                         c->launch, c->maps.ok ? &c->maps : nullptr, &ghosts_done);
        if (e != cudaSuccess) return fail(LBM_ECUDA, "fused kernel launch: %s", cudaGetErrorString(e));
        if (c->maps.ok && B.pull_f && B.pull_g) c->dp.test_stall = 0;   // one stalled TMA step only
        if (timer) timer->end(0, c->launch);
    } else {
        if (timer) timer->begin(c->launch);
        e = launch_psi(c->dp, c->p.precision, B, c->sums(c->slot ^ 1), c->launch);
        if (e != cudaSuccess) return fail(LBM_ECUDA, "psi kernel launch: %s", cudaGetErrorString(e));
        if (timer) {
            timer->end(0, c->launch);
            timer->begin(c->launch);
        }
        if (B.vel) {   // u of every node for the finite-difference div u of the collide pass
            e = launch_velocity(c->dp, c->p.precision, B, c->sums(c->slot), c->launch);
            if (e != cudaSuccess) return fail(LBM_ECUDA, "velocity kernel launch: %s", cudaGetErrorString(e));
        }
        e = launch_collide(c->dp, c->p.precision, B, c->sums(c->slot), c->first ? 1 : 0, c->launch);
        if (e != cudaSuccess) return fail(LBM_ECUDA, "collide kernel launch: %s", cudaGetErrorString(e));
        if (timer) timer->end(1, c->launch);
    }
    // both fields are written every step (frozen ones copied through unchanged, so they stay
    // in their un-streamed "fresh" form)
    c->cur ^= 1;
    if (c->maps.ok && !ghosts_done) {   // the TMA path reads ghost cells: refresh them in the state just written
        if (timer) timer->begin(c->launch);
        e = launch_ghosts(c->dp, c->p.precision, B.dst, c->launch);
        if (e != cudaSuccess) return fail(LBM_ECUDA, "ghost refresh launch: %s", cudaGetErrorString(e));
        if (timer) timer->end(2, c->launch);
    }
    if (!c->p.flow_off) c->fresh_f = false;
    if (!c->p.thermal_off) c->fresh_g = false;
    c->slot ^= 1;
    c->first = false;
    c->steps += 1;
    return LBM_OK;
}

int run_graph(lbm_ctx* c, int n) {
    GraphEntry* hit = nullptr;
    for (int k = 0; k < c->n_graphs; ++k) {
        GraphEntry& g = c->graphs[k];
        if (g.n == n && g.cur == c->cur && g.slot == c->slot) hit = &g;
    }
    if (!hit) {
        int c0 = c->cur, s0 = c->slot;
        bool ff = c->fresh_f, fg = c->fresh_g, fi = c->first;
        long long st = c->steps;
        cudaGraph_t graph;
        // record on a private stream (the legacy default stream cannot be captured); the
        // graph is then replayed on the caller's stream
        if (!c->capture) CK(cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking));
        CK(cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal));
        c->launch = c->capture;
        int rc = LBM_OK;
        for (int k = 0; k < n && rc == LBM_OK; ++k) rc = enqueue_step(c);
        cudaError_t e = cudaStreamEndCapture(c->capture, &graph);
        c->launch = c->stream;
        // the capture only recorded work: put the state back, the replay advances it
        c->cur = c0; c->slot = s0; c->fresh_f = ff; c->fresh_g = fg; c->first = fi; c->steps = st;
        if (rc != LBM_OK) { if (e == cudaSuccess) cudaGraphDestroy(graph); return rc; }
        if (e != cudaSuccess) return fail(LBM_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        cudaGraphExec_t exec;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(LBM_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        if (c->n_graphs == kGraphCache) {
            int lru = 0;
            for (int k = 1; k < c->n_graphs; ++k)
                if (c->graphs[k].last_use < c->graphs[lru].last_use) lru = k;
            cudaGraphExecDestroy(c->graphs[lru].exec);
            c->graphs[lru] = c->graphs[--c->n_graphs];
        }
        GraphEntry& g = c->graphs[c->n_graphs++];
        g.n = n; g.cur = c->cur; g.slot = c->slot; g.exec = exec;
        hit = &g;
    }
    hit->last_use = ++c->use_clock;
    CK(cudaGraphLaunch(hit->exec, c->stream));
    // advance the host-side state exactly as n enqueue_step calls would
    for (int k = 0; k < n; ++k) {
        c->cur ^= 1;
        c->slot ^= 1;
    }
    c->steps += n;
    return LBM_OK;
}

int check_flag(lbm_ctx* c) {
    int h = 0;
    CK(cudaMemcpyAsync(&h, c->base + c->L.flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (h) {
        CK(cudaMemsetAsync(c->base + c->L.flag, 0, sizeof(int), c->stream));
        if (h & 4) return fail(LBM_EBOUNDS, "a kernel index fell outside its buffer (bounds-checked build, step %lld)",
                               c->steps);
        if (h & 2) return fail(LBM_ETIMEOUT, "a bounded pipeline wait in the fused kernel gave up (step %lld)", c->steps);
        return fail(LBM_ENONFINITE, "non-finite rho/T/psi or psi^2 <= 0 after step %lld", c->steps);
    }
    return LBM_OK;
}

}  // namespace

bool gb300lbm::build_tma_maps(const DevParams& d, int precision, void* buf0, void* buf1, int model_ctas,
                              int forced_shape, int forced_zchunk, int max_items, TmaMaps* maps) {
    maps->ok = false;
    if (!tma_eligible(d, precision)) return false;
    int dev = 0, sms = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
    int shape = -1, zchunk = 0, items = 0;
    tma_plan_for(d, model_ctas > 0 ? model_ctas : sms, forced_shape, forced_zchunk, &shape, &zchunk, &items);
    if (shape < 0 || (size_t)optin < tma_smem_bytes(shape, precision)) return false;
    if (items > max_items) return false;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return false;
    }
    EncodeTiledFn encode = (EncodeTiledFn)fn;
    cuuint64_t dims[4] = {(cuuint64_t)d.Ws, (cuuint64_t)d.Hs, (cuuint64_t)d.nz, (cuuint64_t)kSlots};
    const cuuint64_t E = (cuuint64_t)pop_bytes(precision);
    const CUtensorMapDataType dt = precision == LBM_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : precision == LBM_BF16_SHIFTED ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                                      : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    cuuint64_t strides[3] = {(cuuint64_t)d.Rs * E, (cuuint64_t)d.splane * E, (cuuint64_t)d.Ns * E};
    const cuuint32_t bw = (cuuint32_t)tma_box_w(shape, precision), bh = (cuuint32_t)tma_box_h(shape);
    cuuint32_t box14[4] = {bw, bh, 1, 14}, box6[4] = {bw, bh, 1, 6}, es[4] = {1, 1, 1, 1};
    // output tiles, dimensions ordered (x, slot, y, z) to match the [row][slot][x] out buffer; the
    // tensor spans the real nodes only (x < nx, y < ny in storage coordinates + the offsets), and
    // the last tile row gets a box of exactly its rows, so no box ever extends past ny
    const int th = tma_tile_h(shape), ry = d.ny - th * ((d.ny - 1) / th);
    cuuint64_t dims_out[4] = {(cuuint64_t)(d.nx + kGX), (cuuint64_t)kSlots, (cuuint64_t)(d.ny + kGY), (cuuint64_t)d.nz};
    cuuint64_t strides_out[3] = {(cuuint64_t)d.Ns * E, (cuuint64_t)d.Rs * E, (cuuint64_t)d.splane * E};
    cuuint32_t box_out[4] = {(cuuint32_t)tma_tile_w(shape), (cuuint32_t)kSlots, (cuuint32_t)th, 1};
    cuuint32_t box_top[4] = {(cuuint32_t)tma_tile_w(shape), (cuuint32_t)kSlots, (cuuint32_t)ry, 1};
    // ghost boxes over the whole padded plane (they always lie inside it)
    const int tw = tma_tile_w(shape), rx = d.nx - tw * ((d.nx - 1) / tw);
    cuuint64_t dims_pad[4] = {(cuuint64_t)d.Ws, (cuuint64_t)kSlots, (cuuint64_t)d.Hs, (cuuint64_t)d.nz};
    const cuuint32_t gw = (cuuint32_t)tma_ghost_cols(precision);
    cuuint32_t box_gcol[4] = {gw, (cuuint32_t)kSlots, (cuuint32_t)th, 1};
    cuuint32_t box_gcol_top[4] = {gw, (cuuint32_t)kSlots, (cuuint32_t)ry, 1};
    cuuint32_t box_grow[4] = {(cuuint32_t)tw, (cuuint32_t)kSlots, 2, 1};
    cuuint32_t box_grow_right[4] = {(cuuint32_t)rx, (cuuint32_t)kSlots, 2, 1};
    cuuint32_t box_gcor[4] = {gw, (cuuint32_t)kSlots, 2, 1};
    maps->ghosts = tma_ghost_mode(d, shape, precision);
    for (int k = 0; k < 2; ++k) {
        void* g = k == 0 ? buf0 : buf1;
        if (encode(&maps->m14[k], dt, 4, g, dims, strides, box14, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
        if (encode(&maps->m6[k], dt, 4, g, dims, strides, box6, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
        if (encode(&maps->mout[k], dt, 4, g, dims_out, strides_out, box_out, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
        if (encode(&maps->mout_top[k], dt, 4, g, dims_out, strides_out, box_top, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
        if (maps->ghosts == 1) {
            CUtensorMap* gm[5] = {&maps->mgcol[k], &maps->mgcol_top[k], &maps->mgrow[k], &maps->mgrow_right[k],
                                  &maps->mgcor[k]};
            cuuint32_t* gb[5] = {box_gcol, box_gcol_top, box_grow, box_grow_right, box_gcor};
            for (int q = 0; q < 5; ++q)
                if (encode(gm[q], dt, 4, g, dims_pad, strides_out, gb[q], es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                    maps->ghosts = precision == 0 ? 2 : 0;
        }
    }
    maps->sms = sms;
    maps->shape = shape;
    maps->zchunk = zchunk;
    maps->items = items;
    maps->ok = true;
    return true;
}

namespace {

bool make_tma_maps(lbm_ctx* c) {
    return build_tma_maps(c->dp, c->p.precision, c->pbuf(0), c->pbuf(1), 0, c->plan_shape, c->plan_zchunk,
                          max_partials(c->dp), &c->maps);
}

}  // namespace

extern "C" {

void lbm_params_default(lbm_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->nx = p->ny = p->nz = 1;
    p->a = 2.0 / 49.0; p->b = 2.0 / 21.0; p->R = 1.0; p->acentric = 0.344;
    p->tau_e = 1.25; p->tau_v = 0.8; p->tau_q = 1.0; p->tau_pi = 1.0;
    p->cV = 5.0; p->d = 0.95; p->varsigma_q = 1.0; p->varsigma_pi = 1.0;
    p->lambda_mode = 0; p->chi_or_lambda = 0.08;
    p->precision = LBM_FP32;
    p->kernel = LBM_KERNEL_AUTO;
    p->use_graph = 1;
    p->use_tma = 1;
    p->check_nonfinite = 1;
}

int lbm_eos_critical(const lbm_params* p, double* Tc, double* pc) {
    if (!p || !(p->a > 0 && p->b > 0 && p->R > 0)) return fail(LBM_EINVAL, "EOS constants must be positive");
    double t = critical_T(p);
    if (Tc) *Tc = t;
    if (pc) *pc = 0.0778 * p->R * t / p->b;
    return LBM_OK;
}

size_t lbm_workspace_bytes(const lbm_params* p) {
    if (validate(p) != LBM_OK) return 0;
    DevParams d = make_dev(p);
    return layout_of(p, d).total;
}

int lbm_create(const lbm_params* p, lbm_ctx** out) {
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate(p);
    if (rc) return rc;
    lbm_ctx* c = (lbm_ctx*)calloc(1, sizeof(lbm_ctx));
    if (!c) return fail(LBM_ENOMEM, "host allocation failed");
    c->p = *p;
    c->dp = make_dev(p);
    c->L = layout_of(p, c->dp);
    c->stream = (cudaStream_t)p->cuda_stream;
    c->launch = c->stream;
    c->capture = nullptr;
    if (p->workspace) {
        if (p->workspace_bytes < c->L.total || ((uintptr_t)p->workspace & 255)) {
            free(c);
            return fail(LBM_EINVAL, "workspace too small (%zu < %zu) or not 256-byte aligned", p->workspace_bytes,
                        c->L.total);
        }
        c->base = (char*)p->workspace;
        c->owns = false;
    } else {
        cudaError_t e = cudaMalloc((void**)&c->base, c->L.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            free(c);
            return fail(LBM_ENOMEM, "cudaMalloc(%zu): %s", c->L.total, cudaGetErrorString(e));
        }
        c->owns = true;
    }
    c->variant = p->kernel == LBM_KERNEL_AUTO
                     ? (fused_supported(c->dp) && p->divu_mode == 0 ? LBM_KERNEL_FUSED : LBM_KERNEL_TWO_PASS)
                     : p->kernel;
    if (c->variant == LBM_KERNEL_FUSED && !fused_supported(c->dp)) {
        if (c->owns) cudaFree(c->base);
        free(c);
        return fail(LBM_EINVAL, "fused kernel does not support this lattice");
    }
    c->plan_shape = -1;
    c->plan_zchunk = 0;
    c->dp.check_flag = (int*)(c->base + c->L.flag);
    if (c->variant == LBM_KERNEL_FUSED && p->use_tma != 0) make_tma_maps(c);
    cudaError_t e = cudaMemsetAsync(c->base + c->L.sums, 0, c->L.flag + sizeof(int) - c->L.sums, c->stream);
    if (e == cudaSuccess && c->dp.wet) {   // scheme 0: the table is constant; scheme 1: refreshed every step
        c->dp.wall_tab = (const float2*)(c->base + c->L.wall);
        if (c->dp.wet_scheme == 0) {
            e = launch_wall_table(c->dp, c->p.precision, nullptr, 0, (float2*)(c->base + c->L.wall), c->stream);
        } else {   // the wettability map starts from the rest / patch parameters
            c->dp.wall_par = (const float2*)(c->base + c->L.wpar);
            e = launch_wall_params(c->dp, (float2*)(c->base + c->L.wpar), c->stream);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        if (c->owns) cudaFree(c->base);
        free(c);
        return fail(LBM_ECUDA, "initial memset: %s", cudaGetErrorString(e));
    }
    *out = c;
    return LBM_OK;
}

int lbm_init_fields(lbm_ctx* c, const float* rho, const float* T, const float* u) {
    NvtxRange range("lbm_init_fields");
    if (!c) return fail(LBM_EINVAL, "ctx is NULL");
    if (!rho || !T) return fail(LBM_EINVAL, "rho and T are required");
    size_t N = (size_t)c->dp.N;
    // stage host inputs in the second population buffer (>= 26 N elements of >= 2 bytes >= 5 N floats)
    float* stage = (float*)c->pbuf(1);
    const float *drho = rho, *dT = T, *du = u;
    if (!is_device_ptr(rho)) {
        CK(cudaMemcpyAsync(stage, rho, N * 4, cudaMemcpyHostToDevice, c->stream));
        drho = stage;
    }
    if (!is_device_ptr(T)) {
        CK(cudaMemcpyAsync(stage + N, T, N * 4, cudaMemcpyHostToDevice, c->stream));
        dT = stage + N;
    }
    if (u && !is_device_ptr(u)) {
        CK(cudaMemcpyAsync(stage + 2 * N, u, 3 * N * 4, cudaMemcpyHostToDevice, c->stream));
        du = stage + 2 * N;
    }
    drop_graphs(c);
    c->cur = 0;
    c->slot = 0;
    CK(launch_init(c->dp, c->p.precision, c->pbuf(0), drho, dT, du, c->stream));
    if (c->maps.ok) CK(launch_ghosts(c->dp, c->p.precision, c->pbuf(0), c->stream));
    StateBufs B = c->bufs();
    CK(launch_sum_field(drho, c->dp.N, B.partial, B.counter, c->sums(0), c->stream));
    CK(cudaMemsetAsync(c->base + c->L.flag, 0, sizeof(int), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->fresh_f = c->fresh_g = true;
    c->first = true;
    c->initialised = true;
    c->steps = 0;
    return LBM_OK;
}

int lbm_step(lbm_ctx* c, int n) {
    NvtxRange range("lbm_step");
    if (!c) return fail(LBM_EINVAL, "ctx is NULL");
    if (!c->initialised) return fail(LBM_ESTATE, "lbm_step before lbm_init_fields");
    if (n < 0) return fail(LBM_EINVAL, "n < 0");
    int rc = LBM_OK;
    int k = 0;
    // the first step after init reads the un-streamed state and has no phi_s history
    while (k < n && (c->first || (c->fresh_f && !c->p.flow_off) || (c->fresh_g && !c->p.thermal_off))) {
        rc = enqueue_step(c);
        if (rc) return rc;
        ++k;
    }
    if (k < n) {
        if (c->p.use_graph && !c->dp.test_stall) rc = run_graph(c, n - k);   // never capture a stall
        else
            for (; k < n && rc == LBM_OK; ++k) rc = enqueue_step(c);
        if (rc) return rc;
    }
    if (c->p.check_nonfinite) return check_flag(c);
    return LBM_OK;
}

int lbm_step_profiled(lbm_ctx* c, int n, double kernel_ms[3], int launches[3]) {
    if (!c || !kernel_ms || !launches) return fail(LBM_EINVAL, "NULL argument");
    if (!c->initialised) return fail(LBM_ESTATE, "lbm_step before lbm_init_fields");
    for (int k = 0; k < 3; ++k) { kernel_ms[k] = 0.0; launches[k] = 0; }
    int rc = LBM_OK;
    {
        KernelTimer timer;
        for (int k = 0; k < n && rc == LBM_OK; ++k) rc = enqueue_step(c, &timer);
        cudaError_t e = timer.collect(kernel_ms, launches);
        if (rc == LBM_OK && e != cudaSuccess) rc = fail(LBM_ECUDA, "kernel timing: %s", cudaGetErrorString(e));
    }
    if (rc) return rc;
    if (c->p.check_nonfinite) return check_flag(c);
    return LBM_OK;
}

int lbm_get_moments(lbm_ctx* c, float* rho, float* ux, float* uy, float* uz, float* T) {
    NvtxRange range("lbm_get_moments");
    if (!c) return fail(LBM_EINVAL, "ctx is NULL");
    if (!c->initialised) return fail(LBM_ESTATE, "lbm_get_moments before lbm_init_fields");
    size_t N = (size_t)c->dp.N;
    StateBufs B = c->bufs();
    // u carries F_m / 2: a scheme-1 wetting wall's virtual densities must be those of this state
    if (c->dp.wet && c->dp.wet_scheme == 1)
        CK(launch_wall_table(c->dp, c->p.precision, B.src, B.pull_f, (float2*)(c->base + c->L.wall), c->stream));
    CK(launch_psi(c->dp, c->p.precision, B, nullptr, c->stream));
    // outputs staged in the population buffer the next step overwrites anyway
    float* stage = (float*)c->pbuf(c->cur ^ 1);
    float* outs[5] = {rho, ux, uy, uz, T};
    float* dst[5];
    for (int k = 0; k < 5; ++k) dst[k] = outs[k] ? (is_device_ptr(outs[k]) ? outs[k] : stage + k * N) : nullptr;
    CK(launch_moments(c->dp, c->p.precision, B, c->sums(c->slot), dst[0], dst[1], dst[2], dst[3], dst[4], c->stream));
    for (int k = 0; k < 5; ++k)
        if (outs[k] && dst[k] != outs[k])
            CK(cudaMemcpyAsync(outs[k], dst[k], N * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_get_totals(lbm_ctx* c, double* mass, double* T_sum, double* rho_ave) {
    if (!c) return fail(LBM_EINVAL, "ctx is NULL");
    if (!c->initialised) return fail(LBM_ESTATE, "lbm_get_totals before lbm_init_fields");
    StateBufs B = c->bufs();
    CK(launch_psi(c->dp, c->p.precision, B, c->sums(2), c->stream));
    double h[6];
    CK(cudaMemcpyAsync(h, c->sums(0), sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (mass) *mass = h[4];
    if (T_sum) *T_sum = h[5];
    if (rho_ave) *rho_ave = h[2 * c->slot] / (double)c->dp.N;
    return LBM_OK;
}

long long lbm_steps_done(const lbm_ctx* c) { return c ? c->steps : 0; }

// Checkpoint layout: a fixed header, the current population buffer (its device layout: rows of
// slots, ghost cells included), the phi_s history (N floats), the two sums of the next step's rho_ave.
namespace {
struct CkptHeader {
    char magic[8];
    int version, nx, ny, nz, precision, fresh_f, fresh_g, first;
    long long steps, pop_bytes, phis_bytes;
};
const char kCkptMagic[8] = {'G', 'B', '3', 'L', 'B', 'M', 'C', 'K'};
size_t ckpt_pop_bytes(const lbm_ctx* c) { return pop_elems(c->dp) * pop_bytes(c->p.precision); }
}  // namespace

size_t lbm_state_bytes(const lbm_ctx* c) {
    if (!c) return 0;
    return sizeof(CkptHeader) + ckpt_pop_bytes(c) + 4 * (size_t)c->dp.N + 2 * sizeof(double);
}

int lbm_save_state(lbm_ctx* c, void* buf, size_t bytes) {
    if (!c || !buf) return fail(LBM_EINVAL, "ctx and buf are required");
    if (!c->initialised) return fail(LBM_ESTATE, "lbm_save_state before lbm_init_fields");
    if (bytes < lbm_state_bytes(c)) return fail(LBM_EINVAL, "buffer of %zu bytes, %zu needed", bytes, lbm_state_bytes(c));
    CkptHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kCkptMagic, 8);
    h.version = 2;   // 2: rows of slots
    h.nx = c->p.nx; h.ny = c->p.ny; h.nz = c->p.nz; h.precision = c->p.precision;
    h.fresh_f = c->fresh_f; h.fresh_g = c->fresh_g; h.first = c->first;
    h.steps = c->steps;
    h.pop_bytes = (long long)ckpt_pop_bytes(c);
    h.phis_bytes = 4LL * c->dp.N;
    char* out = (char*)buf;
    memcpy(out, &h, sizeof(h));
    out += sizeof(h);
    CK(cudaMemcpyAsync(out, c->pbuf(c->cur), (size_t)h.pop_bytes, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(out + h.pop_bytes, c->base + c->L.phis, (size_t)h.phis_bytes, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(out + h.pop_bytes + h.phis_bytes, c->sums(c->slot), 2 * sizeof(double), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_set_wall_map(lbm_ctx* c, const float* phi, const float* drho) {
    if (!c || !phi || !drho) return fail(LBM_EINVAL, "ctx, phi and drho are required");
    if (!(c->dp.wet && c->dp.wet_scheme == 1)) return fail(LBM_ESTATE, "the context has no scheme-1 wetting wall");
    const size_t M = (size_t)c->dp.nx * c->dp.ny;
    // host inputs staged in the population buffer the next step overwrites anyway
    float* stage = (float*)c->pbuf(c->cur ^ 1);
    const float* dphi = phi;
    const float* ddrho = drho;
    if (!is_device_ptr(phi)) {
        CK(cudaMemcpyAsync(stage, phi, M * 4, cudaMemcpyHostToDevice, c->stream));
        dphi = stage;
    }
    if (!is_device_ptr(drho)) {
        CK(cudaMemcpyAsync(stage + M, drho, M * 4, cudaMemcpyHostToDevice, c->stream));
        ddrho = stage + M;
    }
    int* bad = (int*)(c->base + c->L.wbad);
    int h = 0;
    CK(cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
    CK(launch_wall_map(c->dp, dphi, ddrho, nullptr, bad, 0, c->stream));   // check every value first
    CK(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (h) return fail(LBM_EINVAL, "wall map: every phi must be > 0 and every drho >= 0 (finite)");
    CK(launch_wall_map(c->dp, dphi, ddrho, (float2*)(c->base + c->L.wpar), bad, 1, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_load_state(lbm_ctx* c, const void* buf, size_t bytes) {
    if (!c || !buf) return fail(LBM_EINVAL, "ctx and buf are required");
    if (bytes < sizeof(CkptHeader)) return fail(LBM_EINVAL, "not a checkpoint (%zu bytes)", bytes);
    CkptHeader h;
    memcpy(&h, buf, sizeof(h));
    if (memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != 2) return fail(LBM_EINVAL, "not a checkpoint of this layout");
    if (h.nx != c->p.nx || h.ny != c->p.ny || h.nz != c->p.nz || h.precision != c->p.precision)
        return fail(LBM_EINVAL, "checkpoint of a %d x %d x %d lattice (precision %d), context is %d x %d x %d (%d)",
                    h.nx, h.ny, h.nz, h.precision, c->p.nx, c->p.ny, c->p.nz, c->p.precision);
    if (bytes < lbm_state_bytes(c) || h.pop_bytes != (long long)ckpt_pop_bytes(c) || h.phis_bytes != 4LL * c->dp.N)
        return fail(LBM_EINVAL, "checkpoint is truncated or of another layout");
    const char* in = (const char*)buf + sizeof(h);
    CK(cudaMemcpyAsync(c->pbuf(c->cur), in, (size_t)h.pop_bytes, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->base + c->L.phis, in + h.pop_bytes, (size_t)h.phis_bytes, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->sums(c->slot), in + h.pop_bytes + h.phis_bytes, 2 * sizeof(double), cudaMemcpyHostToDevice,
                       c->stream));
    // the saving context may not have kept the ghost cells (kernels without TMA do not use them)
    if (c->maps.ok && !h.fresh_f && !h.fresh_g) CK(launch_ghosts(c->dp, c->p.precision, c->pbuf(c->cur), c->stream));
    CK(cudaMemsetAsync(c->base + c->L.flag, 0, sizeof(int), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->fresh_f = h.fresh_f != 0;
    c->fresh_g = h.fresh_g != 0;
    c->first = h.first != 0;
    c->steps = h.steps;
    c->initialised = true;
    return LBM_OK;
}

int lbm_plan_shapes(int* tile_w, int* tile_h, int max) {
    const int n = tma_num_shapes();
    for (int k = 0; k < n && k < max; ++k) {
        if (tile_w) tile_w[k] = tma_tile_w(k);
        if (tile_h) tile_h[k] = tma_tile_h(k);
    }
    return n;
}

int lbm_get_plan(const lbm_ctx* c, int* shape, int* zchunk, int* items, int* ctas) {
    if (!c) return fail(LBM_EINVAL, "ctx is NULL");
    const bool ok = c->maps.ok;
    if (shape) *shape = ok ? c->maps.shape : -1;
    if (zchunk) *zchunk = ok ? c->maps.zchunk : 0;
    if (items) *items = ok ? c->maps.items : 0;
    if (ctas) *ctas = ok ? (c->maps.sms < c->maps.items ? c->maps.sms : c->maps.items) : 0;
    return LBM_OK;
}

int lbm_select_plan(lbm_ctx* c, int shape, int zchunk) {
    if (!c) return fail(LBM_EINVAL, "ctx is NULL");
    if (shape < -1 || shape >= tma_num_shapes() || zchunk < 0)
        return fail(LBM_EINVAL, "no tile shape %d (0..%d, -1 automatic) or z-chunk %d < 0", shape,
                    tma_num_shapes() - 1, zchunk);
    if (c->variant != LBM_KERNEL_FUSED || c->p.use_tma == 0 || !tma_eligible(c->dp, c->p.precision))
        return fail(LBM_ESTATE, "the context does not run the TMA kernel");
    const int s0 = c->plan_shape, z0 = c->plan_zchunk;
    c->plan_shape = shape;
    c->plan_zchunk = zchunk;
    drop_graphs(c);   // the graphs captured the old plan's launches
    if (!make_tma_maps(c)) {
        c->plan_shape = s0;
        c->plan_zchunk = z0;
        make_tma_maps(c);
        return fail(LBM_EINVAL, "plan (shape %d, z-chunk %d) does not fit this lattice and GPU", shape, zchunk);
    }
    return LBM_OK;
}

int lbm_autotune(lbm_ctx* c, int steps, double* best_ms) {
    NvtxRange range("lbm_autotune");
    if (!c) return fail(LBM_EINVAL, "ctx is NULL");
    if (!c->initialised) return fail(LBM_ESTATE, "lbm_autotune before lbm_init_fields");
    if (steps < 1) return fail(LBM_EINVAL, "steps must be >= 1");
    if (c->variant != LBM_KERNEL_FUSED || c->p.use_tma == 0 || !c->maps.ok)
        return fail(LBM_ESTATE, "the context does not run the TMA kernel");
    // the first step after lbm_init_fields runs the generic kernel: take it before timing
    int rc = LBM_OK;
    while (rc == LBM_OK && (c->first || c->fresh_f || c->fresh_g)) rc = enqueue_step(c);
    if (rc) return rc;
    const size_t popb = pop_elems(c->dp) * pop_bytes(c->p.precision), phib = 4 * (size_t)c->dp.N;
    const size_t sumb = 8 * sizeof(double);
    char* save = nullptr;
    cudaError_t e = cudaMalloc((void**)&save, popb + phib + sumb);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ENOMEM, "autotune state copy: %s", cudaGetErrorString(e));
    }
    const int c0 = c->cur, sl0 = c->slot;
    const long long st0 = c->steps;
    const int s_keep = c->plan_shape, z_keep = c->plan_zchunk;
    auto save_or_restore = [&](bool restore) -> cudaError_t {
        char* a[3] = {(char*)c->pbuf(c0), c->base + c->L.phis, c->base + c->L.sums};
        char* b[3] = {save, save + popb, save + popb + phib};
        size_t n[3] = {popb, phib, sumb};
        for (int k = 0; k < 3; ++k) {
            cudaError_t r = cudaMemcpyAsync(restore ? a[k] : b[k], restore ? b[k] : a[k], n[k],
                                            cudaMemcpyDeviceToDevice, c->stream);
            if (r != cudaSuccess) return r;
        }
        return cudaSuccess;
    };
    cudaEvent_t ev[2];
    cudaEventCreate(&ev[0]);
    cudaEventCreate(&ev[1]);
    int sms = c->maps.sms;
    float best_t = -1.f;
    int best_shape = -1, best_zc = 0;
    e = save_or_restore(false);
    if (e != cudaSuccess) rc = fail(LBM_ECUDA, "autotune save: %s", cudaGetErrorString(e));
    // candidates: every tile shape with its three best modelled z-chunks and the whole column
    for (int sh = 0; sh < tma_num_shapes() && rc == LBM_OK; ++sh) {
        int zcs[4];
        int nz = tma_zchunk_candidates(c->dp, sms, sh, zcs, 3);
        bool whole = false;
        for (int q = 0; q < nz; ++q) whole |= zcs[q] == c->dp.nz;
        if (!whole) zcs[nz++] = c->dp.nz;
        for (int q = 0; q < nz && rc == LBM_OK; ++q) {
            c->plan_shape = sh;
            c->plan_zchunk = zcs[q];
            drop_graphs(c);
            if (!make_tma_maps(c)) continue;   // does not fit this GPU
            rc = enqueue_step(c);   // warm-up
            cudaEventRecord(ev[0], c->stream);
            for (int k = 0; k < steps && rc == LBM_OK; ++k) rc = enqueue_step(c);
            cudaEventRecord(ev[1], c->stream);
            if (cudaEventSynchronize(ev[1]) != cudaSuccess) rc = fail(LBM_ECUDA, "autotune timing failed");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[0], ev[1]);
            if (rc == LBM_OK && (best_t < 0.f || ms < best_t)) {
                best_t = ms;
                best_shape = sh;
                best_zc = zcs[q];
            }
            e = save_or_restore(true);
            if (e != cudaSuccess && rc == LBM_OK) rc = fail(LBM_ECUDA, "autotune restore: %s", cudaGetErrorString(e));
            c->cur = c0;
            c->slot = sl0;
            c->steps = st0;
        }
    }
    cudaStreamSynchronize(c->stream);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    cudaFree(save);
    c->plan_shape = rc == LBM_OK && best_shape >= 0 ? best_shape : s_keep;
    c->plan_zchunk = rc == LBM_OK && best_shape >= 0 ? best_zc : z_keep;
    drop_graphs(c);
    make_tma_maps(c);
    if (rc == LBM_OK) {
        CK(cudaMemsetAsync(c->base + c->L.flag, 0, sizeof(int), c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if (best_ms) *best_ms = best_t / steps;
    }
    return rc;
}

int lbm_kernel_in_use(const lbm_ctx* c) {
    if (!c) return LBM_EINVAL;
    if (c->variant == LBM_KERNEL_FUSED && c->maps.ok) return LBM_KERNEL_FUSED_TMA;
    return c->variant;
}

void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    drop_graphs(c);
    if (c->capture) cudaStreamDestroy(c->capture);
    if (c->owns && c->base) cudaFree(c->base);
    free(c);
}

const char* lbm_status_str(int s) {
    switch (s) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "out of memory";
    case LBM_ECUDA: return "CUDA error";
    case LBM_ESTATE: return "call out of order";
    case LBM_ENONFINITE: return "non-finite value in the lattice";
    case LBM_ETIMEOUT: return "device wait timed out";
    case LBM_EBOUNDS: return "kernel index out of bounds";
    }
    return "unknown status";
}

const char* lbm_last_error(void) { return g_err; }

// error message hook for the library's other translation units (not exported)
__attribute__((visibility("hidden"))) void gb300lbm_set_error(const char* msg) {
    snprintf(g_err, sizeof(g_err), "%s", msg);
}

}  // extern "C"
