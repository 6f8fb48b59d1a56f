// Batched ensemble C-ABI (lbm_batch_*, declared in include/lbm.h): many independent lattices
// of uneven sizes advanced by one persistent kernel launch per time step.
//
// Device memory of a batch (one allocation):
//   pops[2]   population buffers; instance k owns its block at pop_off_k (the padded rows-of-
//             slots layout of a single lattice, so the per-instance set-up and read-out kernels
//             run unchanged on the instance's block)
//   phis      phi_s history, instances concatenated (node offset field_off_k)
//   psirho    (psi, rho) scratch of the largest instance (read-out only)
//   sums      (sum rho, sum T) per instance: two ping-pong sets (rho_ave of the next step) and
//             one set for lbm_batch_get_totals
//   partial   one double2 per work item (and per block of the read-out reductions)
//   counters  work counter + ticket of the batched kernel, ticket of the read-out reductions
//   flag      non-finite / timeout flag
//   insts     BatchInst table, items: BatchItem table of the current plan
//
// Plan: tile rows (4 or 8 of the 32-wide tile) and the number of z-chunks per column.  Items of
// one instance are contiguous; instances are ordered by size, largest first, so that the atomic
// work counter hands out the longest items first.  lbm_batch_autotune times every candidate plan
// on the current state (which it restores afterwards) and keeps the fastest.
//
// TMA mode (the last plan, tile rows 0): every instance runs the single-lattice TMA kernel on its
// own block (its own tensor maps, tile shape and whole-column items, partial-sum range and
// reduction counter), one launch per instance, fanned out over kSide streams that fork from and
// join the batch's stream, so that the launches of many instances share the GPU.  Instances whose
// tiles cannot write their periodic ghost cells get the ghost refresh kernel after their launch.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_host.h"
#include "lbm_launch.h"

using namespace gb300lbm;

namespace {

struct Plan {
    int ty, zsplit;
};
const Plan kPlans[] = {{8, 1}, {8, 2}, {4, 1}, {4, 2}, {8, 4}, {4, 4}};
const int kNumPlans = (int)(sizeof(kPlans) / sizeof(kPlans[0]));   // persistent batched-kernel plans
const int kTmaPlan = kNumPlans;                                     // TMA mode
const int kSide = 48;   // side streams of the TMA mode (16: 14.4k, 32: 15.3k, 48: 15.5k, 64: 14.8k MLUPS)
const int kTmaChain = 8;                                            // steps of one TMA-mode graph (even)

struct BatchGraph {
    int n, cur, slot, plan;
    bool ghosts_valid;
    cudaGraphExec_t exec;
};
const int kBatchGraphs = 4;

}  // namespace

struct lbm_batch {
    lbm_params p;                      // common parameters (nx, ny, nz: those of instance 0)
    int n;                             // instances
    std::vector<DevParams> dps;        // per-instance device constants
    std::vector<BatchInst> inst;       // host copy of the instance table
    std::vector<int> order;            // instances by size, largest first
    long long nodes;                   // total nodes
    long long pop_elems;               // elements of one population buffer
    int max_N, max_items, max_partial;
    cudaStream_t stream, capture, launch;
    char* base;
    size_t off_pops[2], off_phis, off_psirho, off_sums, off_partial, off_counters, off_flag, off_inst, off_items;
    int plan, n_items, ctas, sms;
    int cur, slot;
    bool fresh_f, fresh_g, first, initialised;
    long long steps;
    BatchGraph graphs[kBatchGraphs];
    int n_graphs;
    // TMA mode
    std::vector<TmaMaps> tmaps;        // per instance (built when the mode is selected)
    std::vector<int> t_part, t_cap;    // first partial slot / item capacity of each instance
    std::vector<int> t_order, t_stream;   // launch order (longest first) and side stream of each instance
    int t_items;                       // items of all instances
    int t_launches;                    // kernel launches of one step (TMA launches + ghost refreshes)
    cudaStream_t side[kSide];
    cudaEvent_t fork, join[kSide];
    bool side_ok;
    bool ghosts_valid;                 // ghost cells of the current buffer hold their periodic images

    char* pbuf(int k) { return base + off_pops[k]; }
    double* sums(int k) { return (double*)(base + off_sums) + (size_t)k * 2 * n; }   // k = 0, 1: ping-pong; 2: totals
    unsigned* counters() { return (unsigned*)(base + off_counters); }   // [0..3] shared, [4 + k] instance k
    float* phis() { return (float*)(base + off_phis); }
    BatchInst* d_inst() { return (BatchInst*)(base + off_inst); }
    BatchItem* d_items() { return (BatchItem*)(base + off_items); }
    // StateBufs of instance k (read-out kernels) or of the whole batch (k < 0)
    StateBufs bufs(int k) {
        const size_t pb = pop_bytes(p.precision);
        StateBufs B;
        const size_t po = k < 0 ? 0 : (size_t)inst[k].pop_off * pb;
        const size_t fo = k < 0 ? 0 : (size_t)inst[k].field_off;
        B.src = pbuf(cur) + po;
        B.dst = pbuf(cur ^ 1) + po;
        B.src_index = cur;
        B.pull_f = fresh_f ? 0 : 1;
        B.pull_g = fresh_g ? 0 : 1;
        B.psirho = (float2*)(base + off_psirho);
        B.phis = phis() + fo;
        B.partial = (double2*)(base + off_partial);
        B.counter = k < 0 ? counters() : counters() + 2;
        B.flag = (int*)(base + off_flag);
        B.vel = nullptr;
        return B;
    }
};

namespace {

int items_of_plan(const lbm_batch* b, const Plan& pl, std::vector<BatchItem>* items, std::vector<BatchInst>* inst) {
    int count = 0;
    for (int idx = 0; idx < b->n; ++idx) {
        const int k = b->order[idx];
        const DevParams& d = b->dps[k];
        const int tx = (d.nx + 31) / 32, ty = (d.ny + pl.ty - 1) / pl.ty;
        int zc = (d.nz + pl.zsplit - 1) / pl.zsplit;
        if (zc < 8) zc = d.nz < 8 ? d.nz : 8;
        const int chunks = (d.nz + zc - 1) / zc;
        if (inst) {
            (*inst)[k].item0 = count;
            (*inst)[k].n_items = tx * ty * chunks;
        }
        for (int c = 0; c < chunks; ++c)
            for (int j = 0; j < ty; ++j)
                for (int i = 0; i < tx; ++i) {
                    if (items) {
                        BatchItem w;
                        w.inst = k;
                        w.x0 = i * 32;
                        w.y0 = j * pl.ty;
                        w.z0 = c * zc;
                        w.z1 = std::min(d.nz, (c + 1) * zc);
                        w.pad_ = 0;
                        items->push_back(w);
                    }
                    ++count;
                }
    }
    return count;
}

void drop_batch_graphs(lbm_batch* b) {
    for (int k = 0; k < b->n_graphs; ++k) cudaGraphExecDestroy(b->graphs[k].exec);
    b->n_graphs = 0;
}

// TMA mode: tensor maps and plan of every instance: whole-column items and the tile shape with
// the least padded volume per node rate (the plan model for one CTA: the instances share the
// GPU; on the 256-instance ensemble 15.2k MLUPS against 14.4k for the model's single-lattice
// choice, the smallest tile); then the instances go to the side streams longest first, each to
// the stream with the least modelled work so far, so that the streams reach each join together.
// LBM_ESTATE if an instance runs neither the TMA nor the generic fused kernel.
int set_tma_plan(lbm_batch* b) {
    if (!b->side_ok) {
        for (int q = 0; q < kSide; ++q) GB300_CK(cudaStreamCreateWithFlags(&b->side[q], cudaStreamNonBlocking));
        GB300_CK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
        for (int q = 0; q < kSide; ++q) GB300_CK(cudaEventCreateWithFlags(&b->join[q], cudaEventDisableTiming));
        b->side_ok = true;
    }
    long long cap = 0;
    for (int k = 0; k < b->n; ++k) cap += b->t_cap[k];
    if (cap > b->max_partial) return fail(LBM_ESTATE, "the TMA mode needs %lld partial sums, the batch holds %d", cap,
                                          b->max_partial);
    const size_t pb = pop_bytes(b->p.precision);
    b->tmaps.assign(b->n, TmaMaps());
    b->t_part.assign(b->n, 0);
    int off = 0, ctas = 0, launches = 0;
    for (int k = 0; k < b->n; ++k) {
        const DevParams& d = b->dps[k];
        const size_t po = (size_t)b->inst[k].pop_off * pb;
        const bool tma = build_tma_maps(d, b->p.precision, b->pbuf(0) + po, b->pbuf(1) + po, 1, -1, d.nz,
                                        b->t_cap[k], &b->tmaps[k]);
        if (!tma && !fused_supported(d))
            return fail(LBM_ESTATE, "instance %d (%d x %d x %d) runs neither the TMA nor the generic fused kernel", k,
                        d.nx, d.ny, d.nz);
        b->t_part[k] = off;
        off += b->t_cap[k];
        launches += tma && !b->tmaps[k].ghosts ? 2 : 1;
        ctas += tma ? std::min(b->tmaps[k].items, b->tmaps[k].sms) : (int)fused_blocks(d);
    }
    b->t_items = off;
    b->t_launches = launches;
    // modelled work of each instance (padded nodes over the tile shape's node rate), streams by LPT
    std::vector<double> work(b->n), load(kSide, 0.0);
    for (int k = 0; k < b->n; ++k) {
        const TmaMaps& m = b->tmaps[k];
        const DevParams& d = b->dps[k];
        work[k] = m.ok ? (double)m.items * tma_tile_w(m.shape) * tma_tile_h(m.shape) * (d.nz + 2) / tma_rate(m.shape)
                       : 1.5 * (double)d.N;
    }
    b->t_order.resize(b->n);
    std::iota(b->t_order.begin(), b->t_order.end(), 0);
    std::stable_sort(b->t_order.begin(), b->t_order.end(), [&](int a, int c) { return work[a] > work[c]; });
    b->t_stream.assign(b->n, 0);
    for (int k : b->t_order) {
        const int q = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        b->t_stream[k] = q;
        load[q] += work[k];
    }
    b->n_items = 0;
    for (int k = 0; k < b->n; ++k) b->n_items += b->tmaps[k].ok ? b->tmaps[k].items : (int)fused_blocks(b->dps[k]);
    b->ctas = ctas;
    b->plan = kTmaPlan;
    drop_batch_graphs(b);
    return LBM_OK;
}

// Upload the instance and item tables of plan `plan` and size the persistent grid.
int set_plan(lbm_batch* b, int plan) {
    if (plan == kTmaPlan) return set_tma_plan(b);
    const Plan& pl = kPlans[plan];
    std::vector<BatchItem> items;
    items.reserve(b->max_items);
    b->n_items = items_of_plan(b, pl, &items, &b->inst);
    GB300_CK(cudaMemcpyAsync(b->d_inst(), b->inst.data(), sizeof(BatchInst) * b->n, cudaMemcpyHostToDevice,
                             b->stream));
    GB300_CK(cudaMemcpyAsync(b->d_items(), items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice,
                             b->stream));
    GB300_CK(cudaStreamSynchronize(b->stream));
    const int per_sm = batch_ctas_per_sm(b->p.precision, pl.ty);
    if (per_sm < 1) return fail(LBM_ECUDA, "batched kernel (tile rows %d) cannot be resident on an SM", pl.ty);
    b->ctas = std::min(b->n_items, per_sm * b->sms);
    b->plan = plan;
    drop_batch_graphs(b);
    return LBM_OK;
}

// m steps in TMA mode: the instances are independent, so each one's chain of m steps (the TMA
// kernel once its state is streamed, the generic fused kernel on the first step, the ghost
// refresh where its tiles do not write their ghost cells) runs on its side stream (assigned by
// set_tma_plan), longest first; the side streams fork from and join the batch's stream once.
int enqueue_tma_steps(lbm_batch* b, int m) {
    cudaError_t e = cudaEventRecord(b->fork, b->launch);
    for (int q = 0; q < kSide && e == cudaSuccess; ++q) e = cudaStreamWaitEvent(b->side[q], b->fork, 0);
    const bool fresh0 = b->first || (b->fresh_f && !b->p.flow_off) || (b->fresh_g && !b->p.thermal_off);
    for (int idx = 0; idx < b->n && e == cudaSuccess; ++idx) {
        const int k = b->t_order[idx];
        cudaStream_t s = b->side[b->t_stream[k]];
        const TmaMaps* maps = &b->tmaps[k];
        StateBufs B0 = b->bufs(k);
        // a state the batched kernel wrote: refresh its ghost cells before the first TMA launch
        if (!fresh0 && !b->ghosts_valid && maps->ok) e = launch_ghosts(b->dps[k], b->p.precision, (void*)B0.src, s);
        for (int j = 0; j < m && e == cudaSuccess; ++j) {
            const int cur = b->cur ^ (j & 1), slot = b->slot ^ (j & 1);
            // a frozen field (flow_off / thermal_off) keeps its un-streamed form on every step
            const bool ff = b->fresh_f && (j == 0 || b->p.flow_off), fg = b->fresh_g && (j == 0 || b->p.thermal_off);
            StateBufs B = B0;
            const size_t po = (size_t)b->inst[k].pop_off * pop_bytes(b->p.precision);
            B.src = b->pbuf(cur) + po;
            B.dst = b->pbuf(cur ^ 1) + po;
            B.src_index = cur;
            B.pull_f = ff ? 0 : 1;
            B.pull_g = fg ? 0 : 1;
            B.partial += b->t_part[k];
            B.counter = b->counters() + 4 + k;
            bool ghosts_done = false;
            e = launch_fused(b->dps[k], b->p.precision, B, b->sums(slot) + 2 * k, b->sums(slot ^ 1) + 2 * k,
                             j == 0 && b->first ? 1 : 0, s, maps, &ghosts_done);
            // the next TMA launch reads ghost cells (the generic kernel wraps its pulls itself)
            if (e == cudaSuccess && !ghosts_done && maps->ok) e = launch_ghosts(b->dps[k], b->p.precision, B.dst, s);
        }
    }
    for (int q = 0; q < kSide && e == cudaSuccess; ++q) {
        e = cudaEventRecord(b->join[q], b->side[q]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->launch, b->join[q], 0);
    }
    if (e != cudaSuccess) return fail(LBM_ECUDA, "TMA-mode steps: %s", cudaGetErrorString(e));
    if (m > 0) {
        b->ghosts_valid = true;
        b->cur ^= m & 1;
        b->slot ^= m & 1;
        if (!b->p.flow_off) b->fresh_f = false;
        if (!b->p.thermal_off) b->fresh_g = false;
        b->first = false;
        b->steps += m;
    }
    return LBM_OK;
}

int enqueue_batch_step(lbm_batch* b) {
    if (b->plan == kTmaPlan) return enqueue_tma_steps(b, 1);
    StateBufs B = b->bufs(-1);
    cudaError_t e = launch_fused_batch(b->dps[0], b->p.precision, kPlans[b->plan].ty, b->d_inst(), b->d_items(),
                                       b->n_items, b->n, B, b->sums(b->slot), b->sums(b->slot ^ 1),
                                       b->first ? 1 : 0, b->ctas, b->launch);
    if (e != cudaSuccess) return fail(LBM_ECUDA, "batched kernel launch: %s", cudaGetErrorString(e));
    b->ghosts_valid = false;   // the batched kernel does not write ghost cells
    b->cur ^= 1;
    b->slot ^= 1;
    if (!b->p.flow_off) b->fresh_f = false;
    if (!b->p.thermal_off) b->fresh_g = false;
    b->first = false;
    b->steps += 1;
    return LBM_OK;
}

// Graph of m steps from the current (cur, slot), captured on first use.
int batch_graph(lbm_batch* b, int m, cudaGraphExec_t* out) {
    BatchGraph* hit = nullptr;
    for (int k = 0; k < b->n_graphs; ++k) {
        BatchGraph& g = b->graphs[k];
        if (g.n == m && g.cur == b->cur && g.slot == b->slot && g.plan == b->plan && g.ghosts_valid == b->ghosts_valid)
            hit = &g;
    }
    if (!hit) {
        const int c0 = b->cur, s0 = b->slot;
        const bool ff = b->fresh_f, fg = b->fresh_g, fi = b->first, gv = b->ghosts_valid;
        const long long st = b->steps;
        if (!b->capture) GB300_CK(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking));
        cudaGraph_t graph;
        GB300_CK(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
        b->launch = b->capture;
        int rc = LBM_OK;
        if (b->plan == kTmaPlan) rc = enqueue_tma_steps(b, m);
        else
            for (int k = 0; k < m && rc == LBM_OK; ++k) rc = enqueue_batch_step(b);
        cudaError_t e = cudaStreamEndCapture(b->capture, &graph);
        b->launch = b->stream;
        b->cur = c0; b->slot = s0; b->fresh_f = ff; b->fresh_g = fg; b->first = fi; b->steps = st;
        b->ghosts_valid = gv;
        if (rc != LBM_OK) { if (e == cudaSuccess) cudaGraphDestroy(graph); return rc; }
        if (e != cudaSuccess) return fail(LBM_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        cudaGraphExec_t exec;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(LBM_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        if (b->n_graphs == kBatchGraphs) {
            cudaGraphExecDestroy(b->graphs[0].exec);
            for (int k = 1; k < b->n_graphs; ++k) b->graphs[k - 1] = b->graphs[k];
            --b->n_graphs;
        }
        BatchGraph& g = b->graphs[b->n_graphs++];
        g.n = m; g.cur = b->cur; g.slot = b->slot; g.plan = b->plan; g.ghosts_valid = b->ghosts_valid; g.exec = exec;
        hit = &g;
    }
    *out = hit->exec;
    return LBM_OK;
}

// n steps by graph replay: one graph of all n steps for a persistent plan (one node a step); in
// the TMA mode (hundreds of launches a step) a graph of kTmaChain steps replayed n / kTmaChain
// times, the remaining steps enqueued directly.
int run_batch_graph(lbm_batch* b, int n) {
    if (b->plan == kTmaPlan && !b->ghosts_valid && n > 0) {
        // a state the batched kernel wrote: one step with the ghost refresh outside the graph,
        // so that the replayed graph carries none
        const int rc = enqueue_tma_steps(b, 1);
        if (rc || --n == 0) return rc;
    }
    const int m = b->plan == kTmaPlan ? std::min(n, kTmaChain) : n;
    cudaGraphExec_t exec = nullptr;
    int rc = batch_graph(b, m, &exec);
    if (rc) return rc;
    for (int r = 0; r < n / m; ++r) {
        GB300_CK(cudaGraphLaunch(exec, b->stream));
        for (int k = 0; k < m; ++k) {   // m is even or n == m: (cur, slot) match the graph again
            b->cur ^= 1;
            b->slot ^= 1;
        }
        b->steps += m;
        b->ghosts_valid = b->plan == kTmaPlan;   // the batched kernel does not write ghost cells
    }
    if (n % m) rc = b->plan == kTmaPlan ? enqueue_tma_steps(b, n % m) : enqueue_batch_step(b);
    return rc;
}

int check_batch_flag(lbm_batch* b) {
    int h = 0;
    GB300_CK(cudaMemcpyAsync(&h, b->base + b->off_flag, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    GB300_CK(cudaStreamSynchronize(b->stream));
    if (h) {
        GB300_CK(cudaMemsetAsync(b->base + b->off_flag, 0, sizeof(int), b->stream));
        if (h & 4) return fail(LBM_EBOUNDS, "a kernel index fell outside its buffer (bounds-checked build, step %lld)",
                               b->steps);
        if (h & 2) return fail(LBM_ETIMEOUT, "a bounded device wait gave up (step %lld)", b->steps);
        return fail(LBM_ENONFINITE, "non-finite rho/T/psi or psi^2 <= 0 in the batch after step %lld", b->steps);
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_create(const lbm_params* common, int n_instances, const int* dims, lbm_batch** out) {
    if (common && common->thermal_q == 19)
        return fail(LBM_EINVAL, "the batched ensemble runs the D3Q7 temperature lattice only");
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!common || !dims) return fail(LBM_EINVAL, "common and dims are required");
    if (n_instances < 1) return fail(LBM_EINVAL, "n_instances must be >= 1");
    if (common->kernel == LBM_KERNEL_TWO_PASS) return fail(LBM_EINVAL, "the batch runs the fused kernel only");
    if (common->divu_mode != 0) return fail(LBM_EINVAL, "the batch computes div u by Eq. 48 only (divu_mode 0)");
    if (common->wall_rho != 0.0 || common->wall_scheme != 0)
        return fail(LBM_EINVAL, "the batch has no wetting wall (wall_rho 0, wall_scheme 0)");
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return fail(LBM_ENOMEM, "host allocation failed");
    b->p = *common;
    b->n = n_instances;
    b->dps.resize(n_instances);
    b->inst.resize(n_instances);
    b->nodes = 0;
    b->pop_elems = 0;
    b->max_N = 0;
    for (int k = 0; k < n_instances; ++k) {
        lbm_params pk = *common;
        pk.nx = dims[3 * k];
        pk.ny = dims[3 * k + 1];
        pk.nz = dims[3 * k + 2];
        int rc = validate(&pk);
        if (rc) {
            char why[256];
            snprintf(why, sizeof(why), "%s", lbm_last_error());
            delete b;
            return fail(rc, "instance %d (%d x %d x %d): %s", k, pk.nx, pk.ny, pk.nz, why);
        }
        DevParams d = make_dev(&pk);
        b->dps[k] = d;
        BatchInst& I = b->inst[k];
        memset(&I, 0, sizeof(I));
        I.nx = d.nx; I.ny = d.ny; I.nz = d.nz; I.Ws = d.Ws; I.Hs = d.Hs;
        I.pop_off = b->pop_elems;
        I.field_off = b->nodes;
        I.inv_N = d.inv_N;
        b->pop_elems += (long long)pop_elems(d);
        b->nodes += d.N;
        b->max_N = std::max(b->max_N, d.N);
    }
    if (b->nodes >= (1LL << 40)) {
        delete b;
        return fail(LBM_EINVAL, "batch too large");
    }
    b->order.resize(n_instances);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(),
                     [&](int a, int c) { return b->dps[a].N > b->dps[c].N; });
    b->max_items = 0;
    for (int q = 0; q < kNumPlans; ++q) b->max_items = std::max(b->max_items, items_of_plan(b, kPlans[q], nullptr, nullptr));
    b->max_partial = b->max_items;
    for (int k = 0; k < n_instances; ++k) b->max_partial = std::max(b->max_partial, max_partials(b->dps[k]));
    // TMA mode: whole-column items, at most the tiles of the smallest tile shape per instance
    // (or the blocks of the generic fused kernel, which runs an instance's first step and every
    // step of an instance the TMA kernel cannot take)
    b->t_cap.assign(n_instances, 0);
    long long t_total = 0;
    for (int k = 0; k < n_instances; ++k) {
        const DevParams& d = b->dps[k];
        b->t_cap[k] = (int)std::min<long long>(fused_blocks(d), 1 << 30);
        for (int sh = 0; sh < tma_num_shapes(); ++sh) {
            const int tiles = ((d.nx + tma_tile_w(sh) - 1) / tma_tile_w(sh)) * ((d.ny + tma_tile_h(sh) - 1) / tma_tile_h(sh));
            b->t_cap[k] = std::max(b->t_cap[k], tiles);
        }
        t_total += b->t_cap[k];
    }
    if (t_total < (1LL << 30)) b->max_partial = std::max(b->max_partial, (int)t_total);

    const size_t pb = pop_bytes(common->precision);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    b->off_pops[0] = take((size_t)b->pop_elems * pb);
    b->off_pops[1] = take((size_t)b->pop_elems * pb);
    b->off_phis = take(4 * (size_t)b->nodes);
    b->off_psirho = take(8 * (size_t)b->max_N);
    b->off_sums = take(sizeof(double) * 6 * (size_t)n_instances);
    b->off_partial = take(sizeof(double2) * (size_t)b->max_partial);
    b->off_counters = take((4 + (size_t)n_instances) * sizeof(unsigned));
    b->off_flag = take(sizeof(int));
    b->off_inst = take(sizeof(BatchInst) * (size_t)n_instances);
    b->off_items = take(sizeof(BatchItem) * (size_t)b->max_items);
    b->stream = (cudaStream_t)common->cuda_stream;
    b->launch = b->stream;
    b->capture = nullptr;
    b->side_ok = false;
    b->ghosts_valid = false;
    b->t_items = 0;
    b->t_launches = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return fail(LBM_ECUDA, "no CUDA device");
    }
    cudaError_t e = cudaMalloc((void**)&b->base, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return fail(LBM_ENOMEM, "cudaMalloc(%zu): %s", off, cudaGetErrorString(e));
    }
    for (auto& d : b->dps) d.check_flag = (int*)(b->base + b->off_flag);
    e = cudaMemsetAsync(b->base + b->off_sums, 0, b->off_inst - b->off_sums, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    int rc = e == cudaSuccess ? set_plan(b, 0) : fail(LBM_ECUDA, "initial memset: %s", cudaGetErrorString(e));
    if (rc) {
        cudaFree(b->base);
        delete b;
        return rc;
    }
    *out = b;
    return LBM_OK;
}

long long lbm_batch_nodes(const lbm_batch* b, int instance) {
    if (!b) return 0;
    if (instance < 0) return b->nodes;
    if (instance >= b->n) return 0;
    return b->dps[instance].N;
}

int lbm_batch_init_fields(lbm_batch* b, const float* rho, const float* T, const float* u) {
    if (!b) return fail(LBM_EINVAL, "batch is NULL");
    if (!rho || !T) return fail(LBM_EINVAL, "rho and T are required");
    const size_t N = (size_t)b->nodes;
    // host inputs are staged in the second population buffer (>= 26 N two-byte elements)
    float* stage = (float*)b->pbuf(1);
    const float *drho = rho, *dT = T, *du = u;
    if (!is_device_ptr(rho)) {
        GB300_CK(cudaMemcpyAsync(stage, rho, N * 4, cudaMemcpyHostToDevice, b->stream));
        drho = stage;
    }
    if (!is_device_ptr(T)) {
        GB300_CK(cudaMemcpyAsync(stage + N, T, N * 4, cudaMemcpyHostToDevice, b->stream));
        dT = stage + N;
    }
    if (u && !is_device_ptr(u)) {
        GB300_CK(cudaMemcpyAsync(stage + 2 * N, u, 3 * N * 4, cudaMemcpyHostToDevice, b->stream));
        du = stage + 2 * N;
    }
    drop_batch_graphs(b);
    b->cur = 0;
    b->slot = 0;
    const size_t pb = pop_bytes(b->p.precision);
    for (int k = 0; k < b->n; ++k) {
        const BatchInst& I = b->inst[k];
        const size_t fo = (size_t)I.field_off;
        GB300_CK(launch_init(b->dps[k], b->p.precision, b->pbuf(0) + (size_t)I.pop_off * pb, drho + fo, dT + fo,
                             du ? du + 3 * fo : nullptr, b->stream));
        StateBufs B = b->bufs(k);
        GB300_CK(launch_sum_field(drho + fo, b->dps[k].N, B.partial, B.counter, b->sums(0) + 2 * k, b->stream));
    }
    GB300_CK(cudaMemsetAsync(b->base + b->off_flag, 0, sizeof(int), b->stream));
    GB300_CK(cudaStreamSynchronize(b->stream));
    b->fresh_f = b->fresh_g = true;
    b->first = true;
    b->ghosts_valid = false;
    b->initialised = true;
    b->steps = 0;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int n) {
    NvtxRange range("lbm_batch_step");
    if (!b) return fail(LBM_EINVAL, "batch is NULL");
    if (!b->initialised) return fail(LBM_ESTATE, "lbm_batch_step before lbm_batch_init_fields");
    if (n < 0) return fail(LBM_EINVAL, "n < 0");
    int rc = LBM_OK, k = 0;
    while (k < n && (b->first || (b->fresh_f && !b->p.flow_off) || (b->fresh_g && !b->p.thermal_off))) {
        rc = enqueue_batch_step(b);
        if (rc) return rc;
        ++k;
    }
    if (k < n) {
        if (b->p.use_graph) rc = run_batch_graph(b, n - k);
        else
            for (; k < n && rc == LBM_OK; ++k) rc = enqueue_batch_step(b);
        if (rc) return rc;
    }
    if (b->p.check_nonfinite) return check_batch_flag(b);
    return LBM_OK;
}

int lbm_batch_autotune(lbm_batch* b, int steps, double* best_ms) {
    if (!b) return fail(LBM_EINVAL, "batch is NULL");
    if (!b->initialised) return fail(LBM_ESTATE, "lbm_batch_autotune before lbm_batch_init_fields");
    if (steps < 1) return fail(LBM_EINVAL, "steps must be >= 1");
    // save the state the candidates advance: populations, phi_s history, rho_ave sums
    const size_t pb = pop_bytes(b->p.precision);
    const size_t pop_bytes_all = (size_t)b->pop_elems * pb, phis_bytes = 4 * (size_t)b->nodes;
    const size_t sums_bytes = sizeof(double) * 4 * (size_t)b->n;
    char* save = nullptr;
    cudaError_t e = cudaMalloc((void**)&save, pop_bytes_all + phis_bytes + sums_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ENOMEM, "autotune state copy: %s", cudaGetErrorString(e));
    }
    const int c0 = b->cur, s0 = b->slot;
    const bool ff = b->fresh_f, fg = b->fresh_g, fi = b->first, gv = b->ghosts_valid;
    const long long st = b->steps;
    auto save_or_restore = [&](bool restore) -> cudaError_t {
        char* a[3] = {b->pbuf(c0), (char*)b->phis(), (char*)b->sums(0)};
        char* s[3] = {save, save + pop_bytes_all, save + pop_bytes_all + phis_bytes};
        size_t n[3] = {pop_bytes_all, phis_bytes, sums_bytes};
        for (int k = 0; k < 3; ++k) {
            cudaError_t r = cudaMemcpyAsync(restore ? a[k] : s[k], restore ? s[k] : a[k], n[k],
                                            cudaMemcpyDeviceToDevice, b->stream);
            if (r != cudaSuccess) return r;
        }
        return cudaSuccess;
    };
    cudaEvent_t ev[2];
    cudaEventCreate(&ev[0]);
    cudaEventCreate(&ev[1]);
    int rc = LBM_OK, best = b->plan;
    float best_t = -1.f;
    e = save_or_restore(false);
    if (e != cudaSuccess) rc = fail(LBM_ECUDA, "autotune save: %s", cudaGetErrorString(e));
    for (int q = 0; q <= kTmaPlan && rc == LBM_OK; ++q) {
        rc = set_plan(b, q);
        if (rc && q == kTmaPlan) {   // an instance the TMA kernel cannot run: not a candidate
            rc = LBM_OK;
            break;
        }
        if (rc) break;
        rc = enqueue_batch_step(b);   // warm-up
        cudaEventRecord(ev[0], b->stream);
        if (q == kTmaPlan && rc == LBM_OK) rc = enqueue_tma_steps(b, steps);
        else
            for (int k = 0; k < steps && rc == LBM_OK; ++k) rc = enqueue_batch_step(b);
        cudaEventRecord(ev[1], b->stream);
        if (cudaEventSynchronize(ev[1]) != cudaSuccess) rc = fail(LBM_ECUDA, "autotune timing failed");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (rc == LBM_OK && (best_t < 0.f || ms < best_t)) {
            best_t = ms;
            best = q;
        }
        e = save_or_restore(true);
        if (e != cudaSuccess && rc == LBM_OK) rc = fail(LBM_ECUDA, "autotune restore: %s", cudaGetErrorString(e));
        b->cur = c0; b->slot = s0; b->fresh_f = ff; b->fresh_g = fg; b->first = fi; b->steps = st;
        b->ghosts_valid = gv;
    }
    cudaStreamSynchronize(b->stream);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    cudaFree(save);
    if (rc == LBM_OK) rc = set_plan(b, best);
    if (rc == LBM_OK) {
        GB300_CK(cudaMemsetAsync(b->base + b->off_flag, 0, sizeof(int), b->stream));
        GB300_CK(cudaStreamSynchronize(b->stream));
    }
    if (best_ms) *best_ms = best_t / steps;
    return rc;
}

int lbm_batch_plan(const lbm_batch* b, int* tile_rows, int* z_split, int* items, int* ctas) {
    if (!b) return fail(LBM_EINVAL, "batch is NULL");
    if (tile_rows) *tile_rows = b->plan == kTmaPlan ? 0 : kPlans[b->plan].ty;
    if (z_split) *z_split = b->plan == kTmaPlan ? 0 : kPlans[b->plan].zsplit;
    if (items) *items = b->n_items;
    if (ctas) *ctas = b->ctas;
    return LBM_OK;
}

int lbm_batch_select_plan(lbm_batch* b, int tile_rows, int z_split) {
    if (!b) return fail(LBM_EINVAL, "batch is NULL");
    if (tile_rows == 0 && z_split == 0) return set_plan(b, kTmaPlan);
    for (int q = 0; q < kNumPlans; ++q)
        if (kPlans[q].ty == tile_rows && kPlans[q].zsplit == z_split) return set_plan(b, q);
    return fail(LBM_EINVAL, "no plan with tile rows %d and %d z-chunks", tile_rows, z_split);
}

int lbm_batch_get_moments(lbm_batch* b, float* rho, float* ux, float* uy, float* uz, float* T) {
    if (!b) return fail(LBM_EINVAL, "batch is NULL");
    if (!b->initialised) return fail(LBM_ESTATE, "lbm_batch_get_moments before lbm_batch_init_fields");
    const size_t N = (size_t)b->nodes;
    float* outs[5] = {rho, ux, uy, uz, T};
    bool dev[5];
    for (int q = 0; q < 5; ++q) dev[q] = outs[q] && is_device_ptr(outs[q]);
    float* stage = (float*)b->pbuf(b->cur ^ 1);   // overwritten by the next step anyway
    for (int k = 0; k < b->n; ++k) {
        StateBufs B = b->bufs(k);
        const size_t fo = (size_t)b->inst[k].field_off;
        float* dst[5];
        for (int q = 0; q < 5; ++q) dst[q] = outs[q] ? (dev[q] ? outs[q] : stage + q * N) + fo : nullptr;
        GB300_CK(launch_psi(b->dps[k], b->p.precision, B, nullptr, b->stream));
        GB300_CK(launch_moments(b->dps[k], b->p.precision, B, b->sums(b->slot) + 2 * k, dst[0], dst[1], dst[2],
                                dst[3], dst[4], b->stream));
    }
    for (int q = 0; q < 5; ++q)
        if (outs[q] && !dev[q])
            GB300_CK(cudaMemcpyAsync(outs[q], stage + q * N, N * 4, cudaMemcpyDeviceToHost, b->stream));
    GB300_CK(cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

int lbm_batch_get_totals(lbm_batch* b, double* sums) {
    if (!b || !sums) return fail(LBM_EINVAL, "NULL argument");
    if (!b->initialised) return fail(LBM_ESTATE, "lbm_batch_get_totals before lbm_batch_init_fields");
    for (int k = 0; k < b->n; ++k) {
        StateBufs B = b->bufs(k);
        GB300_CK(launch_psi(b->dps[k], b->p.precision, B, b->sums(2) + 2 * k, b->stream));
    }
    GB300_CK(cudaMemcpyAsync(sums, b->sums(2), sizeof(double) * 2 * b->n, cudaMemcpyDeviceToHost, b->stream));
    GB300_CK(cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

long long lbm_batch_steps_done(const lbm_batch* b) { return b ? b->steps : 0; }

int lbm_batch_launches_per_step(const lbm_batch* b) {
    if (!b) return fail(LBM_EINVAL, "batch is NULL");
    return b->plan == kTmaPlan ? b->t_launches : 1;
}

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    drop_batch_graphs(b);
    if (b->capture) cudaStreamDestroy(b->capture);
    if (b->side_ok) {
        for (int q = 0; q < kSide; ++q) {
            cudaStreamDestroy(b->side[q]);
            cudaEventDestroy(b->join[q]);
        }
        cudaEventDestroy(b->fork);
    }
    if (b->base) cudaFree(b->base);
    delete b;
}

}  // extern "C"
