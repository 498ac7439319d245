// Many beams in one dedispersion launch, its CUDA graph, and the schedule autotuner.
//
// A batch holds one plan per beam (uneven trial counts, DM ranges and lengths).  Its
// work list has one item per CTA tile of every beam -- (beam, trial block, time tile) --
// and the launch one CTA per item, in list order: beams by decreasing cost (the small
// ones fill the last wave), each beam's tiles in the plain launch's grouped order.  The
// graph captures the launch and, when bound, every beam's channel statistics and boxcar
// S/N, so one graph launch processes a block of all beams.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <new>
#include <sstream>
#include <string>

#include "dd_internal.h"
#include "dd_trace.h"

struct dd_batch_s {
    std::vector<dd_plan_s*> plans;
    bool u8 = false, pair = true;
    bool rl = false;         // run-length beams (per-channel prefix sums, then differences)
    bool short_taps = true;  // every plan's tap runs fit one register window (run-length
                             // beams: every plan shares difference rows in the CTA)
    std::vector<uint32_t*> d_prefix;  // run-length beams: each beam's prefix sums
    std::vector<int64_t> ldp;
    std::vector<dd::BatchItem> items;
    size_t smem = 0;
    int grid = 0;
    int device = -1;
    int64_t units = 0;  // sum over beams of trials x outputs
    dd::DedispArgs* d_args = nullptr;
    dd::BatchItem* d_items = nullptr;
    bool bound = false;
    // per-beam buffers bound for the boxcar stage of the graph
    std::vector<const void*> in;
    std::vector<int64_t> in_ld;
    std::vector<void*> out;
    std::vector<int64_t> out_ld;
    std::vector<int32_t> widths;
    std::vector<double*> mean, sd;
    std::vector<float*> peak;
    std::vector<int32_t*> arg;
    bool box_bound = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

int64_t plan_t_out(const dd_plan_s* p) { return p->band.nsamp - p->dmax; }

void free_batch_dev(dd_batch_s* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (uint32_t* q : b->d_prefix) cudaFree(q);
    b->d_prefix.clear();
    b->ldp.clear();
    cudaFree(b->d_args);
    cudaFree(b->d_items);
    b->exec = nullptr;
    b->graph = nullptr;
    b->d_args = nullptr;
    b->d_items = nullptr;
}

// Work list: one item per CTA tile, with the tile's FMA count (run-length beams: its
// trial-channel pairs, each costing the same per output whatever its taps) plus a fixed
// per-stage cost as the estimate; sorted largest first.
// The work list: beams in decreasing order of estimated cost (so that the small ones fill
// the last wave), and within a beam the plain launch's tile order: trial blocks taken
// kGroupBlocks at a time, blocks fastest within a group and then time tiles, so that the
// CTAs working together share the beam's input columns and stage records in L2.
void build_items(dd_batch_s* b) {
    constexpr int kGroupBlocks = 16;
    struct Beam {
        double cost;
        int beam;
    };
    std::vector<Beam> order;
    b->units = 0;
    for (int beam = 0; beam < (int)b->plans.size(); ++beam) {
        const dd_plan_s* p = b->plans[beam];
        const int64_t t_out = plan_t_out(p);
        const int nst = (p->nchan + p->cs - 1) / p->cs;
        const int64_t tile = (int64_t)dd::chunk_t(p->pair) * p->nch;
        const int64_t ntile = (t_out + tile - 1) / tile;
        double taps = 0;
        for (int64_t i = 0; i < (int64_t)p->ndm * p->nchan; ++i) taps += p->rl ? 1.0 : p->taps[(size_t)i];
        b->units += (int64_t)p->ndm * t_out;
        order.push_back({taps * (double)t_out + 2.0e4 * nst * ntile * p->nblk, beam});
    }
    std::stable_sort(order.begin(), order.end(), [](const Beam& x, const Beam& y) { return x.cost > y.cost; });
    b->items.clear();
    for (const Beam& bm : order) {
        const dd_plan_s* p = b->plans[bm.beam];
        const int64_t t_out = plan_t_out(p);
        const int64_t tile = (int64_t)dd::chunk_t(p->pair) * p->nch;
        const int ntile = (int)((t_out + tile - 1) / tile);
        for (int g0 = 0; g0 < p->nblk; g0 += kGroupBlocks)
            for (int tx = 0; tx < ntile; ++tx)
                for (int blk = g0; blk < std::min(p->nblk, g0 + kGroupBlocks); ++blk) {
                    dd::BatchItem it;
                    it.beam = bm.beam;
                    it.blk = blk;
                    it.tx = tx;
                    it.pad = 0;
                    b->items.push_back(it);
                }
    }
}

bool aligned16(const void* ptr) { return ((uintptr_t)ptr & 15u) == 0; }

}  // namespace

extern "C" {

dd_status dd_batch_create(dd_batch_t* out, const dd_plan_t* plans, int32_t nbeams) {
    if (!out || !plans || nbeams < 1) return DD_ERR_ARG;
    *out = nullptr;
    for (int i = 0; i < nbeams; ++i) {
        if (!plans[i]) return DD_ERR_ARG;
        if (plans[i]->band.in_type != plans[0]->band.in_type || plans[i]->pair != plans[0]->pair)
            return DD_ERR_ARG;
        if (plan_t_out(plans[i]) < 1) return DD_ERR_ARG;
        // one kernel serves the batch: every beam on the same tap-sum path
        if (plans[i]->rl != plans[0]->rl || plans[i]->rl_b != plans[0]->rl_b) return DD_ERR_UNSUPPORTED;
        if (plans[i]->rl && plans[i]->band.nsamp > ((int64_t)1 << 24)) return DD_ERR_UNSUPPORTED;
    }
    dd_batch_s* b = new (std::nothrow) dd_batch_s;
    if (!b) return DD_ERR_OOM;
    b->plans.assign(plans, plans + nbeams);
    b->u8 = plans[0]->band.in_type == DD_U8;
    b->pair = plans[0]->pair;
    b->rl = plans[0]->rl;
    for (auto* p : b->plans) b->smem = std::max(b->smem, dd::dedisp_smem_for(p));
    build_items(b);
    *out = b;
    return DD_OK;
}

dd_status dd_batch_bind(dd_batch_t b, const void* const* d_in, const int64_t* in_ld,
                        void* const* d_out, const int64_t* out_ld) {
    if (!b || !d_in || !in_ld || !d_out || !out_ld) return DD_ERR_ARG;
    const int nb = (int)b->plans.size();
    std::vector<dd::DedispArgs> args(nb);
    for (int i = 0; i < nb; ++i) {
        dd_plan_s* p = b->plans[i];
        if (p->rl != b->rl || p->pair != b->pair || (b->rl && p->rl_b != b->plans[0]->rl_b))
            return DD_ERR_UNSUPPORTED;  // a plan changed path since dd_batch_create
        const int64_t esz = p->band.in_type == DD_U8 ? 1 : 4;
        const int64_t t_out = plan_t_out(p);
        if (!d_in[i] || !d_out[i] || !aligned16(d_in[i]) || (in_ld[i] * esz) % 16 != 0 ||
            in_ld[i] < p->band.nsamp || out_ld[i] < t_out)
            return DD_ERR_ARG;
        dd_status st = dd::upload_tables(p);
        if (st != DD_OK) return st;
    }
    // plans may have been retuned since dd_batch_create: rebuild the work list
    b->smem = 0;
    for (auto* p : b->plans) b->smem = std::max(b->smem, dd::dedisp_smem_for(p));
    build_items(b);
    free_batch_dev(b);
    for (int i = 0; i < nb; ++i) {
        dd_plan_s* p = b->plans[i];
        const int64_t t_out = plan_t_out(p);
        if (!b->rl) {
            dd::fill_dedisp_args(p, d_in[i], in_ld[i], 0, t_out, d_out[i], out_ld[i], &args[i]);
            continue;
        }
        // run-length beams read their own prefix sums, which the batch owns
        const int64_t ldp = (p->band.nsamp + 1 + 3) & ~(int64_t)3;
        uint32_t* q = nullptr;
        const cudaError_t e = cudaMalloc((void**)&q, (size_t)ldp * p->nchan * sizeof(uint32_t));
        if (e != cudaSuccess) {
            free_batch_dev(b);
            return dd::cuda_status(e);
        }
        b->d_prefix.push_back(q);
        b->ldp.push_back(ldp);
        dd::fill_dedisp_args(p, q, ldp, 0, t_out, d_out[i], out_ld[i], &args[i]);
    }
    int dev = -1, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return dd::cuda_status(e);
    b->short_taps = true;
    for (auto* p : b->plans)
        b->short_taps = b->short_taps && (p->rl ? p->rl_b : p->pair ? p->umax <= dd::kRPair : p->kmax <= dd::kRInt);
    const int per_sm = dd::dedisp_batched_blocks_per_sm(b->u8, b->pair, b->short_taps, b->smem, b->rl);
    if (per_sm < 1) return DD_ERR_UNSUPPORTED;
    if (b->items.size() >= (size_t)INT32_MAX) return DD_ERR_UNSUPPORTED;
    b->grid = (int)b->items.size();  // one CTA per work item
    b->device = dev;
    e = cudaMalloc((void**)&b->d_args, nb * sizeof(dd::DedispArgs));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_items, b->items.size() * sizeof(dd::BatchItem));
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_args, args.data(), nb * sizeof(dd::DedispArgs), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_items, b->items.data(), b->items.size() * sizeof(dd::BatchItem),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_batch_dev(b);
        return dd::cuda_status(e);
    }
    b->in.assign(d_in, d_in + nb);
    b->in_ld.assign(in_ld, in_ld + nb);
    b->out.assign(d_out, d_out + nb);
    b->out_ld.assign(out_ld, out_ld + nb);
    b->bound = true;
    b->box_bound = false;
    dd::log_msg(1, "batch of %d beams (%s): %zu work items (one CTA each, %d resident per SM on %d SMs), "
             "%zu bytes of shared memory", nb, b->rl ? "run-length sums" : (b->pair ? "fp32 pair units" : "exact integer sums"),
             b->items.size(), per_sm, sms, b->smem);
    return DD_OK;
}

dd_status dd_batch_dedisperse(dd_batch_t b, void* stream) {
    DD_TRACE("dd_batch_dedisperse");
    if (!b) return DD_ERR_ARG;
    if (!b->bound) return DD_ERR_STATE;
    if (b->rl)  // every beam's prefix sums first
        for (size_t i = 0; i < b->plans.size(); ++i) {
            const dd_status st = dd::launch_prefix_into(b->plans[i], b->in[i], b->in_ld[i], 0,
                                                        b->plans[i]->band.nsamp, b->d_prefix[i], b->ldp[i],
                                                        (cudaStream_t)stream);
            if (st != DD_OK) return st;
        }
    return dd::launch_dedisperse_batched(b->u8, b->pair, b->short_taps, b->d_args, b->d_items, (int32_t)b->items.size(),
                                         b->smem, (cudaStream_t)stream, b->rl);
}

dd_status dd_batch_bind_boxcar(dd_batch_t b, const int32_t* widths, int32_t nw, double* const* d_mean,
                               double* const* d_std, float* const* d_peak, int32_t* const* d_arg) {
    if (!b || !widths || nw < 1 || !d_mean || !d_std || !d_peak || !d_arg) return DD_ERR_ARG;
    if (!b->bound) return DD_ERR_STATE;
    const int nb = (int)b->plans.size();
    for (int i = 0; i < nb; ++i) {
        if (!d_mean[i] || !d_std[i] || !d_peak[i] || !d_arg[i]) return DD_ERR_ARG;
        if (widths[nw - 1] > plan_t_out(b->plans[i])) return DD_ERR_ARG;
    }
    for (int i = 1; i < nw; ++i)
        if (widths[i] <= widths[i - 1] || widths[0] < 1) return DD_ERR_ARG;
    b->widths.assign(widths, widths + nw);
    b->mean.assign(d_mean, d_mean + nb);
    b->sd.assign(d_std, d_std + nb);
    b->peak.assign(d_peak, d_peak + nb);
    b->arg.assign(d_arg, d_arg + nb);
    b->box_bound = true;
    return DD_OK;
}

// Runs one block of every beam: the batched dedispersion launch and, when bound,
// every beam's channel statistics and boxcar S/N.
static dd_status batch_run(dd_batch_s* b, cudaStream_t s) {
    dd_status st = dd_batch_dedisperse(b, s);
    if (st != DD_OK || !b->box_bound) return st;
    for (size_t i = 0; i < b->plans.size(); ++i) {
        dd_plan_s* p = b->plans[i];
        st = dd_channel_stats(p, b->in[i], b->in_ld[i], 0, p->band.nsamp, b->mean[i], b->sd[i], s);
        if (st != DD_OK) return st;
        st = dd_boxcar_snr(p, b->out[i], b->out_ld[i], plan_t_out(p), b->widths.data(),
                           (int32_t)b->widths.size(), b->mean[i], b->sd[i], b->peak[i], b->arg[i],
                           INFINITY, nullptr, 0, nullptr, s);
        if (st != DD_OK) return st;
    }
    return DD_OK;
}

dd_status dd_batch_run(dd_batch_t b, void* stream) {
    DD_TRACE("dd_batch_run");
    if (!b) return DD_ERR_ARG;
    if (!b->bound) return DD_ERR_STATE;
    return batch_run(b, (cudaStream_t)stream);
}

dd_status dd_batch_capture(dd_batch_t b, void* stream) {
    if (!b || !stream) return DD_ERR_ARG;
    if (!b->bound) return DD_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    // one eager pass first: it creates every plan's workspace, which a capture may not
    dd_status st = batch_run(b, s);
    if (st != DD_OK) return st;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return dd::cuda_status(e);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return dd::cuda_status(e);
    st = batch_run(b, s);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (st != DD_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return dd::cuda_status(e);
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    return dd::cuda_status(e);
}

dd_status dd_batch_replay(dd_batch_t b, void* stream) {
    DD_TRACE("dd_batch_replay");
    if (!b) return DD_ERR_ARG;
    if (!b->exec) return DD_ERR_STATE;
    return dd::cuda_status(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
}

dd_status dd_batch_info(dd_batch_t b, int32_t* nitems, int32_t* grid, int64_t* units) {
    if (!b) return DD_ERR_ARG;
    if (nitems) *nitems = (int32_t)b->items.size();
    if (grid) *grid = b->grid;
    if (units) *units = b->units;
    return DD_OK;
}

dd_status dd_batch_destroy(dd_batch_t b) {
    if (!b) return DD_ERR_ARG;
    free_batch_dev(b);
    delete b;
    return DD_OK;
}

}  // extern "C"
