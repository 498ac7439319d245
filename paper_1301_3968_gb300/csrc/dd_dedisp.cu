// Profiled dedispersion, eq. p_dedisp (Sec. 2.1): the plain and batched kernels, the
// prefix pass of the run-length path and their launchers.  The tile itself (work
// decomposition, staging, sums) is in dd_tile.cuh.
#include "dd_tile.cuh"

namespace dd {
namespace {


// Order of the tiles.  Run-length path: trial blocks along x, time tiles along y, so that
// the CTAs resident together share time tiles and each tile's prefix rows come from L2
// for all trial blocks (instead of every trial block reading the whole prefix array from
// DRAM).  Other paths: the grid is (time tiles, trial blocks) and runs in groups of
// kGroupBlocks trial blocks, blocks fastest within a group and then time tiles, so that
// each group reads the input about once from DRAM (and its blocks' stage records from
// L2) instead of each trial block re-reading the input.
constexpr int kGroupBlocks = 16;
template <typename TIN, bool PAIR, int NBUF, int SHORT>
__global__ void __launch_bounds__(kWarps * 32, 2) k_dedisp(DedispArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ TileState ts;
    if (threadIdx.x == 0) init_pipeline<NBUF>(pipeline_area(smem, a.smem_bytes, NBUF), ts);
    __syncthreads();
    if constexpr (std::is_same<TIN, uint32_t>::value) {
        dedisp_tile<TIN, PAIR, NBUF, false, SHORT>(a, smem, blockIdx.x, blockIdx.y, ts);
    } else {
        const int ntile = (int)gridDim.x, nblk = (int)gridDim.y;
        const int L = (int)blockIdx.y * ntile + (int)blockIdx.x;  // < 2^31: grid.y <= 65535
        const int g = L / (kGroupBlocks * ntile), r = L - g * kGroupBlocks * ntile;
        const int gb = min(kGroupBlocks, nblk - g * kGroupBlocks);
        dedisp_tile<TIN, PAIR, NBUF, false, SHORT>(a, smem, g * kGroupBlocks + r % gb, r / gb, ts);
    }
}

// Batched form: one CTA per work item (beam, trial block, time tile) of the list, in list
// order (beams by decreasing cost, each in the plain grid's tile order); the hardware
// starts CTAs in index order as earlier ones finish, which balances uneven beams.
// Measured on 36 beams: a persistent form whose CTAs took items from an atomic counter
// was 3.6 % slower (and slower than separate launches).
template <typename TIN, bool PAIR, int NBUF, int SHORT>
__global__ void __launch_bounds__(kWarps * 32, 2) k_dedisp_batched(const DedispArgs* beams,
                                                                    const BatchItem* items,
                                                                    uint32_t smem_bytes) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ TileState ts;
    __shared__ DedispArgs sa;
    if (threadIdx.x == 0) init_pipeline<NBUF>(pipeline_area(smem, smem_bytes, NBUF), ts);
    const BatchItem it = items[blockIdx.x];
    if (threadIdx.x == 0) {
        sa = beams[it.beam];
        sa.smem_bytes = smem_bytes;
    }
    __syncthreads();
    dedisp_tile<TIN, PAIR, NBUF, false, SHORT>(sa, smem, it.blk, it.tx, ts);
}

template <typename TIN, bool PAIR, int NBUF, int SHORT = 0>
dd_status run(DedispArgs a, cudaStream_t s) {
    const int nu = kWarps / a.nch * upw<TIN>();
    const size_t smem = smem_for<TIN, PAIR, NBUF>(a.lcap, a.kpad, a.cs, a.nch, a.nchan,
                                                  std::is_same<TIN, uint32_t>::value && SHORT != 0, a.blen);
    a.smem_bytes = (uint32_t)smem;
    auto kern = k_dedisp<TIN, PAIR, NBUF, SHORT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e);
    const int64_t tile = (int64_t)chunk_t(PAIR) * a.nch;
    const int db = (PAIR ? 2 : 1) * nu;
    const unsigned ntile = (unsigned)((a.t_out + tile - 1) / tile), nblk = (unsigned)((a.ndm + db - 1) / db);
    const bool blk_x = std::is_same<TIN, uint32_t>::value;
    dim3 grid(blk_x ? nblk : ntile, blk_x ? ntile : nblk, (unsigned)a.nsplit);
    if (grid.y > 65535 || a.nsplit < 1 || a.nsplit > 64) return DD_ERR_UNSUPPORTED;
    if ((int64_t)grid.x * grid.y >= INT32_MAX) return DD_ERR_UNSUPPORTED;  // the tile index is int
    kern<<<grid, kWarps * 32, smem, s>>>(a);
    return cuda_status(cudaGetLastError());
}

template <typename TIN, bool PAIR, int NBUF, int SHORT = 0>
dd_status run_batched(const DedispArgs* d_args, const BatchItem* d_items, int32_t nitems, size_t smem,
                      cudaStream_t s) {
    auto kern = k_dedisp_batched<TIN, PAIR, NBUF, SHORT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e);
    if (nitems < 1) return DD_OK;
    kern<<<(unsigned)nitems, kWarps * 32, smem, s>>>(d_args, d_items, (uint32_t)smem);
    return cuda_status(cudaGetLastError());
}

template <typename TIN, bool PAIR, int NBUF, int SHORT = 0>
int blocks_per_sm(size_t smem) {
    int n = 0;
    auto kern = k_dedisp_batched<TIN, PAIR, NBUF, SHORT>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kWarps * 32, smem) != cudaSuccess) return 0;
    return n;
}

// Builds the pair records' (w0, w1) weights from the device weights [d][c][kpad] and
// the tap table, at each entry's weight offset: tap k holds each trial's own tap k,
// zero past its taps (the entries themselves do not change).  One warp per entry.
__global__ void k_repack_w(const float* w, const int32_t* taps, unsigned char* rec, int32_t rec_bytes,
                           int32_t w_off, int32_t nchan, int32_t ndm, int32_t cs, int32_t nu,
                           int32_t kpad, int32_t nst) {
    const int rid = blockIdx.x;  // record = (block, stage)
    const int blk = rid / nst, st = rid - blk * nst;
    const int4* ent = (const int4*)(rec + (int64_t)rid * rec_bytes);
    float* dst = (float*)(rec + (int64_t)rid * rec_bytes + w_off);
    const int lane = threadIdx.x & 31;
    for (int e = threadIdx.x >> 5; e < nu * cs; e += blockDim.x >> 5) {
        const int j = e / cs, ci = e - j * cs;
        const int d0 = blk * 2 * nu + 2 * j, c = st * cs + ci;
        if (d0 >= ndm || c >= nchan) continue;
        const int4 q = ent[e];
        const int64_t dc0 = (int64_t)d0 * nchan + c, dc1 = dc0 + nchan;
        const int n0 = taps[dc0], n1 = d0 + 1 < ndm ? taps[dc1] : 0;
        for (int k = lane; k < q.y; k += 32) {
            dst[2 * (q.w + k)] = k < n0 ? w[dc0 * kpad + k] : 0.f;
            dst[2 * (q.w + k) + 1] = k < n1 ? w[dc1 * kpad + k] : 0.f;
        }
    }
}

// Run-length path, first step: per-channel prefix sums of the uint8 samples,
// P[c][i] = sum_{j<i} I[c][t_offset + j] for 0 <= i <= n (uint32; zero from n + 1 to
// the row's end).  One CTA per channel walks its row in blocks of 4096 samples: each
// thread sums 16 consecutive samples, a warp scan and a scan of the 8 warp totals
// place it, and the block total carries to the next block.
__global__ void __launch_bounds__(256) k_prefix(const uint8_t* in, int64_t ld, int64_t t_offset,
                                                int64_t n, uint32_t* P, int64_t ldp) {
    const int c = blockIdx.x;
    const uint8_t* row = in + (int64_t)c * ld + t_offset;
    uint32_t* prow = P + (int64_t)c * ldp;
    __shared__ uint32_t wsum[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool vec = (((uintptr_t)row) & 15) == 0;
    uint32_t carry = 0;
    int64_t end = 0;
    for (int64_t base = 0; base < n; base += 4096) {
        const int64_t i0 = base + 16 * tid;
        uint32_t v[16];
        if (vec && i0 + 16 <= n) {
            const uint4 q = *(const uint4*)(row + i0);
            const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = (w4[k >> 2] >> (8 * (k & 3))) & 0xffu;
        } else {
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = i0 + k < n ? (uint32_t)row[i0 + k] : 0u;
        }
        uint32_t sum = 0;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const uint32_t x = v[k];
            v[k] = sum;  // exclusive within the thread
            sum += x;
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        uint32_t before = 0, total = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const uint32_t x = wsum[w];
            before += w < warp ? x : 0u;
            total += x;
        }
        const uint32_t off = carry + before + incl - sum;
        if (i0 + 16 <= ldp) {
            uint4* dst = (uint4*)(prow + i0);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                uint4 o4;
                o4.x = i0 + 4 * k + 0 <= n ? off + v[4 * k + 0] : 0u;
                o4.y = i0 + 4 * k + 1 <= n ? off + v[4 * k + 1] : 0u;
                o4.z = i0 + 4 * k + 2 <= n ? off + v[4 * k + 2] : 0u;
                o4.w = i0 + 4 * k + 3 <= n ? off + v[4 * k + 3] : 0u;
                dst[k] = o4;
            }
        } else {
            for (int k = 0; k < 16 && i0 + k < ldp; ++k) prow[i0 + k] = i0 + k <= n ? off + v[k] : 0u;
        }
        carry += total;
        end = base + 4096;
        __syncthreads();  // wsum is rewritten by the next block
    }
    // P[n] when no block reached it, and the zero tail of the row
    if (tid == 0)
        for (int64_t i = end > n ? end : n; i < ldp; ++i) prow[i] = i == n ? carry : 0u;
}

}  // namespace


dd_status launch_repack(dd_plan_s* p, cudaStream_t s) {
    if (!p->pair) return DD_OK;
    const int nu = kWarps / p->nch;
    const int nst = (p->nchan + p->cs - 1) / p->cs;
    const StageGeom g(p->band.in_type == DD_U8 ? 1 : 4, true, p->lcap, p->kw, p->cs, nu);
    k_repack_w<<<p->nblk * nst, 256, 0, s>>>(p->dev.w, p->dev.taps, p->dev.rec, g.rec_bytes, g.w_off,
                                              p->nchan, p->ndm, p->cs, nu, p->kpad, nst);
    return cuda_status(cudaGetLastError());
}

void fill_dedisp_args(const dd_plan_s* p, const void* in, int64_t ld, int64_t t_offset,
                      int64_t t_out, void* out, int64_t out_ld, DedispArgs* a) {
    a->in = in;
    a->ld = ld;
    a->t_offset = t_offset;
    a->out = out;
    a->out_ld = out_ld;
    a->t_out = (int32_t)t_out;
    a->rec = p->dev.rec;
    a->blk_lo = p->dev.blk_lo;
    a->nchan = p->nchan;
    a->ndm = p->ndm;
    a->lcap = p->lcap;
    a->blen = p->blen;
    a->cs = p->cs;
    a->nch = p->nch;
    a->kpad = p->pair ? p->kw : 0;
    a->status = p->dev.status;
    a->skip_stage = p->debug_skip_stage;
    a->wait_ns = p->wait_ns;
    a->smem_bytes = (uint32_t)dedisp_smem_for(p);
    a->nsplit = 1;
    a->split_ld = 0;
}

size_t dedisp_smem_for(const dd_plan_s* p) {
    const int kp = p->pair ? p->kw : 0;
    if (p->rl) return smem_for<uint32_t, false, kStagesRl>(p->lcap, 0, p->cs, p->nch, p->nchan, p->rl_b, p->blen);
    if (!p->pair) return smem_for<uint8_t, false, kStagesInt>(p->lcap, kp, p->cs, p->nch, p->nchan);
    if (p->band.in_type == DD_U8) return smem_for<uint8_t, true, kStagesPair>(p->lcap, kp, p->cs, p->nch, p->nchan);
    return smem_for<float, true, kStagesPair>(p->lcap, kp, p->cs, p->nch, p->nchan);
}

dd_status launch_dedisperse(dd_plan_s* p, const void* in, int64_t ld, int64_t t_offset,
                            int64_t t_out, void* out, int64_t out_ld, cudaStream_t s, int nsplit,
                            int64_t split_ld) {
    DedispArgs a;
    fill_dedisp_args(p, in, ld, t_offset, t_out, out, out_ld, &a);
    a.nsplit = nsplit;
    a.split_ld = split_ld;
    const bool u8 = p->band.in_type == DD_U8;
    if (!p->pair)
        return p->kmax <= kRInt ? run<uint8_t, false, kStagesInt, 1>(a, s) : run<uint8_t, false, kStagesInt>(a, s);
    // union windows of at most R taps: one unrolled pass; at most 2R: two; longer: a loop
    const int passes = p->umax <= kRPair ? 1 : (p->umax <= 2 * kRPair ? 2 : 0);
    if (u8) {
        if (passes == 1) return run<uint8_t, true, kStagesPair, 1>(a, s);
        if (passes == 2) return run<uint8_t, true, kStagesPair, 2>(a, s);
        return run<uint8_t, true, kStagesPair>(a, s);
    }
    if (passes == 1) return run<float, true, kStagesPair, 1>(a, s);
    if (passes == 2) return run<float, true, kStagesPair, 2>(a, s);
    return run<float, true, kStagesPair>(a, s);
}

// Prefix sums of columns t_offset .. t_offset + nsamp - 1 into caller-owned P
// [nchan][ldp] (ldp >= nsamp + 1).
dd_status launch_prefix_into(const dd_plan_s* p, const void* in, int64_t ld, int64_t t_offset,
                             int64_t nsamp, uint32_t* P, int64_t ldp, cudaStream_t s) {
    k_prefix<<<p->nchan, 256, 0, s>>>((const uint8_t*)in, ld, t_offset, nsamp, P, ldp);
    return cuda_status(cudaGetLastError());
}

// Run-length path: prefix sums of columns t_offset .. t_offset + nsamp - 1 into the
// plan's scratch, then the run-length sums over them.
dd_status launch_prefix(dd_plan_s* p, const void* in, int64_t ld, int64_t t_offset, int64_t nsamp,
                        int64_t* ldp_out, cudaStream_t s) {
    const int64_t ldp = (nsamp + 1 + 3) & ~(int64_t)3;
    *ldp_out = ldp;
    const int64_t need = ldp * p->nchan;
    if (need > p->prefix_elems) {
        cudaFree(p->d_prefix);
        p->d_prefix = nullptr;
        p->prefix_elems = 0;
        cudaError_t e = cudaMalloc((void**)&p->d_prefix, (size_t)need * sizeof(uint32_t));
        if (e != cudaSuccess) return cuda_status(e);
        p->prefix_elems = need;
    }
    k_prefix<<<p->nchan, 256, 0, s>>>((const uint8_t*)in, ld, t_offset, nsamp, p->d_prefix, ldp);
    return cuda_status(cudaGetLastError());
}

dd_status launch_dedisperse_rl(dd_plan_s* p, const void* in, int64_t ld, int64_t t_offset,
                               int64_t nsamp, void* out, int64_t out_ld, cudaStream_t s) {
    int64_t ldp = 0;
    const dd_status st = launch_prefix(p, in, ld, t_offset, nsamp, &ldp, s);
    if (st != DD_OK) return st;
    DedispArgs a;
    fill_dedisp_args(p, p->d_prefix, ldp, 0, nsamp - p->dmax, out, out_ld, &a);
    return p->rl_b ? run<uint32_t, false, kStagesRl, 1>(a, s) : run<uint32_t, false, kStagesRl>(a, s);
}

dd_status launch_dedisperse_batched(bool u8, bool pair, bool short_taps, const DedispArgs* d_args,
                                    const BatchItem* d_items, int32_t nitems, size_t smem, cudaStream_t s,
                                    bool rl) {
    if (rl)  // run-length beams: short_taps = difference rows shared by the CTA
        return short_taps ? run_batched<uint32_t, false, kStagesRl, 1>(d_args, d_items, nitems, smem, s)
                          : run_batched<uint32_t, false, kStagesRl>(d_args, d_items, nitems, smem, s);
    if (!pair)
        return short_taps ? run_batched<uint8_t, false, kStagesInt, 1>(d_args, d_items, nitems, smem, s)
                          : run_batched<uint8_t, false, kStagesInt>(d_args, d_items, nitems, smem, s);
    if (u8)
        return short_taps ? run_batched<uint8_t, true, kStagesPair, 1>(d_args, d_items, nitems, smem, s)
                          : run_batched<uint8_t, true, kStagesPair>(d_args, d_items, nitems, smem, s);
    return short_taps ? run_batched<float, true, kStagesPair, 1>(d_args, d_items, nitems, smem, s)
                      : run_batched<float, true, kStagesPair>(d_args, d_items, nitems, smem, s);
}

int dedisp_batched_blocks_per_sm(bool u8, bool pair, bool short_taps, size_t smem, bool rl) {
    if (rl) return short_taps ? blocks_per_sm<uint32_t, false, kStagesRl, 1>(smem) : blocks_per_sm<uint32_t, false, kStagesRl>(smem);
    if (!pair) return short_taps ? blocks_per_sm<uint8_t, false, kStagesInt, 1>(smem) : blocks_per_sm<uint8_t, false, kStagesInt>(smem);
    if (u8) return short_taps ? blocks_per_sm<uint8_t, true, kStagesPair, 1>(smem) : blocks_per_sm<uint8_t, true, kStagesPair>(smem);
    return short_taps ? blocks_per_sm<float, true, kStagesPair, 1>(smem) : blocks_per_sm<float, true, kStagesPair>(smem);
}

}  // namespace dd
