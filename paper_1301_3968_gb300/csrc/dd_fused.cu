// Dedispersion fused with the boxcar S/N scan (eq. p_dedisp followed by eq. snr with
// boxcars, Sec. 5): the dedispersed series never leaves the chip.  The dedispersion
// CTAs scan their tiles in shared memory (dd_fused_scan.cuh); this file holds the fused
// kernel and its launcher, the pass over the windows that strip boundaries cut and the
// pass that turns the merged maxima into S/N.  Results equal dd_dedisperse followed by
// dd_boxcar_snr bit for bit: integer plans take the maximum of the same exact sums
// around the same per-trial offset, fp32 plans the same fp32 prefix-chain sums as the
// unfused fp32 scan, both with the earliest start, converted by the same normaliser.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cstdint>

#include "dd_internal.h"
#include "dd_tile.cuh"
#include "dd_trace.h"

namespace dd {
namespace {

// Fused dedispersion + boxcar scan, one CTA per part: part s walks the items (trial
// block, time tile) starts[s] .. starts[s + 1] - 1 in order (block-major), a strip per
// trial block it touches.  CTA i takes part order[i] (the hardware starts CTAs in index
// order as earlier ones finish; measured on the CRAFT-like block, parts handed out by an
// atomic counter to persistent CTAs ran 11 % slower, and a fixed round-robin 3 %).
// PAIR: fp32 pair units (fp32 sums, two trials per warp group).
template <typename TIN, bool PAIR, int NBUF, int SHORT>
__global__ void __launch_bounds__(kWarps * 32, 2) k_dedisp_fused(DedispArgs a, const FusedArgs f) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ TileState ts;
    if (threadIdx.x == 0) init_pipeline<NBUF>(pipeline_area(smem, a.smem_bytes, NBUF), ts);
    __syncthreads();
    // the tile's strip, kept in shared memory so that no per-strip state stays live in
    // registers across the channel sums (thread 0 writes it before each tile; the tile's
    // barriers order it, and the epilogue's last barrier ends its readers)
    __shared__ fused::FusedTile ft;
    const int s = (int)f.order[blockIdx.x];
    const int i0 = (int)f.starts[s], i1 = (int)f.starts[s + 1];  // items < 2^31 (host check)
    for (int it = i0; it < i1; ++it) {
        const int blk = it / f.tiles;
        const int tx = it - blk * f.tiles;
        if (threadIdx.x == 0) {
            const int L = chunk_t(PAIR) * a.nch;
            const int tpc = kWarps / a.nch * upw<TIN>() * (PAIR ? 2 : 1);
            const int tx0 = it - tx <= i0 ? i0 - (it - tx) : 0;                    // strip start
            const int tx1 = i1 - (it - tx) < f.tiles ? i1 - (it - tx) : f.tiles;  // strip end
            ft.first = tx == tx0;
            ft.last = tx == tx1 - 1;
            ft.s1 = min((int64_t)tx1 * L, (int64_t)a.t_out);
            ft.carry = f.carry + (int64_t)s * tpc * f.C;
            ft.seam_in = tx0 > 0 ? f.seam + (int64_t)s * tpc * 2 * f.C : nullptr;
            ft.seam_out = tx1 < f.tiles ? f.seam + (int64_t)(s + 1) * tpc * 2 * f.C : nullptr;
        }
        if (!dedisp_tile<TIN, PAIR, NBUF, true, SHORT, true>(a, smem, blk, tx, ts, &f, &ft)) break;
    }
}

template <typename TIN, bool PAIR, int NBUF, int SHORT>
dd_status run_fused(DedispArgs a, const FusedArgs& f, size_t smem, cudaStream_t s) {
    a.smem_bytes = (uint32_t)smem;
    auto kern = k_dedisp_fused<TIN, PAIR, NBUF, SHORT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e);
    kern<<<(unsigned)f.nparts, kWarps * 32, smem, s>>>(a, f);
    return cuda_status(cudaGetLastError());
}

template <typename TIN, bool PAIR, int NBUF, int SHORT>
int fused_bps(size_t smem) {
    int n = 0;
    auto kern = k_dedisp_fused<TIN, PAIR, NBUF, SHORT>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kWarps * 32, smem) != cudaSuccess) return 0;
    return n;
}


// Windows that cross the boundary between parts k-1 and k inside a trial block (start
// t < B < t + w, t + w <= t_out), one CTA per (boundary, trial of the block): the 2C
// outputs around B, a prefix over them, and per width the largest sum with its earliest
// start, merged into the key.
__global__ void __launch_bounds__(256) k_fused_seam(const FusedArgs f, int32_t L, int32_t t_out,
                                                    int32_t ndm, int32_t tpc) {
    extern __shared__ uint32_t pf[];  // [2C + 1]
    const int kb = blockIdx.x + 1, local = blockIdx.y;  // the boundary between parts kb - 1 and kb
    const int64_t item = f.starts[kb];
    const int blk = (int)(item / f.tiles);
    const int tx = (int)(item - (int64_t)blk * f.tiles);
    const int d = blk * tpc + local;
    if (tx == 0 || d >= ndm) return;  // a part boundary between blocks has no seam
    const int C = f.C;
    const int32_t* v = f.seam + ((int64_t)kb * tpc + local) * 2 * C;
    const int64_t B = (int64_t)tx * L;  // first output of part kb in this block
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < 32) {
        uint32_t carry = 0;
        if (lane == 0) pf[0] = 0;
        for (int k0 = 0; k0 < 2 * C; k0 += 32) {
            const int kl = k0 + lane;
            uint32_t x = kl < 2 * C ? (uint32_t)v[kl] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (kl < 2 * C) pf[kl + 1] = carry + x;
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
    }
    __syncthreads();
    const int64_t base = B - C;  // output of index 0 of the seam
    for (int j = tid; j < f.nw; j += blockDim.x) {
        const int w = f.w0 + j;
        int best = INT_MIN, bt = -1;
        for (int64_t t = B - w + 1; t < B; ++t) {
            if (t + w > t_out) break;
            const int ki = (int)(t - base);
            const int val = (int)(pf[ki + w] - pf[ki]);
            if (val > best) {
                best = val;
                bt = (int)t;
            }
        }
        if (bt >= 0) atomicMax(f.key + (int64_t)d * f.nw + j, fused_key(best, bt));
    }
}

// Merged (value, start) -> S/N exactly as the unfused boxcar kernel converts it.
__global__ void __launch_bounds__(256) k_fused_final(const unsigned long long* key, int32_t ndm, int32_t nw,
                                                     const float* mu, const float* isd, float* peak,
                                                     int32_t* arg, float thresh, dd_candidate* cands,
                                                     int32_t cap, int32_t* ncands) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)ndm * nw) return;
    const unsigned long long k = key[i];
    const int b = (int)((uint32_t)(k >> 32) ^ 0x80000000u);
    const int t = k ? (int)(0xffffffffu - (uint32_t)k) : -1;
    const float snr = (float)(((double)b - (double)mu[i]) * (double)isd[i]);
    peak[i] = snr;
    arg[i] = t;
    if (cands && snr > thresh) {
        const int c = atomicAdd(ncands, 1);
        if (c < cap) {
            dd_candidate cd;
            cd.dm_index = (int32_t)(i / nw);
            cd.width_index = (int32_t)(i % nw);
            cd.t = t;
            cd.snr = snr;
            cands[c] = cd;
        }
    }
}

// fp32 plans: the windows of the segments that begin before the boundary B between
// parts kb - 1 and kb inside a trial block and end past it (chain start m * kBoxSeg < B
// < t + w, t + w <= t_out), one CTA per (boundary, trial of the block), one thread per
// (segment, width): each forms the segment's prefix chain from the 2C outputs around B
// (C = wmax + kBoxSeg - 2 reaches back to the earliest such chain start) and merges the
// largest sum with its earliest start into the key.
__global__ void __launch_bounds__(128) k_fused_seam_f32(const FusedArgs f, int32_t L, int32_t t_out,
                                                        int32_t ndm, int32_t tpc) {
    constexpr int S = kBoxSeg;
    const int kb = blockIdx.x + 1, local = blockIdx.y;
    const int64_t item = f.starts[kb];
    const int blk = (int)(item / f.tiles);
    const int tx = (int)(item - (int64_t)blk * f.tiles);
    const int d = blk * tpc + local;
    if (tx == 0 || d >= ndm) return;  // a part boundary between blocks has no seam
    const int C = f.C;
    const float* v = (const float*)f.seam + ((int64_t)kb * tpc + local) * 2 * C;
    const int64_t B = (int64_t)tx * L;  // first output of part kb in this block
    const int64_t base = B - C;         // output of index 0 of the seam (>= 0: B >= L >= C)
    const int64_t m_lo = (base + S - 1) / S, m_hi = (B + S - 1) / S;
    const int nseg = (int)(m_hi - m_lo);
    const int64_t e_abs = min((int64_t)t_out, B + C);  // outputs at or past it are not read
    for (int i = threadIdx.x; i < nseg * f.nw; i += blockDim.x) {
        const int sg = i / f.nw, j = i - sg * f.nw;
        const int64_t t0 = (m_lo + sg) * S;
        const int w = f.w0 + j;
        const float* x = v + (t0 - base);
        const int e_rel = (int)(e_abs - t0);
        auto ld = [&](int k) { return k < e_rel ? x[k] : 0.f; };
        float r = 0.f, p = 0.f;
        for (int k = 0; k < w; ++k) r += ld(k);
        float best = -FLT_MAX;
        int bt = -1;
        for (int s = 0; s < S; ++s) {
            const int64_t t = t0 + s;
            if (t + w > t_out) break;
            if (t + w > B) {
                const float val = r - p;
                if (bt < 0 || val > best) {
                    best = val;
                    bt = (int)t;
                }
            }
            p += ld(s);
            r += ld(s + w);
        }
        if (bt >= 0) atomicMax(f.key + (int64_t)d * f.nw + j, fused_key_f32(best, bt));
    }
}

// Merged (value, start) of fp32 plans -> S/N exactly as the unfused boxcar kernel
// converts it.
__global__ void __launch_bounds__(256) k_fused_final_f32(const unsigned long long* key, int32_t ndm,
                                                         int32_t nw, const float* mu, const float* isd,
                                                         float* peak, int32_t* arg, float thresh,
                                                         dd_candidate* cands, int32_t cap, int32_t* ncands) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)ndm * nw) return;
    const unsigned long long k = key[i];
    const float b = k ? fused_key_value_f32(k) : -FLT_MAX;
    const int t = k ? (int)(0xffffffffu - (uint32_t)k) : -1;
    const float snr = (float)(((double)b - (double)mu[i]) * (double)isd[i]);
    peak[i] = snr;
    arg[i] = t;
    if (cands && snr > thresh) {
        const int c = atomicAdd(ncands, 1);
        if (c < cap) {
            dd_candidate cd;
            cd.dm_index = (int32_t)(i / nw);
            cd.width_index = (int32_t)(i % nw);
            cd.t = t;
            cd.snr = snr;
            cands[c] = cd;
        }
    }
}

template <typename T>
dd_status grow(T** buf, int64_t* have, int64_t need) {
    if (need <= *have) return DD_OK;
    cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    cudaError_t e = cudaMalloc((void**)buf, (size_t)std::max<int64_t>(need, 1) * sizeof(T));
    if (e != cudaSuccess) return cuda_status(e);
    *have = need;
    return DD_OK;
}

// Cuts the items (block-major, `tiles` per block) into nparts contiguous, non-empty
// parts of about equal cost.  A tile of block b costs cost[b] (the last tile of every
// block `last_frac` of that); parts start where the cumulative cost crosses s / nparts
// of the total.
std::vector<int64_t> cut_parts(const std::vector<double>& cost, int tiles, double last_frac, int nparts) {
    const int64_t nblk = (int64_t)cost.size();
    const int64_t n = nblk * tiles;
    std::vector<double> cum(nblk + 1, 0.0);
    const double per_blk_tiles = tiles - 1 + last_frac;
    for (int64_t b = 0; b < nblk; ++b) cum[b + 1] = cum[b] + cost[b] * per_blk_tiles;
    std::vector<int64_t> st(nparts + 1);
    st[0] = 0;
    st[nparts] = n;
    int64_t b = 0;
    for (int s = 1; s < nparts; ++s) {
        const double target = cum[nblk] * s / nparts;
        while (b + 1 < nblk && cum[b + 1] <= target) ++b;
        const double in = cost[b] > 0 ? (target - cum[b]) / cost[b] : 0.0;
        int64_t it = b * tiles + std::min<int64_t>(tiles - 1, std::max<int64_t>(0, (int64_t)(in + 0.5)));
        it = std::max(it, st[s - 1] + 1);
        it = std::min(it, n - (nparts - s));
        st[s] = it;
    }
    return st;
}

// Cuts every trial block into nseg segments at the same time tiles (the block-major
// items stay contiguous per part), and orders the CTAs segment by segment, so that the
// CTAs resident together work on the same time tiles of different trial blocks and stage
// the same input columns, which then come from L2.  Returns the parts' first items
// (plus the end) and the launch order (CTA i takes part order[i]).
void aligned_parts(int64_t nblk, int tiles, int nseg, std::vector<int64_t>* starts,
                   std::vector<int64_t>* order) {
    starts->clear();
    for (int64_t b = 0; b < nblk; ++b)
        for (int k = 0; k < nseg; ++k) starts->push_back(b * tiles + (int64_t)tiles * k / nseg);
    starts->push_back(nblk * tiles);
    order->clear();
    for (int k = 0; k < nseg; ++k)
        for (int64_t b = 0; b < nblk; ++b) order->push_back(b * nseg + k);
}

// aligned_parts' cut with the blocks taken gb at a time: within a group of gb blocks the
// parts go segment by segment, and the groups one after another, so that the CTAs
// working together stay on about gb blocks (whose stage records then stay in L2).
void grouped_parts(int64_t nblk, int tiles, int nseg, int64_t gb, std::vector<int64_t>* starts,
                   std::vector<int64_t>* order) {
    aligned_parts(nblk, tiles, nseg, starts, order);
    order->clear();
    for (int64_t g0 = 0; g0 < nblk; g0 += gb)
        for (int k = 0; k < nseg; ++k)
            for (int64_t b = g0; b < std::min(nblk, g0 + gb); ++b) order->push_back(b * nseg + k);
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

constexpr int64_t kFusedGroup = 16;  // trial blocks per group of fp32 fused parts

}  // namespace

size_t fused_smem_for(const dd_plan_s* p, int rowlen, int C) {
    const int nbuf = p->rl ? kStagesRl : (p->pair ? kStagesPair : kStagesInt);
    // fp32 pair units: a row per trial; run-length path: a row per warp group and the
    // group's other trials' sums
    const int nrow = kWarps / p->nch * (p->pair ? 2 : 1);
    // and the warps' scratch of the earliest-start search
    const int spill = (p->rl ? kWarps * (kRlUnits - 1) * chunk_t(false) : 0) + kWarps * fused::kChainFloats;
    const size_t rows = (size_t)(fused_rows_ints(nrow, rowlen, C) + spill) * 4 + nbuf * 8 + 2 * nbuf * 4;
    return (std::max(dedisp_smem_for(p), rows) + 15) & ~(size_t)15;
}

// Pair path: union windows of at most R taps, one unrolled pass; at most 2R, two; longer,
// a loop (as the plain launch).
int pair_passes(const dd_plan_s* p) { return p->umax <= kRPair ? 1 : (p->umax <= 2 * kRPair ? 2 : 0); }

int fused_blocks_per_sm(const dd_plan_s* p, size_t smem) {
    if (p->rl) return p->rl_b ? fused_bps<uint32_t, false, kStagesRl, 1>(smem) : fused_bps<uint32_t, false, kStagesRl, 0>(smem);
    if (p->pair) {
        const int np = pair_passes(p);
        if (p->band.in_type == DD_U8)
            return np == 1 ? fused_bps<uint8_t, true, kStagesPair, 1>(smem)
                           : (np == 2 ? fused_bps<uint8_t, true, kStagesPair, 2>(smem) : fused_bps<uint8_t, true, kStagesPair, 0>(smem));
        return np == 1 ? fused_bps<float, true, kStagesPair, 1>(smem)
                       : (np == 2 ? fused_bps<float, true, kStagesPair, 2>(smem) : fused_bps<float, true, kStagesPair, 0>(smem));
    }
    return p->kmax <= kRInt ? fused_bps<uint8_t, false, kStagesInt, 1>(smem) : fused_bps<uint8_t, false, kStagesInt, 0>(smem);
}

dd_status launch_dedisperse_fused(const dd_plan_s* p, DedispArgs a, const FusedArgs& f, size_t smem,
                                  cudaStream_t s) {
    if (p->rl)
        return p->rl_b ? run_fused<uint32_t, false, kStagesRl, 1>(a, f, smem, s) : run_fused<uint32_t, false, kStagesRl, 0>(a, f, smem, s);
    if (p->pair) {
        const int np = pair_passes(p);
        if (p->band.in_type == DD_U8)
            return np == 1 ? run_fused<uint8_t, true, kStagesPair, 1>(a, f, smem, s)
                           : (np == 2 ? run_fused<uint8_t, true, kStagesPair, 2>(a, f, smem, s)
                                      : run_fused<uint8_t, true, kStagesPair, 0>(a, f, smem, s));
        return np == 1 ? run_fused<float, true, kStagesPair, 1>(a, f, smem, s)
                       : (np == 2 ? run_fused<float, true, kStagesPair, 2>(a, f, smem, s)
                                  : run_fused<float, true, kStagesPair, 0>(a, f, smem, s));
    }
    return p->kmax <= kRInt ? run_fused<uint8_t, false, kStagesInt, 1>(a, f, smem, s)
                            : run_fused<uint8_t, false, kStagesInt, 0>(a, f, smem, s);
}

}  // namespace dd

extern "C" dd_status dd_dedisperse_boxcar(dd_plan_t p, const void* in, int64_t in_ld, int64_t t_offset,
                                          int64_t nsamp, const int32_t* widths, int32_t nw,
                                          const double* mean, const double* sd, float* peak,
                                          int32_t* arg, float thresh, dd_candidate* cands,
                                          int32_t cap, int32_t* ncands, void* stream) {
    DD_TRACE("dd_dedisperse_boxcar");
    dd::log_msg(2, "dd_dedisperse_boxcar: %d trials, t_offset %lld, nsamp %lld, %d widths", p ? p->ndm : 0, (long long)t_offset, (long long)nsamp, nw);
    using namespace dd;
    if (!p || !in || !widths || nw < 1 || !mean || !sd || !peak || !arg) return DD_ERR_ARG;
    if (cands && (!ncands || cap < 0)) return DD_ERR_ARG;
    if (nsamp <= 0) nsamp = p->band.nsamp;
    if (t_offset < 0 || nsamp <= p->dmax || t_offset + nsamp > in_ld) return DD_ERR_ARG;
    const int64_t t_out = nsamp - p->dmax;
    for (int i = 0; i < nw; ++i) {
        if (widths[i] < 1 || widths[i] > t_out) return DD_ERR_ARG;
        if (i && widths[i] <= widths[i - 1]) return DD_ERR_ARG;
    }
    const bool fp = p->pair;  // fp32 sums (fp32 input, or weighted uint8)
    if (!fp && (p->band.in_type != DD_U8 || !p->out_int)) return DD_ERR_UNSUPPORTED;
    if (widths[nw - 1] - widths[0] != nw - 1) return DD_ERR_UNSUPPORTED;  // w_j = w_0 + j only
    const int L = chunk_t(fp) * p->nch;
    // carried outputs: the longest window (integer), or back to its prefix chain's start
    const int C = fp ? widths[nw - 1] + kBoxSeg - 2 : widths[nw - 1] - 1;
    if (C > L) return DD_ERR_UNSUPPORTED;
    const int64_t esz = p->band.in_type == DD_U8 ? 1 : 4;
    if (!aligned16(in) || (in_ld * esz) % 16 != 0) return DD_ERR_ARG;
    if (t_out > INT32_MAX - chunk_t(fp) * kWarps || in_ld > (int64_t)1 << 40) return DD_ERR_OVERFLOW;
    if (p->rl && nsamp > ((int64_t)1 << 24)) return DD_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    dd_status st = upload_tables(p);
    if (st != DD_OK) return st;
    if ((st = launch_norm(p, widths, nw, mean, sd, s)) != DD_OK) return st;

    DedispArgs a;
    if (p->rl) {
        int64_t ldp = 0;
        if ((st = launch_prefix(p, in, in_ld, t_offset, nsamp, &ldp, s)) != DD_OK) return st;
        fill_dedisp_args(p, p->d_prefix, ldp, 0, t_out, nullptr, 0, &a);
    } else {
        fill_dedisp_args(p, in, in_ld, t_offset, t_out, nullptr, 0, &a);
    }
    const int tiles = (int)((t_out + L - 1) / L);
    const int tpc = kWarps / p->nch * (p->rl ? kRlUnits : 1) * (fp ? 2 : 1);
    const int64_t nblk = (p->ndm + tpc - 1) / tpc;
    // row: C carried outputs, the tile and 32 spare (fp32: 48); the last tile's extra
    // starts read up to C + 14 past a row (fp32: 15 past the row's windows), into the
    // next one or the padding behind the last
    const int rowlen = L + C + (fp ? 48 : 32);
    const size_t smem = fused_smem_for(p, rowlen, C);
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_status(e);
    const int bps = fused_blocks_per_sm(p, smem);
    if (bps < 1) return DD_ERR_UNSUPPORTED;
    const int64_t nitems = nblk * tiles;
    if (nitems >= INT32_MAX) return DD_ERR_UNSUPPORTED;
    // k parts per resident CTA, k = items / (16 x resident CTAs) clamped to 1..8: parts of
    // at least ~16 tiles, so that the seams and carry-less first tiles stay a small share
    // (measured on the large low-band block: 2.4k-2.7k parts beat 300 and 11k)
    const int64_t slots = (int64_t)bps * nsm;
    const int64_t k_per = std::max<int64_t>(1, std::min<int64_t>(8, nblk * tiles / (16 * slots)));
    std::vector<int64_t> starts, order;
    int nparts = 0;
    if (p->debug_fused_parts > 0) {
        // test hook: that many parts of about equal cost, in block-major order (cost of a
        // tile: constant on the run-length path, the block's taps plus a per-channel
        // constant on the direct path)
        nparts = (int)std::min<int64_t>(p->debug_fused_parts, nitems);
        std::vector<double> cost((size_t)nblk, 1.0);
        if (!p->rl)
            for (int64_t b = 0; b < nblk; ++b) {
                double c = 0.0;
                for (int64_t d = b * tpc; d < std::min<int64_t>((b + 1) * tpc, p->ndm); ++d)
                    for (int ch = 0; ch < p->nchan; ++ch) c += p->taps[(size_t)d * p->nchan + ch] + 4.0;
                cost[(size_t)b] = c;
            }
        const double last_frac = (double)(t_out - (int64_t)(tiles - 1) * L) / L;
        starts = cut_parts(cost, tiles, last_frac, nparts);
        for (int i = 0; i < nparts; ++i) order.push_back(i);
    } else if (fp) {
        // fp32 stage records hold every tap's weight pair (544 kB per 16-trial block of the
        // CRAFT-like list), so the CTAs working together must share few blocks: groups of
        // kFusedGroup blocks, each block cut into as many segments as fill the resident CTAs
        const int64_t gb = std::min<int64_t>(nblk, kFusedGroup);
        const int nseg = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (slots + gb - 1) / gb));
        grouped_parts(nblk, tiles, nseg, gb, &starts, &order);
        nparts = (int)(starts.size() - 1);
    } else {
        // up to k_per parts per resident CTA, every block cut at the same time tiles and
        // taken segment by segment, so that the CTAs working together stage the same input
        // columns (from L2)
        const int nseg = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, k_per * slots / nblk));
        aligned_parts(nblk, tiles, nseg, &starts, &order);
        nparts = (int)(starts.size() - 1);
    }
    if ((int64_t)nparts * tpc * 2 * C >= INT32_MAX || nparts < 1) return DD_ERR_UNSUPPORTED;
    log_msg(1, "fused scan: %s sums, %d parts of %lld tiles (%lld trial blocks x %d), %d CTAs per SM, "
            "carry %d, %zu bytes of shared memory", fp ? "fp32" : "integer", nparts,
            (long long)(nitems / nparts), (long long)nblk, tiles, bps, C, smem);
    starts.insert(starts.end(), order.begin(), order.end());  // one table: starts, then order

    FusedArgs f;
    f.w0 = widths[0];
    f.nw = nw;
    f.C = C;
    f.rowlen = rowlen;
    f.nparts = nparts;
    f.tiles = tiles;
    f.mlim = INT_MAX / widths[nw - 1];
    f.off = p->dev.off;
    int64_t have_starts = (int64_t)p->fstarts.size();
    if (starts != p->fstarts) {
        if ((int64_t)starts.size() > have_starts || !p->d_fstarts) {
            cudaFree(p->d_fstarts);
            p->d_fstarts = nullptr;
            p->fstarts.clear();
            if ((e = cudaMalloc((void**)&p->d_fstarts, starts.size() * sizeof(int64_t))) != cudaSuccess)
                return cuda_status(e);
        }
        e = cudaMemcpyAsync(p->d_fstarts, starts.data(), starts.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_status(e);
        p->fstarts = starts;
    }
    f.starts = p->d_fstarts;
    f.order = p->d_fstarts + nparts + 1;
    if ((st = grow(&p->d_fkey, &p->fkey_elems, (int64_t)p->ndm * nw)) != DD_OK) return st;
    if ((st = grow(&p->d_fcarry, &p->fcarry_elems, (int64_t)nparts * tpc * C)) != DD_OK) return st;
    if ((st = grow(&p->d_fseam, &p->fseam_elems, (int64_t)nparts * tpc * 2 * C)) != DD_OK) return st;
    f.key = p->d_fkey;
    f.carry = p->d_fcarry;
    f.seam = p->d_fseam;
    e = cudaMemsetAsync(f.key, 0, (size_t)p->ndm * nw * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_status(e);
    if ((st = launch_dedisperse_fused(p, a, f, smem, s)) != DD_OK) return st;
    if (nparts > 1 && fp) {
        k_fused_seam_f32<<<dim3((unsigned)(nparts - 1), (unsigned)tpc), 128, 0, s>>>(f, L, (int32_t)t_out,
                                                                                   p->ndm, tpc);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    } else if (nparts > 1 && C > 0) {
        k_fused_seam<<<dim3((unsigned)(nparts - 1), (unsigned)tpc), 256, (size_t)(2 * C + 1) * 4, s>>>(
            f, L, (int32_t)t_out, p->ndm, tpc);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    }
    const int64_t n = (int64_t)p->ndm * nw;
    const unsigned nb = (unsigned)((n + 255) / 256);
    if (fp)
        k_fused_final_f32<<<nb, 256, 0, s>>>(f.key, p->ndm, nw, p->dev.mu, p->dev.isd, peak, arg, thresh, cands,
                                             cap, ncands);
    else
        k_fused_final<<<nb, 256, 0, s>>>(f.key, p->ndm, nw, p->dev.mu, p->dev.isd, peak, arg, thresh, cands,
                                         cap, ncands);
    return cuda_status(cudaGetLastError());
}

extern "C" dd_status dd_test_set_fused_parts(dd_plan_t p, int32_t nparts) {
    if (!p || nparts < 0) return DD_ERR_ARG;
    p->debug_fused_parts = nparts;
    return DD_OK;
}
