// Device side of the dedispersion tile (eq. p_dedisp, Sec. 2.1), shared by the plain,
// batched and fused kernels (dd_dedisp.cu, dd_fused.cu).  Every definition sits in an
// unnamed namespace: each translation unit that includes it has its own copy.
//
// Profiled dedispersion, eq. p_dedisp (Sec. 2.1):
//
//   out[d][t] = sum_c sum_{k < n_dc} w_dck * I[c][t_offset + t + delta_dc + k]
//
// Work decomposition (sm_103a):
//   * A CTA has kWarps = 8 warps covering 8 / nch warp-groups x nch time chunks.  On the
//     fp32 path a warp unit sums two adjacent trials from one shared register window
//     whose registers hold each trial's own sample (their delays differ by a few samples
//     at most on a trial list of eq. trial DMs); on the exact integer path a warp sums
//     one trial, on the run-length path three.  A chunk is 32 * R outputs and lane l
//     owns outputs chunk_start + l*R + r, r < R (R = kRPair on the pair path, kRInt
//     otherwise).  The plan picks the most trials per CTA whose staged window fits in
//     shared memory.
//   * Channels are streamed in stages of cs rows through a ring of NBUF shared-memory
//     buffers (two on the pair and run-length paths, four on the integer path).  For each
//     channel the CTA stages the window that all its trials read -- [T0 + min delta,
//     T0 + tile + max(delta + n)) rounded to 16-byte chunks -- with one bulk copy
//     (cp.async.bulk, the TMA engine), plus one bulk copy of the stage's profile record
//     (window starts, taps, weights).  Each buffer has a full mbarrier that counts the
//     copied bytes.
//   * Warps do not synchronise with each other per stage: after consuming a buffer each
//     warp increments the buffer's counter, and the last of the 8 refills it with the
//     stage NBUF ahead.  A warp can run up to NBUF-1 stages ahead of the slowest one.  (The
//     run-length path with shared difference rows is the exception: the CTA builds the
//     rows together, with one barrier per stage.)
//   * Every wait is bounded by time; a wait that runs out records DD_ERR_TIMEOUT in the
//     plan's status word, the CTA drains its own copies in flight and returns.
//   * Inner loop: a register window of R samples slides along the taps.  Pair path: per
//     tap one or two shared-memory loads, one weight-pair broadcast and R packed FMAs
//     (fma.rn.f32x2, 2 x R fp32 FMAs).  Integer path: per two taps one load and R
//     three-input adds.  Run-length path: per output two loads and one add (one load with
//     shared difference rows), whatever the tap count.  R is odd, so the lane-strided
//     loads hit 32 distinct banks.
//   * Sums run over channels, then taps, in a fixed order, so results are
//     deterministic.
//   * Results are transposed through shared memory so that global stores coalesce.
#pragma once

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "dd_debug.cuh"
#include "dd_internal.h"
#include "dd_packed.cuh"
#include "dd_fused_scan.cuh"

namespace dd {
namespace {

__device__ __forceinline__ uint32_t su32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(su32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
// Waits for the phase of `bar` with the given parity, for at most limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if ((int64_t)(global_ns() - t0) > limit_ns) return false;
    }
    return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            su32(dst)),
        "l"(src), "r"(bytes), "r"(su32(bar))
        : "memory");
}

template <typename TIN>
struct Elem;
template <>
struct Elem<uint8_t> {
    static constexpr int Q = 16;  // elements per 16-byte chunk
};
template <>
struct Elem<float> {
    static constexpr int Q = 4;
};
template <>
struct Elem<uint32_t> {  // prefix sums of the run-length path
    static constexpr int Q = 4;
};

// Warp units per warp: kRlUnits trials on the run-length path (staged rows of uint32
// prefix sums), one unit otherwise.
template <typename TIN>
__host__ __device__ constexpr int upw() {
    return std::is_same<TIN, uint32_t>::value ? kRlUnits : 1;
}

template <typename TACC, typename TIN>
__device__ __forceinline__ TACC cvt(TIN v) {
    return (TACC)v;
}

// Packed pairs for the fp32 pair units (dd_packed.cuh): one 64-bit register holds
// (trial 0, trial 1) accumulators, weights or window samples, and one fma.rn.f32x2
// performs both trials' fused multiply-adds.

struct Smem {
    unsigned char* stages;
    int* lo_all;
    uint32_t* brows;  // difference rows (run-length path with shared rows)
    uint64_t* full;
    int* cnt;
    int* issued;
};

__device__ __forceinline__ unsigned char* pipeline_area(unsigned char* smem, size_t smem_bytes, int nbuf);

template <int NBUF>
__device__ __forceinline__ Smem carve(unsigned char* smem, const StageGeom& g, size_t smem_bytes,
                                      int nchan) {
    Smem s;
    s.stages = smem;
    s.lo_all = (int*)(smem + NBUF * g.bytes);
    s.brows = (uint32_t*)(smem + NBUF * g.bytes + ((4 * nchan + 15) & ~15));
    s.full = (uint64_t*)pipeline_area(smem, smem_bytes, NBUF);
    s.cnt = (int*)(s.full + NBUF);
    s.issued = s.cnt + NBUF;
    return s;
}

// Issues the bulk copies of stage `stage` into buffer `b` (one thread).  In the common
// case every staged window lies inside its row and each channel is one full-length
// copy; CTAs whose windows run past the end of the rows (`tail`) zero the missing part
// first and copy only what exists.
template <typename TIN, int NBUF>
__device__ void issue_stage(const DedispArgs& a, const StageGeom& g, const Smem& sm, int blk,
                            int stage, int b, int64_t base, bool tail) {
    constexpr int Q = Elem<TIN>::Q;
    if (stage == a.skip_stage) return;  // test hook: this stage is never filled
    unsigned char* buf = sm.stages + b * g.bytes;
    const int c0 = stage * a.cs;
    const int csn = min(a.cs, a.nchan - c0);
    const TIN* in = (const TIN*)a.in;
    const int nst = (a.nchan + a.cs - 1) / a.cs;
    const unsigned char* rec = a.rec + ((int64_t)blk * nst + stage) * g.rec_bytes;
    const uint32_t row_bytes = (uint32_t)a.lcap * sizeof(TIN);
    if (kDebug) {  // every copied window inside its row and its stage buffer
        bool ok = (int64_t)csn * row_bytes <= g.rows_bytes && c0 >= 0 && csn > 0;
        for (int ci = 0; ci < csn; ++ci) {
            const int64_t a0 = (base + sm.lo_all[c0 + ci]) & ~(int64_t)(Q - 1);
            ok = ok && a0 >= 0 && (tail || a0 + a.lcap <= a.ld);
        }
        if (!dbg_ok(ok, a.status)) {  // complete the phase without copies
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(su32(&sm.full[b])) : "memory");
            sm.issued[b] += 1;
            return;
        }
    }
    if (!tail) {
        mbar_expect_tx(&sm.full[b], (uint32_t)csn * row_bytes + g.rec_bytes);
        for (int ci = 0; ci < csn; ++ci) {
            const int c = c0 + ci;
            const int64_t a0 = (base + sm.lo_all[c]) & ~(int64_t)(Q - 1);
            bulk_g2s(buf + ci * row_bytes, in + (int64_t)c * a.ld + a0, row_bytes, &sm.full[b]);
        }
        bulk_g2s(buf + g.rec_off, rec, (uint32_t)g.rec_bytes, &sm.full[b]);
        sm.issued[b] += 1;
        return;
    }
    uint32_t bytes = g.rec_bytes;
    // zero the parts of the windows past the end of the rows first (generic stores,
    // published by the barrier's arrive below)
    for (int ci = 0; ci < csn; ++ci) {
        const int64_t a0 = (base + sm.lo_all[c0 + ci]) & ~(int64_t)(Q - 1);
        const int64_t nin = max((int64_t)0, min((int64_t)a.lcap, a.ld - a0));
        if (nin < a.lcap) {
            uint4* z = (uint4*)(buf + ((int64_t)ci * a.lcap + nin) * sizeof(TIN));
            const int nz = (int)((a.lcap - nin) * sizeof(TIN) / 16);
            for (int i = 0; i < nz; ++i) z[i] = make_uint4(0, 0, 0, 0);
        }
        bytes += (uint32_t)(nin * sizeof(TIN));
    }
    fence_proxy_async();
    mbar_expect_tx(&sm.full[b], bytes);
    for (int ci = 0; ci < csn; ++ci) {
        const int c = c0 + ci;
        const int64_t a0 = (base + sm.lo_all[c]) & ~(int64_t)(Q - 1);
        const int64_t nin = max((int64_t)0, min((int64_t)a.lcap, a.ld - a0));
        if (nin > 0)
            bulk_g2s(buf + (int64_t)ci * a.lcap * sizeof(TIN), in + (int64_t)c * a.ld + a0,
                     (uint32_t)(nin * sizeof(TIN)), &sm.full[b]);
    }
    bulk_g2s(buf + g.rec_off, rec, (uint32_t)g.rec_bytes, &sm.full[b]);
    sm.issued[b] += 1;
}

// One stage of one warp unit, exact integer sums of uint8 samples with unit weights:
// for each of the stage's channels a register window of R samples slides along the
// taps.  At tap k output r reads window sample r + k, held in register (r + k) mod R;
// after the tap, sample k (no longer needed) is replaced by sample k + R.  Taps go two
// at a time, one three-input add per output (the second tap's last output reads sample
// R + k, loaded before the add).  SHORT: no tap run is longer than R, one unrolled pass.
template <typename TIN, int SHORT>
__device__ __forceinline__ void stage_int(const TIN* rows, const int2* ent, const int* lo,
                                          int csn, int lcap, int bq, int lane_off,
                                          int (&acc)[kRInt], int32_t* status) {
    constexpr int Q = Elem<TIN>::Q;
    constexpr int R = kRInt;
    for (int ci = 0; ci < csn; ++ci) {
        const int2 q = ent[ci];  // (window start - block minimum, taps)
        const int n = q.y;
        const int i0 = ((bq + lo[ci]) & (Q - 1)) + q.x + lane_off;
        if (!dbg_ok(q.x >= 0 && n >= 1 && i0 + R + n <= lcap, status)) continue;
        const TIN* p = rows + ci * lcap + i0;
        __builtin_assume(__isShared(p));
        int win[R];
#pragma unroll
        for (int j = 0; j < R; ++j) win[j] = (int)p[j];
        for (int k0 = 0; k0 < (SHORT == 1 ? 1 : n); k0 += R) {
#pragma unroll
            for (int kk = 0; kk < R; kk += 2) {
                if (k0 + kk >= n) break;
                if (kk + 1 < R && k0 + kk + 1 < n) {
                    const int nk = (int)p[R + k0 + kk];
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        acc[r] += win[(r + kk) % R] + (r == R - 1 ? nk : win[(r + kk + 1) % R]);
                    win[kk] = nk;
                    win[kk + 1] = (int)p[R + k0 + kk + 1];
                } else {
#pragma unroll
                    for (int r = 0; r < R; ++r) acc[r] += win[(r + kk) % R];
                    win[kk] = (int)p[R + k0 + kk];
                }
            }
        }
    }
}

// One stage of one warp unit on the run-length path (uint8 samples, unit weights): the
// staged rows hold the channels' prefix sums P[i] = sum_{j<i} I[j], and the unit's n
// taps starting at delta sum to P[t + delta + n] - P[t + delta].  Two loads and one
// add per output whatever n is; the uint32 difference is exact (taken modulo 2^32 and
// at most 255 n).
__device__ __forceinline__ void stage_rl(const uint32_t* rows, const int2* ent, const int* lo,
                                         int csn, int lcap, int bq, int lane_off, int (&acc)[kRInt],
                                         int32_t* status) {
    constexpr int R = kRInt;
    for (int ci = 0; ci < csn; ++ci) {
        const int2 q = ent[ci];  // (run start - block minimum, taps)
        const int i0 = ((bq + lo[ci]) & 3) + q.x + lane_off;
        if (!dbg_ok(q.x >= 0 && q.y >= 1 && i0 + q.y + R <= lcap, status)) continue;
        const uint32_t* p = rows + ci * lcap + i0;
        const uint32_t* pe = p + q.y;
        __builtin_assume(__isShared(p));
        __builtin_assume(__isShared(pe));
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] += (int)(pe[r] - p[r]);
    }
}

// The same sums from difference rows the CTA has built for the stage: brows holds, per
// channel, B_q[i] = P[i + n_q] - P[i] for the block's (at most two) tap counts n_q, and
// the unit's entry is (run start, q).  One load and one add per output.
__device__ __forceinline__ void stage_rl_rows(const uint32_t* brows, const int2* ent, const int* lo,
                                              int csn, int lcap, int bq, int lane_off, int (&acc)[kRInt],
                                              int32_t* status) {
    constexpr int R = kRInt;
    for (int ci = 0; ci < csn; ++ci) {
        const int2 q = ent[ci];  // (run start - block minimum, index of the tap count)
        const int i0 = ((bq + lo[ci]) & 3) + q.x + lane_off;
        if (!dbg_ok(q.x >= 0 && (q.y == 0 || q.y == 1) && i0 + R <= lcap, status)) continue;
        const uint32_t* p = brows + (ci * 2 + q.y) * lcap + i0;
        __builtin_assume(__isShared(p));
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] += (int)p[r];
    }
}

// One channel of a pair unit on the fp32 path: two adjacent trials share the register
// window.  Window register j holds (sample j of trial 0's run, sample j of trial 1's
// run) -- the same sample duplicated when the runs start together (SHIFT false), else
// the two samples s apart -- and the weights are (w0, w1) pairs, zero past a trial's
// own taps, so each tap costs one weight-pair broadcast, one or two window loads and R
// packed FMAs (2 x R fp32 FMAs) for max(n0, n1) taps.  SHORT: the plan's units have at
// most R taps (one unrolled pass) or 2R (two passes).  Sums run over channels, then
// taps, in a fixed order (deterministic); single-precision accumulation of the
// ~10^3-10^4 terms of an output stays orders of magnitude inside the 1e-5 scale-aware
// bound.
template <typename TIN, int SHORT, bool SHIFT>
__device__ __forceinline__ void pair_channel(const TIN* p, int s, int n, const uint64_t* wk,
                                             uint64_t (&acc)[kRPair]) {
    constexpr int R = kRPair;
    const TIN* p2 = p + s;  // trial 1's run
    auto ld = [&](int j) -> uint64_t {
        if constexpr (SHIFT) return pk2((float)p[j], (float)p2[j]);
        else return pk_dup((float)p[j]);
    };
    uint64_t win[R];
#pragma unroll
    for (int j = 0; j < R; ++j) win[j] = ld(j);
    if constexpr (SHORT == 1) {
#pragma unroll
        for (int kk = 0; kk < R; ++kk) {
            if (kk >= n) break;
            const uint64_t w = wk[kk];
#pragma unroll
            for (int r = 0; r < R; ++r) fma2(acc[r], w, win[(r + kk) % R]);
            win[kk] = ld(R + kk);
        }
    } else if constexpr (SHORT == 2) {  // at most 2R taps: two unrolled passes
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int kk = 0; kk < R; ++kk) {
                if (h * R + kk >= n) break;
                const uint64_t w = wk[h * R + kk];
#pragma unroll
                for (int r = 0; r < R; ++r) fma2(acc[r], w, win[(r + kk) % R]);
                win[kk] = ld(R + h * R + kk);
            }
        }
    } else {
        for (int k0 = 0; k0 < n; k0 += R) {
#pragma unroll
            for (int kk = 0; kk < R; ++kk) {
                if (k0 + kk >= n) break;
                const uint64_t w = wk[k0 + kk];
#pragma unroll
                for (int r = 0; r < R; ++r) fma2(acc[r], w, win[(r + kk) % R]);
                win[kk] = ld(R + k0 + kk);
            }
        }
    }
}

// One stage of one pair unit: its entries are (trial 0's start - block minimum,
// max(n0, n1), trial 1's start - trial 0's, offset of the entry's weight pairs in the
// record's weight list).
template <typename TIN, int SHORT>
__device__ __forceinline__ void stage_pair(const TIN* rows, const int4* ent, const float2* wts,
                                           const int* lo, int csn, int lcap, int bq,
                                           int lane_off, uint64_t (&acc)[kRPair], int wpairs,
                                           int32_t* status) {
    constexpr int Q = Elem<TIN>::Q;
    for (int ci = 0; ci < csn; ++ci) {
        const int4 q = ent[ci];
        const int i0 = ((bq + lo[ci]) & (Q - 1)) + q.x + lane_off;
        if (!dbg_ok(q.x >= 0 && q.y >= 1 && i0 + min(q.z, 0) >= 0 && i0 + max(q.z, 0) + kRPair + q.y <= lcap &&
                        q.w >= 0 && q.w + q.y <= wpairs,
                    status))
            continue;
        const TIN* p = rows + ci * lcap + i0;
        const uint64_t* wk = (const uint64_t*)(wts + q.w);
        __builtin_assume(__isShared(p));
        __builtin_assume(__isShared(wk));
        if (q.z == 0)
            pair_channel<TIN, SHORT, false>(p, 0, q.y, wk, acc);
        else
            pair_channel<TIN, SHORT, true>(p, q.z, q.y, wk, acc);
    }
}

template <typename TACC, int R>
__device__ __forceinline__ void store_row(unsigned char* smem, const TACC (&acc)[R], int warp,
                                          int lane, int64_t tw, int32_t t_out, TACC* out,
                                          int64_t out_ld = INT64_MAX, int32_t* status = nullptr) {
    TACC* st = (TACC*)smem + warp * (32 * R);
#pragma unroll
    for (int r = 0; r < R; ++r) st[lane * R + r] = acc[r];
    __syncwarp();
    if (out) {
#pragma unroll 4
        for (int j = 0; j < R; ++j) {
            const int64_t t = tw + j * 32 + lane;
            if (t < t_out && dbg_ok(t >= 0 && t < out_ld, status)) out[t] = st[j * 32 + lane];
        }
    }
    __syncwarp();
}

// Per-CTA pipeline state kept in shared memory across tiles (the batched kernel runs
// many tiles per CTA): uses[b] counts completed uses of buffer b, which fixes the
// parity of the barrier phase that the next use waits for.
struct TileState {
    int uses[kStagesMax];
};

// One CTA tile: trial block `blk`, time tile `tx` of the plan described by `a`.
// Returns false (on every thread) if a bounded wait ran out.
// `a` is taken by value: with a reference to the kernel parameter the compiler picked
// a register allocation for the FMA loop that ran 11 % slower.
// FUSED: instead of storing the tile, scan it for boxcar maxima (fa: the scan's
// arguments, ft: the strip the tile belongs to); exact sums on the integer paths, the
// unfused fp32 scan's prefix chains on the pair path.
template <typename TIN, bool PAIR, int NBUF, bool MULTI, int SHORT, bool FUSED = false>
__device__ __forceinline__ bool dedisp_tile(const DedispArgs a, unsigned char* smem, int blk,
                                            int tx, TileState& ts, const FusedArgs* fa = nullptr,
                                            const fused::FusedTile* ft = nullptr) {
    constexpr int R = lane_r(PAIR);
    constexpr int TT = 32 * R;          // outputs per warp time chunk
    constexpr int Q = Elem<TIN>::Q;
    constexpr int TPW = PAIR ? 2 : 1;   // trials per warp unit
    constexpr bool RL = std::is_same<TIN, uint32_t>::value;
    // SHORT on the run-length path: the CTA shares difference rows per stage
    constexpr bool BROW = RL && SHORT != 0;
    constexpr int UPW = upw<TIN>();     // warp units per warp
    using TACC = typename std::conditional<PAIR, float, int>::type;
    const int cs = a.cs;
    const int nu = kWarps / a.nch * UPW;  // warp units per CTA
    const StageGeom g((int)sizeof(TIN), PAIR, a.lcap, a.kpad, cs, nu, BROW, a.blen);
    const Smem sm = carve<NBUF>(smem, g, a.smem_bytes, a.nchan);
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int wu = warp / a.nch, chunk = warp - wu * a.nch;
    const int dmi = wu * UPW;                                 // first unit of the warp
    const int d = blk * (TPW * nu) + dmi * TPW;               // its first trial
    const int64_t t0 = (int64_t)tx * TT * a.nch;              // CTA time start
    const int64_t tw = t0 + (int64_t)chunk * TT;               // warp time start
    const int64_t base = a.t_offset + t0;
    const int nst = (a.nchan + cs - 1) / cs;
    // the CTA's stages: a contiguous share of the channel sum when the launch splits it
    // (blockIdx.z = split, partial sums to separate outputs), else all of them
    const int split = (int)blockIdx.z;
    const int s_lo = (int)((int64_t)split * nst / a.nsplit);
    const int nloc = (int)((int64_t)(split + 1) * nst / a.nsplit) - s_lo;

    // per-channel block minima; does any staged window run past the end of its row?
    int past_end = 0;
    for (int c = tid; c < a.nchan; c += blockDim.x) {
        const int lo = a.blk_lo[(int64_t)blk * a.nchan + c];
        sm.lo_all[c] = lo;
        past_end |= (((base + lo) & ~(int64_t)(Q - 1)) + a.lcap > a.ld) ? 1 : 0;
    }
    const bool tail = __syncthreads_or(past_end) != 0;
    if (tid == 0)
        for (int i = 0; i < NBUF && i < nloc; ++i) issue_stage<TIN, NBUF>(a, g, sm, blk, s_lo + i, i, base, tail);

    TACC acc0[R];
    uint64_t accp[PAIR ? R : 1];    // packed (trial 0, trial 1) sums of a pair unit
    int accr[RL ? UPW - 1 : 1][R];  // the warp's further units (run-length path)
#pragma unroll
    for (int r = 0; r < R; ++r) acc0[r] = TACC(0);
#pragma unroll
    for (int r = 0; r < (PAIR ? R : 1); ++r) accp[r] = 0ull;
#pragma unroll
    for (int u = 0; u < (RL ? UPW - 1 : 1); ++u)
#pragma unroll
        for (int r = 0; r < R; ++r) accr[u][r] = 0;
    const int bq = (int)(base & (Q - 1));
    const int lane_off = chunk * TT + lane * R;
    bool ok = true;

    if constexpr (BROW) {
        // Run-length path with difference rows shared by the CTA.  The rows of stage i
        // (B_q[j] = P[j + n_q] - P[j], per channel and tap count, over the positions its
        // trials read) are built by all threads one stage ahead, into half i & 1 of the
        // row area, together with a copy of the stage's entries; so the prefix buffer of a
        // stage is refilled as soon as its rows are built, and one CTA barrier per stage
        // both publishes the next rows and ends the reads of the current ones.
        const int* lo_all = (const int*)(smem + NBUF * g.bytes);
        auto build = [&](int i) {  // stage s_lo + i, from its prefix buffer
            const unsigned char* buf = smem + (i % NBUF) * g.bytes;
            const uint32_t* rows = (const uint32_t*)buf;
            const int4* nlist = (const int4*)(buf + g.rec_off + g.w_off);
            const int2* esrc = (const int2*)(buf + g.rec_off);
            uint32_t* half = sm.brows + (i & 1) * g.bhalf_words;
            int2* edst = (int2*)(half + cs * 2 * a.blen);
            for (int e = tid; e < nu * cs; e += kWarps * 32) edst[e] = esrc[e];
            const int csn = min(cs, a.nchan - (s_lo + i) * cs);
            for (int ci = 0; ci < csn; ++ci) {
                const int4 nn = nlist[ci];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int n = q ? nn.y : nn.x;
                    const int len = q ? nn.w : nn.z;
                    if (n <= 0) continue;
                    if (!dbg_ok(len >= 0 && len <= a.blen && len + n <= a.lcap, a.status)) continue;
                    const uint32_t* pr = rows + ci * a.lcap;
                    uint32_t* br = half + (ci * 2 + q) * a.blen;
#pragma unroll 4
                    for (int j = tid; j < len; j += kWarps * 32) br[j] = pr[j + n] - pr[j];
                }
            }
        };
        auto parity_of = [&](int i) {
            return (uint32_t)(((MULTI ? ts.uses[i % NBUF] : 0) + i / NBUF) & 1);
        };
        bool got = nloc > 0 ? mbar_wait_bounded(&sm.full[0], parity_of(0), a.wait_ns) : true;
        if (got && nloc > 0) build(0);
        if (__syncthreads_or(!got)) {
            if (tid == 0) atomicExch(a.status, (int)DD_ERR_TIMEOUT);
            ok = false;
        } else if (tid == 0 && NBUF < nloc) {
            issue_stage<TIN, NBUF>(a, g, sm, blk, s_lo + NBUF, 0, base, tail);
        }
        for (int i = 0; ok && i < nloc; ++i) {
            if (i + 1 < nloc) {
                got = mbar_wait_bounded(&sm.full[(i + 1) % NBUF], parity_of(i + 1), a.wait_ns);
                if (got) build(i + 1);
            }
            const uint32_t* half = sm.brows + (i & 1) * g.bhalf_words;
            const int2* ent = (const int2*)(half + cs * 2 * a.blen) + dmi * cs;
            const int c0 = (s_lo + i) * cs;
            const int csn = min(cs, a.nchan - c0);
            if (d < a.ndm) stage_rl_rows(half, ent, lo_all + c0, csn, a.blen, bq, lane_off, acc0, a.status);
#pragma unroll
            for (int u = 1; u < UPW; ++u)
                if (d + u < a.ndm)
                    stage_rl_rows(half, ent + u * cs, lo_all + c0, csn, a.blen, bq, lane_off, accr[u - 1],
                                  a.status);
            if (__syncthreads_or(!got)) {
                if (tid == 0) atomicExch(a.status, (int)DD_ERR_TIMEOUT);
                ok = false;
                break;
            }
            if (tid == 0 && i + 1 + NBUF < nloc)
                issue_stage<TIN, NBUF>(a, g, sm, blk, s_lo + i + 1 + NBUF, (i + 1) % NBUF, base, tail);
        }
    }

    // every other path: warps go through the ring on their own, the last one out of a
    // buffer refills it
    for (int i = 0; !BROW && i < nloc; ++i) {
        const int s = s_lo + i;
        const int b = i % NBUF;
        // a one-tile CTA starts every buffer at phase 0; a persistent CTA continues
        const uint32_t parity = (uint32_t)(((MULTI ? ts.uses[b] : 0) + i / NBUF) & 1);
        const bool got = mbar_wait_bounded(&sm.full[b], parity, a.wait_ns);
        if (!__all_sync(0xffffffffu, got)) {
            if (lane == 0) atomicExch(a.status, (int)DD_ERR_TIMEOUT);
            ok = false;
            break;
        }
        if constexpr (RL) {
            const unsigned char* buf = smem + b * g.bytes;
            const uint32_t* rows = (const uint32_t*)buf;
            const int2* ent = (const int2*)(buf + g.rec_off) + dmi * cs;
            const int* lo_all = (const int*)(smem + NBUF * g.bytes);
            const int c0 = s * cs;
            const int csn = min(cs, a.nchan - c0);
            if (d < a.ndm) stage_rl(rows, ent, lo_all + c0, csn, a.lcap, bq, lane_off, acc0, a.status);
#pragma unroll
            for (int u = 1; u < UPW; ++u)
                if (d + u < a.ndm)
                    stage_rl(rows, ent + u * cs, lo_all + c0, csn, a.lcap, bq, lane_off, accr[u - 1], a.status);
        } else if (d < a.ndm) {
            // pointers derived from the __shared__ array itself, so that every access
            // below compiles to a shared-memory load
            const unsigned char* buf = smem + b * g.bytes;
            const TIN* rows = (const TIN*)buf;
            const int2* ent = (const int2*)(buf + g.rec_off) + dmi * cs;
            const int* lo_all = (const int*)(smem + NBUF * g.bytes);
            const int c0 = s * cs;
            const int csn = min(cs, a.nchan - c0);
            if constexpr (PAIR) {
                const int4* ent4 = (const int4*)(buf + g.rec_off) + dmi * cs;
                const float2* wts = (const float2*)(buf + g.rec_off + g.w_off);
                stage_pair<TIN, SHORT>(rows, ent4, wts, lo_all + c0, csn, a.lcap, bq, lane_off, accp,
                                       a.kpad, a.status);
            } else {
                stage_int<TIN, SHORT>(rows, ent, lo_all + c0, csn, a.lcap, bq, lane_off, acc0, a.status);
            }
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            const int old = atomicAdd(&sm.cnt[b], 1);
            if (old == kWarps - 1) {  // last warp out refills the buffer
                sm.cnt[b] = 0;
                if (i + NBUF < nloc) issue_stage<TIN, NBUF>(a, g, sm, blk, s + NBUF, b, base, tail);
            }
        }
    }

    __syncthreads();
    if (!ok && tid == 0) {  // no copy may still be in flight when the CTA leaves
        for (int b = 0; b < NBUF; ++b)
            if (sm.issued[b] > 0 &&
                !mbar_wait_bounded(&sm.full[b], (uint32_t)((sm.issued[b] - 1) & 1), a.wait_ns))
                atomicExch(a.status, (int)DD_ERR_TIMEOUT);
    }
    if (!__syncthreads_and(ok)) return false;
    if (MULTI && tid == 0)
        for (int b = 0; b < NBUF && b < nloc; ++b) ts.uses[b] += (nloc - b + NBUF - 1) / NBUF;

    if constexpr (FUSED) {
        if constexpr (PAIR) {
            float f0[R], f1[R];
#pragma unroll
            for (int r = 0; r < R; ++r) unpk(accp[r], f0[r], f1[r]);
            fused::epilogue_f32<R>(a, *fa, smem, wu, chunk, lane, d, t0, *ft, f0, f1);
        } else {
            fused::epilogue<UPW, RL ? UPW - 1 : 1>(a, *fa, smem, wu, chunk, lane, d, t0, *ft, acc0, accr);
        }
        return true;
    }
    // transpose through shared memory and store coalesced, one trial row at a time
    TACC* out = (TACC*)a.out + (int64_t)split * a.split_ld;
    float acc1[PAIR ? R : 1];
    if constexpr (PAIR) {
#pragma unroll
        for (int r = 0; r < R; ++r) unpk(accp[r], acc0[r], acc1[r]);
    }
    const int64_t oldx = a.out_ld;  // a row's extent
    store_row<TACC, R>(smem, acc0, warp, lane, tw, a.t_out, d < a.ndm ? out + (int64_t)d * a.out_ld : nullptr,
                       oldx, a.status);
    if constexpr (PAIR)
        store_row<float, R>(smem, acc1, warp, lane, tw, a.t_out,
                         d + 1 < a.ndm ? (float*)out + (int64_t)(d + 1) * a.out_ld : nullptr, oldx, a.status);
    if constexpr (RL) {
#pragma unroll
        for (int u = 1; u < UPW; ++u)
            store_row<int, R>(smem, accr[u - 1], warp, lane, tw, a.t_out,
                           d + u < a.ndm ? (int*)out + (int64_t)(d + u) * a.out_ld : nullptr, oldx, a.status);
    }
    if (MULTI) __syncthreads();  // the staging area is the next tile's stage buffers
    return true;
}

template <int NBUF>
__device__ __forceinline__ void init_pipeline(unsigned char* smem_tail_full, TileState& ts) {
    uint64_t* full = (uint64_t*)smem_tail_full;
    int* cnt = (int*)(full + NBUF);
    int* issued = cnt + NBUF;
    for (int b = 0; b < NBUF; ++b) {
        mbar_init(&full[b], 1);
        cnt[b] = 0;
        issued[b] = 0;
        ts.uses[b] = 0;
    }
    fence_mbar_init();
}

// Barriers and counters sit after the stage buffers and the per-channel minima; their
// offset depends on the plan's geometry, so the kernels place them at a fixed offset
// from the end of the dynamic shared memory instead.
__device__ __forceinline__ unsigned char* pipeline_area(unsigned char* smem, size_t smem_bytes, int nbuf) {
    return smem + smem_bytes - (size_t)(nbuf * 8 + 2 * nbuf * 4);
}

// Dynamic shared memory of a launch: the plan's stages, per-channel minima and
// barriers, and at least the output transpose area plus the barriers (which sit at the
// end and survive the transpose).
template <typename TIN, bool PAIR, int NBUF>
size_t smem_for(int lcap, int kpad, int cs, int nch, int nchan, bool brow = false, int blen = 0) {
    const StageGeom g((int)sizeof(TIN), PAIR, lcap, kpad, cs, kWarps / nch * upw<TIN>(), brow, blen);
    size_t smem = (size_t)dedisp_smem_bytes(g, NBUF, nchan);
    const size_t st = (size_t)kStoreBytes + NBUF * 8 + 2 * NBUF * 4;
    if (smem < st) smem = st;
    return (smem + 15) & ~(size_t)15;
}

}  // namespace
}  // namespace dd
