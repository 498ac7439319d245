// Boxcar scan of finished dedispersion tiles inside the dedispersion CTA: the fused
// path of dd_dedisperse_boxcar (contiguous widths w0 .. w0 + nw - 1).  Integer plans
// (exact sums) first, then fp32 plans (the unfused fp32 scan's prefix chains).
// Included by dd_tile.cuh.
//
// A CTA walks its part of the launch's (trial block, time tile) items in order, a strip
// of consecutive tiles per trial block it touches.  After a tile's channel sum, each
// warp group writes its trial's outputs, minus the trial's offset o_d, into a shared-
// memory row behind the last C = wmax - 1 outputs of the previous tile (the carry), so
// that the row holds x[T0 - C .. T0 + L).  The tile then owns the window starts
// t in [T0 - C, T0 + L - C): every window of width <= wmax from such a start lies in
// the row.  The strip's first tile has no carry and starts at the strip start; its last
// tile also takes the starts up to the strip end, with windows cut off there; windows
// that cross a strip boundary are left to the seam pass (dd_fused.cu).
//
// Lane l of a warp owns the kRInt starts i0 = l * kRInt + s of a row segment and walks
// them for G widths at a time with a rotating register window of prefix sums: one
// subtract and one max per (start, width), in uint32 arithmetic whose differences are
// exact while every window sum of x - o fits int32 (checked per output against mlim;
// DD_ERR_OVERFLOW otherwise).  A warp reduction gives the tile's maximum per width;
// only where it beats (or ties from an earlier start) the merged maximum read from
// `key` is the earliest start searched -- the earliest segment holding the maximum
// writes its prefix values to the warp's scratch and the lanes test one start each --
// and (value, start) merged with one 64-bit atomicMax.
#pragma once

#include <cfloat>
#include <climits>

#include "dd_internal.h"

namespace dd {
namespace fused {
namespace {

constexpr int G = 16;  // widths per register window

// A warp's shared scratch for the earliest-start search (4-byte words): the prefix values
// P_0 .. P_30 of one segment, then P_{w0g} .. P_{w0g+45} (every P_s and P_{s+w} that a
// width of the group forms).
constexpr int kChainFloats = 80;

// S = kRInt starts of one lane segment (x = row + i0) for widths w0g + j, j < G.
// q = sum_{k < w0g} x[k] on entry.  !FULL: starts outside [i_lo, i_hi) and windows
// ending past row index e_hi are left out.
template <bool FULL>
__device__ __forceinline__ void scan_segment(const int* x, uint32_t q, int w0g, int i0, int i_lo,
                                             int i_hi, int e_hi, int (&seg)[G]) {
    constexpr int S = kRInt;
    uint32_t win[G];
    win[0] = q;
#pragma unroll
    for (int j = 1; j < G; ++j) win[j] = win[j - 1] + (uint32_t)x[w0g + j - 1];
    uint32_t p = 0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
#pragma unroll
        for (int j = 0; j < G; ++j) {
            int v = (int)(win[(j + s) % G] - p);
            if (!FULL) v = (i0 + s >= i_lo && i0 + s < i_hi && i0 + s + w0g + j <= e_hi) ? v : INT_MIN;
            seg[j] = max(seg[j], v);
        }
        p += (uint32_t)x[s];
        win[s % G] = win[(s + G - 1) % G] + (uint32_t)x[s + w0g + G - 1];
    }
}

// Maximum over the warp of seg[j] for all j at once (each exchange level halves the
// values a lane keeps): lanes 2j and 2j + 1 return the maximum for j.
__device__ __forceinline__ int warp_max16(const int (&seg)[G], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
    int v8[8], v4[4], v2[2];
#pragma unroll
    for (int j = 0; j < 8; ++j)
        v8[j] = max(b4 ? seg[j + 8] : seg[j], __shfl_xor_sync(0xffffffffu, b4 ? seg[j] : seg[j + 8], 16));
#pragma unroll
    for (int j = 0; j < 4; ++j)
        v4[j] = max(b3 ? v8[j + 4] : v8[j], __shfl_xor_sync(0xffffffffu, b3 ? v8[j] : v8[j + 4], 8));
#pragma unroll
    for (int j = 0; j < 2; ++j)
        v2[j] = max(b2 ? v4[j + 2] : v4[j], __shfl_xor_sync(0xffffffffu, b2 ? v4[j] : v4[j + 2], 4));
    int v = max(b1 ? v2[1] : v2[0], __shfl_xor_sync(0xffffffffu, b1 ? v2[0] : v2[1], 2));
    return max(v, __shfl_xor_sync(0xffffffffu, v, 1));
}

// Upper bound of every sum the FULL scan of one width group would form:
// max_{s, j} P[s + w0g + j] - min_s P[s] <= Q + Mrel, with P the prefix of the segment,
// Q = P[w0g] - min_s P[s] and Mrel = max(0, max_m sum_{k=w0g}^{w0g+m} x[k]), m < cnt + 29.
// Q is a window sum of at most wmax values and Mrel one of at most 45, so both are exact
// in int32 when wmax >= 46 (every such sum fits, by the overflow check).
__device__ __forceinline__ long long group_bound(const int* x, uint32_t q, uint32_t pmin, int w0g, int cnt) {
    int r = 0, mrel = 0;
    for (int m = 0; m < cnt + 29; ++m) {
        r += x[w0g + m];
        mrel = max(mrel, r);
    }
    return (long long)(int)(q - pmin) + mrel;
}

// Width groups from kPruneW on skip the scan of segments whose group_bound is below
// the smallest merged maximum of the group (strictly: a tie from an earlier start could
// still win), which on noise-like series is most of them.
constexpr int kPruneW = 48;

// The scan of one row for one trial (warp-uniform arguments; see epilogue).
__device__ __forceinline__ void scan_row(const FusedArgs& f, const int* row, uint32_t* chain,
                                      unsigned long long* keyrow, int64_t T0, int C, int chunk, int nch,
                                      int lane, int i_lo, int i_hi, int e_hi) {
    constexpr int R = kRInt, TT = 32 * R;
    __builtin_assume(__isShared(row));
    const int ng = (f.nw + G - 1) / G;
    const int jl = lane >> 1;
    for (int k = chunk; k * TT < i_hi; k += nch) {
        const int i0 = k * TT + lane * R;
        const int* x = row + i0;
        const bool any = i0 + R > i_lo && i0 < i_hi;
        const bool inner = i0 >= i_lo && i0 + R <= i_hi;
        const int t_lo = (int)(T0 - C) + max(k * TT, i_lo);  // earliest start of the pass
        // lanes without a start here read nothing (their segment may lie past the row)
        uint32_t q = 0, pmin = 0;
        if (any) {
            for (int kk = 0; kk < f.w0; ++kk) q += (uint32_t)x[kk];
            if (inner) {  // min_s P[s] over the segment's starts (sums of <= 30 values)
                int r = 0, mn = 0;
                for (int s = 0; s < R - 1; ++s) {
                    r += x[s];
                    mn = min(mn, r);
                }
                pmin = (uint32_t)mn;
            }
        }
        for (int g = 0; g < ng; ++g) {
            const int w0g = f.w0 + g * G;
            const int cnt = min(G, f.nw - g * G);
            unsigned long long bk = 0;
            if (!(lane & 1) && jl < cnt) bk = __ldcg(keyrow + g * G + jl);
            const int bv = (int)((uint32_t)(bk >> 32) ^ 0x80000000u);
            const int bt = (int)(0xffffffffu - (uint32_t)bk);
            const bool full = inner && i0 + R - 1 + w0g + cnt - 1 <= e_hi;
            bool scan = any;
            if (w0g >= kPruneW) {
                // the smallest merged maximum over the group's widths
                int thr = (!(lane & 1) && jl < cnt) ? bv : INT_MAX;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) thr = min(thr, __shfl_xor_sync(0xffffffffu, thr, o));
                if (full && group_bound(x, q, pmin, w0g, cnt) < (long long)thr) scan = false;
            }
            if (__any_sync(0xffffffffu, scan)) {
                int seg[G];
#pragma unroll
                for (int j = 0; j < G; ++j) seg[j] = INT_MIN;
                if (scan && full)
                    scan_segment<true>(x, q, w0g, i0, i_lo, i_hi, e_hi, seg);
                else if (scan)
                    scan_segment<false>(x, q, w0g, i0, i_lo, i_hi, e_hi, seg);
                const int mx = warp_max16(seg, lane);
                const bool better = !(lane & 1) && jl < cnt && mx > INT_MIN &&
                                    (mx > bv || (mx == bv && t_lo < bt));
                // widths whose maximum beats (or ties from an earlier start) the merged one:
                // the earliest segment holding it writes its prefix values to the warp's
                // scratch, and the lanes test one start each for every such width that this
                // segment holds first
                unsigned need = __ballot_sync(0xffffffffu, better);
                auto holder = [&](int hl) {  // earliest lane whose segment holds width hl / 2's maximum
                    const int j = hl >> 1;
                    const int mj = __shfl_sync(0xffffffffu, mx, hl);
                    int sj = INT_MIN;
#pragma unroll
                    for (int jj = 0; jj < G; ++jj) sj = jj == j ? seg[jj] : sj;
                    return __ffs(__ballot_sync(0xffffffffu, scan && sj == mj)) - 1;
                };
                while (need) {  // warp-uniform
                    const int h = holder(__ffs(need) - 1);
                    if (lane == h) {
                        uint32_t P = 0;
                        for (int kk = 0; kk <= w0g + 45; ++kk) {
                            if (kk < R) chain[kk] = P;
                            if (kk >= w0g) chain[R + kk - w0g] = P;
                            P += (uint32_t)x[kk];
                        }
                    }
                    __syncwarp();
                    const int ih = __shfl_sync(0xffffffffu, i0, h);
                    for (unsigned rest = need; rest; rest &= rest - 1) {
                        const int hl = __ffs(rest) - 1;
                        if (holder(hl) != h) continue;  // held first by another segment: a later round
                        const int j = hl >> 1;
                        const int mj = __shfl_sync(0xffffffffu, mx, hl);
                        const int i = ih + lane;
                        const bool eq = lane < R && i >= i_lo && i < i_hi && i + w0g + j <= e_hi &&
                                        (int)(chain[R + lane + j] - chain[lane]) == mj;
                        const unsigned st = __ballot_sync(0xffffffffu, eq);
                        if (lane == 0 && st)
                            atomicMax(keyrow + g * G + j, fused_key(mj, (int)(T0 - C) + ih + __ffs(st) - 1));
                        need &= ~(1u << hl);
                    }
                    __syncwarp();  // the scratch is rewritten for the next holder
                }
            }
            if (any)
#pragma unroll
                for (int kk = 0; kk < G; ++kk) q += (uint32_t)x[w0g + kk];
        }
    }
}

// Where a strip of one trial block starts and ends, and what its CTA carries and passes
// on.  seam_in / seam_out: the strip starts / ends inside the block, so its first /
// last C outputs go to that seam ([trial in block][2C], second / first half).
struct FusedTile {
    int64_t s1;         // end of the strip (exclusive), at most t_out
    bool first, last;   // first / last tile of the strip
    int32_t* carry;     // [trials per CTA][C]
    int32_t* seam_in;
    int32_t* seam_out;
};

// The fused epilogue of one tile (every thread of the CTA calls it).  NU trials per
// warp group (acc0, then accr[0 .. NU - 2]); d = the group's first trial, T0 = the
// tile's first output.

template <int NU, int NX>
__device__ __forceinline__ void epilogue(const DedispArgs& a, const FusedArgs& f, unsigned char* smem,
                                         int wu, int chunk, int lane, int d, int64_t T0,
                                         const FusedTile& ft,
                                         const int (&acc0)[kRInt], const int (&accr)[NX][kRInt]) {
    constexpr int R = kRInt, TT = 32 * R;
    const int L = TT * a.nch;
    const int C = f.C;
    int* row = (int*)smem + wu * f.rowlen;
    const int64_t S1 = ft.s1;
    const bool first = ft.first, last = ft.last;
    // row index i holds output T0 - C + i
    const int i_lo = first ? C : 0;             // first start owned by the tile
    const int e_hi = (int)(S1 - T0) + C;        // windows end at or before this index
    const int i_hi = last ? e_hi - f.w0 + 1 : L;  // starts below this index
    // the other trials' sums wait in shared memory behind the rows, so that no
    // accumulator stays live across a scan
    int* spill = (int*)smem + fused_rows_ints(kWarps / a.nch, f.rowlen, C) +
                 (threadIdx.x >> 5) * (NU - 1) * TT + lane * R;
#pragma unroll
    for (int u = 1; u < NU; ++u)
#pragma unroll
        for (int r = 0; r < R; ++r) spill[(u - 1) * TT + r] = accr[u - 1][r];
    // the warp's scratch for the earliest-start search lies behind the spilled sums
    uint32_t* chain = (uint32_t*)smem + fused_rows_ints(kWarps / a.nch, f.rowlen, C) + kWarps * (NU - 1) * TT +
                      (threadIdx.x >> 5) * kChainFloats;
#pragma unroll
    for (int u = 0; u < NU; ++u) {
        __syncthreads();  // the rows are free (stages consumed, or the previous trial scanned)
        const int du = d + u;
        const bool live = du < a.ndm;
        const int o = live ? (int)f.off[du] : 0;
        const int ib = C + chunk * TT + lane * R;
        const int64_t tb = T0 + chunk * TT + lane * R;
        int m = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int v = (u == 0 ? acc0[r] : spill[(u - 1) * TT + r]) - o;
            row[ib + r] = v;
            if (tb + r < S1) m = max(m, abs(v));
        }
        if (live && m > f.mlim) atomicExch(a.status, (int)DD_ERR_OVERFLOW);
        const int64_t cb = (int64_t)(wu * NU + u) * C;  // this trial's carry and seam rows
        if (live && chunk == 0 && !first)
            for (int k = lane; k < C; k += 32) row[k] = ft.carry[cb + k];
        __syncthreads();  // the row and its carry are complete
        if (!live) continue;
        if (chunk == 0) {
            if (!last)
                for (int k = lane; k < C; k += 32) ft.carry[cb + k] = row[L + k];
            if (first && ft.seam_in)
                for (int k = lane; k < C; k += 32) ft.seam_in[2 * cb + C + k] = row[C + k];
            if (last && ft.seam_out)
                for (int k = lane; k < C; k += 32) ft.seam_out[2 * cb + k] = row[e_hi - C + k];
        }
        scan_row(f, row, chain, f.key + (int64_t)du * f.nw, T0, C, chunk, a.nch, lane, i_lo, i_hi, e_hi);
    }
    // the next tile's bulk copies overwrite the rows
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
}


// ----------------------------------------------------------------------------- fp32 plans
//
// The unfused fp32 scan (k_boxcar_run) gives each thread kBoxSeg consecutive starts from
// a multiple of kBoxSeg and forms the segment's prefix chain P_0 = 0,
// P_{k+1} = P_k + x[k] (x = series - o_d in fp32), left to right; the window of width w
// at start s sums to P_{s+w} - P_s.  fp32 addition is deterministic, so a chain formed
// the same way anywhere gives the same sums bit for bit.  The fused scan therefore
// walks whole segments: a tile owns the segments whose first start lies in its start
// range, reads them from its shared-memory row (C = wmax + kBoxSeg - 2 outputs carried
// from the previous tile reach back to any such segment), and keeps the window ends
// that its strip holds; windows of a segment that begins before a strip boundary and
// ends past it go to the seam pass (dd_fused.cu).

// Segment at x (kBoxSeg starts) for widths w0g + j, j < G; q = P_{w0g}.  !FULL: windows
// ending past index e_rel are left out and no sample at or past it is read.  FULL
// reads up to 15 samples past the last window of the group's widths below cnt.
template <bool FULL>
__device__ __forceinline__ void scan_segment_f32(const float* x, float q, int w0g, int e_rel,
                                                 float (&seg)[G]) {
    constexpr int S = kBoxSeg;
    auto ld = [&](int k) { return (FULL || k < e_rel) ? x[k] : 0.f; };
    float win[G];
    win[0] = q;
#pragma unroll
    for (int j = 1; j < G; ++j) win[j] = win[j - 1] + ld(w0g + j - 1);
    float p = 0.f;
    // two starts per step, their sums merged with one three-input max
#pragma unroll
    for (int s = 0; s < S; s += 2) {
        float v0[G];
#pragma unroll
        for (int j = 0; j < G; ++j) {
            v0[j] = win[(j + s) % G] - p;
            if (!FULL) v0[j] = (s + w0g + j <= e_rel) ? v0[j] : -FLT_MAX;
        }
        if (s + 1 < S) {
            p += ld(s);
            win[s % G] = win[(s + G - 1) % G] + ld(s + w0g + G - 1);
#pragma unroll
            for (int j = 0; j < G; ++j) {
                float v = win[(j + s + 1) % G] - p;
                if (!FULL) v = (s + 1 + w0g + j <= e_rel) ? v : -FLT_MAX;
                seg[j] = max3(seg[j], v0[j], v);
            }
            if (s + 2 < S) {
                p += ld(s + 1);
                win[(s + 1) % G] = win[(s + G) % G] + ld(s + w0g + G);
            }
        } else {
#pragma unroll
            for (int j = 0; j < G; ++j) seg[j] = fmaxf(seg[j], v0[j]);
        }
    }
}

// warp_max16 for fp32 maxima (fmaxf, as the unfused scan).
__device__ __forceinline__ float warp_max16_f32(const float (&seg)[G], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
    float v8[8], v4[4], v2[2];
#pragma unroll
    for (int j = 0; j < 8; ++j)
        v8[j] = fmaxf(b4 ? seg[j + 8] : seg[j], __shfl_xor_sync(0xffffffffu, b4 ? seg[j] : seg[j + 8], 16));
#pragma unroll
    for (int j = 0; j < 4; ++j)
        v4[j] = fmaxf(b3 ? v8[j + 4] : v8[j], __shfl_xor_sync(0xffffffffu, b3 ? v8[j] : v8[j + 4], 8));
#pragma unroll
    for (int j = 0; j < 2; ++j)
        v2[j] = fmaxf(b2 ? v4[j + 2] : v4[j], __shfl_xor_sync(0xffffffffu, b2 ? v4[j] : v4[j + 2], 4));
    const float v = fmaxf(b1 ? v2[1] : v2[0], __shfl_xor_sync(0xffffffffu, b1 ? v2[0] : v2[1], 2));
    return fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 1));
}

// The segments m_lo <= m < m_hi of one trial's row (row index of output t: t - base;
// windows end at or before row index e_hi), 32 per warp pass, passes shared by the
// nch warps of the trial's group.  Arguments are warp-uniform.
__device__ __forceinline__ void scan_row_f32(int w0, int nw, const float* row, float* chain,
                                             unsigned long long* keyrow, int64_t base, int chunk, int nch,
                                             int lane, int64_t m_lo, int64_t m_hi, int e_hi) {
    constexpr int S = kBoxSeg;
    __builtin_assume(__isShared(row));
    const int ng = (nw + G - 1) / G;
    const int jl = lane >> 1;
    for (int64_t mb = m_lo + (int64_t)chunk * 32; mb < m_hi; mb += (int64_t)nch * 32) {
        const int64_t m = mb + lane;
        const bool any = m < m_hi;
        const int i0 = any ? (int)(m * S - base) : 0;
        const float* x = row + i0;
        const int e_rel = e_hi - i0;
        const int t_first = (int)(mb * S);  // earliest start of the pass
        float q = 0.f;
        if (any)
            for (int k = 0; k < w0; ++k) q += k < e_rel ? x[k] : 0.f;
        for (int g = 0; g < ng; ++g) {
            const int w0g = w0 + g * G;
            const int cnt = min(G, nw - g * G);
            unsigned long long bk = 0;
            if (!(lane & 1) && jl < cnt) bk = __ldcg(keyrow + g * G + jl);
            const float bv = bk ? fused_key_value_f32(bk) : -INFINITY;
            const int bt = (int)(0xffffffffu - (uint32_t)bk);
            const bool full = any && S - 1 + w0g + cnt - 1 <= e_rel;
            float seg[G];
#pragma unroll
            for (int j = 0; j < G; ++j) seg[j] = -FLT_MAX;
            if (full)
                scan_segment_f32<true>(x, q, w0g, e_rel, seg);
            else if (any)
                scan_segment_f32<false>(x, q, w0g, e_rel, seg);
            const float mx = warp_max16_f32(seg, lane);
            const bool better = !(lane & 1) && jl < cnt && mx > -FLT_MAX &&
                                (mx > bv || (mx == bv && t_first < bt));
            // widths whose maximum beats the merged one: the earliest segment holding it
            // writes its chain to the warp's scratch, and the lanes test one start each for
            // every such width that this segment holds first
            unsigned need = __ballot_sync(0xffffffffu, better);
            auto holder = [&](int hl) {  // earliest lane whose segment holds width hl / 2's maximum
                const int j = hl >> 1;
                const float mj = __shfl_sync(0xffffffffu, mx, hl);
                float sj = -FLT_MAX;
#pragma unroll
                for (int jj = 0; jj < G; ++jj) sj = jj == j ? seg[jj] : sj;
                return __ffs(__ballot_sync(0xffffffffu, any && sj == mj)) - 1;
            };
            while (need) {  // warp-uniform
                const int h = holder(__ffs(need) - 1);
                if (lane == h) {
                    float P = 0.f;
                    for (int k = 0; k <= w0g + 45; ++k) {
                        if (k < S) chain[k] = P;
                        if (k >= w0g) chain[S + k - w0g] = P;
                        P += k < e_rel ? x[k] : 0.f;
                    }
                }
                __syncwarp();
                const int eh = __shfl_sync(0xffffffffu, e_rel, h);
                const int th = __shfl_sync(0xffffffffu, (int)(m * S), h);
                for (unsigned rest = need; rest; rest &= rest - 1) {
                    const int hl = __ffs(rest) - 1;
                    if (holder(hl) != h) continue;  // held first by another segment: a later round
                    const int j = hl >> 1;
                    const float mj = __shfl_sync(0xffffffffu, mx, hl);
                    const bool eq = lane < S && lane + w0g + j <= eh && chain[S + lane + j] - chain[lane] == mj;
                    const unsigned st = __ballot_sync(0xffffffffu, eq);
                    if (lane == 0 && st) atomicMax(keyrow + g * G + j, fused_key_f32(mj, th + __ffs(st) - 1));
                    need &= ~(1u << hl);
                }
                __syncwarp();  // the scratch is rewritten for the next holder
            }
            if (any)
#pragma unroll
                for (int kk = 0; kk < G; ++kk) q += w0g + kk < e_rel ? x[w0g + kk] : 0.f;
        }
    }
}

// Carries, seams and the scan of a warp group's two trial rows (rows[u], trial d + u).
// Not inlined: its registers are then allocated apart from the channel sums', which
// keep the whole register file (the call comes once per tile).
__device__ __noinline__ void scan_pair_rows_f32(float* rows, float* chain, int rowlen, int w0, int nw, int C,
                                                int L, unsigned long long* key, int ndm, int d, int cb0,
                                                int chunk, int nch, int lane, int64_t base, int64_t m_lo,
                                                int64_t m_hi, int e_hi, bool first, bool last,
                                                float* carry, float* seam_in, float* seam_out) {
    for (int u = 0; u < 2; ++u) {
        const int du = d + u;
        if (du >= ndm) break;
        float* row = rows + u * rowlen;
        const int64_t cb = (int64_t)(cb0 + u) * C;  // this trial's carry and seam rows
        if (chunk == 0) {
            if (!last)
                for (int k = lane; k < C; k += 32) carry[cb + k] = row[L + k];
            if (first && seam_in)
                for (int k = lane; k < C; k += 32) seam_in[2 * cb + C + k] = row[C + k];
            if (last && seam_out)
                for (int k = lane; k < C; k += 32) seam_out[2 * cb + k] = row[e_hi - C + k];
        }
        scan_row_f32(w0, nw, row, chain, key + (int64_t)du * nw, base, chunk, nch, lane, m_lo, m_hi, e_hi);
    }
}

// The fused epilogue of one fp32 pair tile (every thread of the CTA calls it): the warp
// group's two trials d, d + 1 (sums acc0, acc1), T0 = the tile's first output; one row
// per trial.  The tile owns the segments whose first start lies in [T0 - C, T0 + L - C)
// (the strip's first tile: from T0; its last: up to the strip end S1, windows ending at
// or before S1).
template <int R>
__device__ __forceinline__ void epilogue_f32(const DedispArgs& a, const FusedArgs& f, unsigned char* smem,
                                             int wu, int chunk, int lane, int d, int64_t T0,
                                             const FusedTile& ft, const float (&acc0)[R],
                                             const float (&acc1)[R]) {
    constexpr int S = kBoxSeg, TT = 32 * R;
    const int L = TT * a.nch;
    const int C = f.C;
    float* rows = (float*)smem + 2 * wu * f.rowlen;
    const int64_t S1 = ft.s1;
    const bool first = ft.first, last = ft.last;
    const int64_t base = T0 - C;  // output of row index 0
    const int e_hi = (int)((last ? S1 : T0 + L) - base);
    const int64_t t_lo = first ? T0 : base, t_hi = last ? S1 : T0 + L - C;
    const int64_t m_lo = (t_lo + S - 1) / S, m_hi = (t_hi + S - 1) / S;
    float* carry = (float*)ft.carry;
    const int ib = C + chunk * TT + lane * R;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const bool live = d + u < a.ndm;
        const float o = live ? (float)f.off[d + u] : 0.f;
        float* row = rows + u * f.rowlen;
#pragma unroll
        for (int r = 0; r < R; ++r) row[ib + r] = (u == 0 ? acc0[r] : acc1[r]) - o;
        if (live && chunk == 0 && !first)
            for (int k = lane; k < C; k += 32) row[k] = carry[(int64_t)(wu * 2 + u) * C + k];
    }
    __syncthreads();  // the rows and their carries are complete
    // the warp's chain scratch lies behind the rows
    float* chain = (float*)smem + fused_rows_ints(2 * kWarps / a.nch, f.rowlen, C) + (threadIdx.x >> 5) * kChainFloats;
    scan_pair_rows_f32(rows, chain, f.rowlen, f.w0, f.nw, C, L, f.key, a.ndm, d, wu * 2, chunk, a.nch, lane,
                       base, m_lo, m_hi, e_hi, first, last, carry, (float*)ft.seam_in, (float*)ft.seam_out);
    // the next tile's bulk copies overwrite the rows
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
}

}  // namespace
}  // namespace fused
}  // namespace dd
