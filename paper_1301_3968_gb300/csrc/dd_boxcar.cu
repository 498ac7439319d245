// Detection statistic: per-channel noise statistics, the boxcar normaliser and the
// boxcar S/N scan (eq. snr and eq. P_N_dedisp, Sec. 2.1; boxcar detector, Sec. 5).
//
//   B_w[t] = sum_{j<w} x[d][t+j],      snr = (B_w - mu_dw) / sigma_dw
//   mu_dw = w * sum_c mu_c s_dc          (s_dc = sum_k w_dck)
//   sigma_dw^2 = sum_c sigma_c^2 Q_dc(w),  Q_dc(w) = || w_dc (*) 1_w ||^2
//
// All reductions run in a fixed order, so results are deterministic.
#include <cfloat>
#include <type_traits>
#include <climits>
#include <algorithm>
#include <cstdint>

#include "dd_async.cuh"
#include "dd_debug.cuh"
#include "dd_internal.h"

namespace dd {
namespace {

// ----------------------------------------------------------------------------- stats

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One CTA per channel.  uint8: exact int64 sums of x and x^2.  fp32: sums of (x - x0)
// and (x - x0)^2 around x0 = the mean of the row's first 256 samples, which keeps the
// variance free of cancellation for rows with a large mean.  Each thread sums runs of 32
// of its samples as unevaluated pairs hi + lo of fp32 values (Knuth's TwoSum for every
// addition, squares split exactly by an FMA), which carry about twice fp32's precision,
// and adds the run sums in double: the slow FP64 pipe then sees two adds per 32 samples
// instead of three operations per sample, with the double-precision result unchanged.
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float a) {
    const float s = hi + a;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (a - bp);
    hi = s;
}

template <typename TIN>
__global__ void __launch_bounds__(256) k_chan_stats(const TIN* in, int64_t ld, int64_t t_offset,
                                                    int64_t n, double* mean, double* sd) {
    const int c = blockIdx.x;
    const TIN* row = in + (int64_t)c * ld + t_offset;
    __shared__ double sh1[8], sh2[8];
    __shared__ long long si1[8], si2[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (sizeof(TIN) == 1) {
        long long s1 = 0, s2 = 0;
        for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
            long long v = (long long)row[t];
            s1 += v;
            s2 += v * v;
        }
        s1 = warp_sum(s1);
        s2 = warp_sum(s2);
        if (lane == 0) {
            si1[warp] = s1;
            si2[warp] = s2;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long a = 0, b = 0;
            for (int i = 0; i < 8; ++i) {
                a += si1[i];
                b += si2[i];
            }
            const double m = (double)a / (double)n;
            double var = (double)b / (double)n - m * m;
            mean[c] = m;
            sd[c] = sqrt(var > 0 ? var : 0.0);
        }
    } else {
        __shared__ float sx0;
        if (warp == 0) {  // x0: the mean of the first min(n, 256) samples
            const int n0 = (int)(n < 256 ? n : 256);
            float a = 0.f;
            for (int t = lane; t < n0; t += 32) a += (float)row[t];
            a = warp_sum(a);
            if (lane == 0) sx0 = a / (float)n0;
        }
        __syncthreads();
        const float x0 = sx0;
        double s1 = 0, s2 = 0;
        for (int64_t t0 = threadIdx.x; t0 < n; t0 += (int64_t)blockDim.x * 32) {
            float h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
#pragma unroll 8
            for (int k = 0; k < 32; ++k) {
                const int64_t t = t0 + (int64_t)k * blockDim.x;
                const float x = t < n ? (float)row[t] : x0;
                // x - x0 = vh + vl exactly (TwoSum)
                const float vh = x - x0;
                const float bp = vh - x;
                const float vl = (x - (vh - bp)) + (-x0 - bp);
                two_sum_add(h1, l1, vh);
                l1 += vl;
                // (vh + vl)^2 = p + (the FMA's exact remainder of vh^2) + 2 vh vl + vl^2
                const float p = vh * vh;
                l2 += fmaf(vh, vh, -p) + 2.f * vh * vl;
                two_sum_add(h2, l2, p);
            }
            s1 += (double)h1 + (double)l1;
            s2 += (double)h2 + (double)l2;
        }
        s1 = warp_sum(s1);
        s2 = warp_sum(s2);
        if (lane == 0) {
            sh1[warp] = s1;
            sh2[warp] = s2;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0, b = 0;
            for (int i = 0; i < 8; ++i) {
                a += sh1[i];
                b += sh2[i];
            }
            const double m = a / (double)n;
            double var = b / (double)n - m * m;
            mean[c] = (double)x0 + m;
            sd[c] = sqrt(var > 0 ? var : 0.0);
        }
    }
}

// ----------------------------------------------------------------------------- normaliser

// || 1_n (*) 1_w ||^2: a trapezoid with plateau min(n,w) of length |n-w|+1.
__device__ __forceinline__ float q_unit(int n, int w) {
    const float m = (float)min(n, w);
    return (m - 1.f) * m * (2.f * m - 1.f) / 3.f + m * m * (float)(abs(n - w) + 1);
}

// Weights are staged in shared memory when a channel's taps fit kNormStageK words: 256
// channels at a time, copied with coalesced loads, rows at an odd stride (conflict-free
// for the per-channel loops below).
constexpr int kNormStageK = 47;
__host__ __device__ inline int norm_stage_stride(int kpad) { return kpad | 1; }

// One CTA per trial, one thread per channel (256 at a time).  The per-trial offset o_d
// (rounded for integer series) = expected mean of x_d = sum_c mean_c sum_k w_dck, and per
// width the warp sums of sigma_c^2 Q_dc(w), Q_dc(w) = ||w_dc (*) 1_w||^2, accumulated per
// warp and then across warps.  wstage: the weights are staged (the stride of a row), or 0.
__global__ void __launch_bounds__(256) k_norm(const int32_t* taps, const float* w, int32_t kpad,
                                              int32_t nchan, const double* mean, const double* sd,
                                              const int32_t* widths, int32_t nw, int int_off,
                                              int32_t wstage, double* off, float* mu_out, float* isd_out) {
    extern __shared__ float red[];  // [8][nw], then the staged weights [256][wstage]
    float* sw = red + 8 * nw;
    __shared__ double shm[8];
    const int d = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t* tp = taps + (int64_t)d * nchan;
    const float* wd = w ? w + (int64_t)d * nchan * kpad : nullptr;
    for (int i = threadIdx.x; i < 8 * nw; i += blockDim.x) red[i] = 0.f;

    double m1 = 0.0;
    for (int c0 = 0; c0 < nchan; c0 += 256) {
        const int cn = min(256, nchan - c0);
        if (wd && wstage) {
            __syncthreads();  // the previous channels' weights are consumed
            const float* src = wd + (int64_t)c0 * kpad;
            for (int i = threadIdx.x; i < cn * kpad; i += blockDim.x) {
                const int r = i / kpad;
                sw[r * wstage + (i - r * kpad)] = src[i];
            }
        }
        __syncthreads();  // the staged weights (and, first time, the zeroed sums) are visible
        const int c = c0 + (int)threadIdx.x;
        const bool ok = c < nchan;
        const int n = ok ? tp[c] : 1;
        const float s2 = ok ? (float)(sd[c] * sd[c]) : 0.f;
        // weighted taps: A = (sum w)^2 and Bp = 2 sum_{D>=1} D R(D) give
        // Q(w) = w A - Bp for w >= n; shorter widths use the direct sum.
        float A = 0.f, Bp = 0.f;
        const float* wk = (wd && ok) ? (wstage ? sw + threadIdx.x * wstage : wd + (int64_t)c * kpad) : nullptr;
        float ssum = (float)n;
        if (wk) {
            ssum = 0.f;
            for (int k = 0; k < n; ++k) ssum += wk[k];
            A = ssum * ssum;
            for (int D = 1; D < n; ++D) {
                float r = 0.f;
                for (int k = 0; k + D < n; ++k) r += wk[k] * wk[k + D];
                Bp += 2.f * (float)D * r;
            }
        }
        if (ok) m1 += mean[c] * (double)ssum;
        for (int j = 0; j < nw; ++j) {
            const int wdt = widths[j];
            float q;
            if (!wk) {
                q = q_unit(n, wdt);
            } else if (wdt >= n) {
                q = (float)wdt * A - Bp;
            } else {
                float v = 0.f;
                q = 0.f;
                for (int m = 0; m < n + wdt - 1; ++m) {
                    if (m < n) v += wk[m];
                    if (m >= wdt) v -= wk[m - wdt];
                    q += v * v;
                }
            }
            float contrib = warp_sum(s2 * q);
            if (lane == 0) red[warp * nw + j] += contrib;
        }
    }
    m1 = warp_sum(m1);
    if (lane == 0) shm[warp] = m1;
    __syncthreads();
    double mu1 = 0.0;
    for (int i = 0; i < 8; ++i) mu1 += shm[i];
    const double o = int_off ? rint(mu1) : mu1;
    for (int j = threadIdx.x; j < nw; j += blockDim.x) {
        float v = 0.f;
        for (int i = 0; i < 8; ++i) v += red[i * nw + j];
        mu_out[(int64_t)d * nw + j] = (float)((double)widths[j] * (mu1 - o));
        isd_out[(int64_t)d * nw + j] = v > 0.f ? 1.0f / sqrtf(v) : 0.f;
    }
    if (threadIdx.x == 0) off[d] = o;
}

// ----------------------------------------------------------------------------- boxcar scan

struct BoxArgs {
    const void* x;
    int64_t ld;
    int32_t t_len;
    int32_t ndm;
    const int32_t* widths;
    int32_t nw;
    const double* off;
    const float* mu;
    const float* isd;
    float* peak;
    int32_t* arg;
    float thresh;
    dd_candidate* cands;
    int32_t cap;
    int32_t* ncands;
    // rows taken by this launch: all (narrow == nullptr), or those whose flag narrow[d]
    // equals narrow_sel (the int32 launch takes the flagged rows, the int64 one the rest)
    const uint8_t* narrow;
    int32_t narrow_sel;
    int32_t* status;  // the plan's device status word (debug-build bounds checks)
    int32_t gpc;      // k_boxcar_run: width groups per CTA (1, 2, 4 or 8)
};

template <typename T>
__device__ __forceinline__ T lowest();
template <>
__device__ __forceinline__ float lowest<float>() { return -FLT_MAX; }
template <>
__device__ __forceinline__ int lowest<int>() { return INT_MIN; }
template <>
__device__ __forceinline__ long long lowest<long long>() { return LLONG_MIN; }

constexpr int kBoxS = kBoxSeg;  // samples per thread segment
constexpr int kBoxG = 16;  // widths per CTA

// grid (width groups, trials).  The CTA walks the row in chunks of 256*S samples;
// thread segments keep G running boxcar sums and their maxima in registers.
template <typename TX, typename TB>
__global__ void __launch_bounds__(256) k_boxcar(BoxArgs a) {
    constexpr int S = kBoxS, G = kBoxG;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TX* xs = (TX*)smem_raw;
    __shared__ TB rb[8][G];
    __shared__ int ri[8][G];
    const int d = blockIdx.y;
    const int j0 = blockIdx.x * G;
    const int cnt = min(G, a.nw - j0);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int wl[G];
#pragma unroll
    for (int j = 0; j < G; ++j) wl[j] = j < cnt ? a.widths[j0 + j] : INT_MAX / 2;
    const int wmin = wl[0], wmax = a.widths[j0 + cnt - 1];
    const TX o = (TX)a.off[d];
    const TX* xrow = (const TX*)a.x + (int64_t)d * a.ld;
    TB best[G];
    int bi[G];
#pragma unroll
    for (int j = 0; j < G; ++j) {
        best[j] = lowest<TB>();
        bi[j] = -1;
    }
    const int tvalid = a.t_len - wmin + 1;
    const int chunk = 256 * S;
    for (int tc = 0; tc < tvalid; tc += chunk) {
        __syncthreads();
        for (int i = tid; i < chunk + wmax + 1; i += 256) {
            const int t = tc + i;
            xs[i] = t < a.t_len ? (TX)(xrow[t] - o) : TX(0);
        }
        __syncthreads();
        const int ls = tid * S;
        TB B[G];
        TB run = TB(0);
        int idx = 0;
#pragma unroll
        for (int j = 0; j < G; ++j) {
            if (j < cnt) {
                while (idx < wl[j]) {
                    run += (TB)xs[ls + idx];
                    ++idx;
                }
            }
            B[j] = run;
        }
        for (int s = 0; s < S; ++s) {
            const int t = tc + ls + s;
            const TB x0 = (TB)xs[ls + s];
#pragma unroll
            for (int j = 0; j < G; ++j) {
                if (j < cnt) {
                    if (t + wl[j] <= a.t_len && B[j] > best[j]) {
                        best[j] = B[j];
                        bi[j] = t;
                    }
                    B[j] += (TB)xs[ls + s + wl[j]] - x0;
                }
            }
        }
    }
    // reduce (max, earliest t) over the CTA
#pragma unroll
    for (int j = 0; j < G; ++j) {
        TB b = best[j];
        int i = bi[j];
#pragma unroll
        for (int ofs = 16; ofs > 0; ofs >>= 1) {
            const TB ob = __shfl_xor_sync(0xffffffffu, b, ofs);
            const int oi = __shfl_xor_sync(0xffffffffu, i, ofs);
            if (oi >= 0 && (i < 0 || ob > b || (ob == b && oi < i))) {
                b = ob;
                i = oi;
            }
        }
        if (lane == 0) {
            rb[warp][j] = b;
            ri[warp][j] = i;
        }
    }
    __syncthreads();
    if (tid < cnt) {
        const int j = tid;
        TB b = rb[0][j];
        int i = ri[0][j];
        for (int k = 1; k < 8; ++k) {
            const TB ob = rb[k][j];
            const int oi = ri[k][j];
            if (oi >= 0 && (i < 0 || ob > b || (ob == b && oi < i))) {
                b = ob;
                i = oi;
            }
        }
        const int64_t o2 = (int64_t)d * a.nw + j0 + j;
        if (!dbg_ok(d < a.ndm && j0 + j < a.nw, a.status)) return;
        const float snr = (float)(((double)b - (double)a.mu[o2]) * (double)a.isd[o2]);
        a.peak[o2] = snr;
        a.arg[o2] = i;
        if (a.cands && snr > a.thresh) {
            const int k = atomicAdd(a.ncands, 1);
            if (k < a.cap) {
                dd_candidate cd;
                cd.dm_index = d;
                cd.width_index = j0 + j;
                cd.t = i;
                cd.snr = snr;
                a.cands[k] = cd;
            }
        }
    }
}

// Contiguous width lists (w_j = w_0 + j): the sums come from a per-thread prefix
// sequence instead of G running sums.  Each thread owns S consecutive start times of
// a chunk and walks P[i] = sum_{k<i} x[ls + k] (P[0] = 0, one add per step, in index
// order), keeping P[s + w_0 + j] for the G widths in a rotating register window, so
// B_j(t) = P[s + w_j] - P[s] costs one subtract and one max per (t, width).  Integer
// series accumulate in unsigned arithmetic: the difference is exact modulo 2^bits and
// the true sum fits the signed type (the plan's bound), so wrap-around in P is harmless.
// The hot loop keeps only maxima.  A thread records, per width, the chunk in which its
// segment maximum last rose strictly; the CTA picks the largest value and the earliest
// (chunk, thread), i.e. the earliest segment holding the maximum, and one thread per
// width then recomputes that segment's sums from global memory with the same
// recurrence (bit-identical values) to find the earliest time.
template <typename TB>
struct Acc;
template <>
struct Acc<float> {
    using U = float;
};
template <>
struct Acc<int> {
    using U = unsigned int;
};
template <>
struct Acc<long long> {
    using U = unsigned long long;
};

template <typename TX, typename TB>
__device__ __forceinline__ typename Acc<TB>::U to_acc(TX v) {
    using U = typename Acc<TB>::U;
    return (U)(TB)v;
}

// xl: the thread's staged samples (raw series values); o: the trial's offset, taken
// off each sample as it is read.
template <typename TX, typename TB, bool FULL>
__device__ __forceinline__ void run_segment(const TX* xl, TX o, int w0, int t0, int t_len,
                                            TB (&seg)[kBoxG]) {
    constexpr int S = kBoxS, G = kBoxG;
    using U = typename Acc<TB>::U;
    U p = U(0);
    U q = U(0);
    for (int k = 0; k < w0; ++k) q += to_acc<TX, TB>((TX)(xl[k] - o));
    U win[G];
    win[0] = q;
#pragma unroll
    for (int j = 1; j < G; ++j) win[j] = win[j - 1] + to_acc<TX, TB>((TX)(xl[w0 + j - 1] - o));
    // two starts per step, their sums merged with one three-input max
#pragma unroll
    for (int s = 0; s < S; s += 2) {
        TB v0[G];
#pragma unroll
        for (int j = 0; j < G; ++j) {
            v0[j] = (TB)(win[(j + s) % G] - p);
            if (!FULL) v0[j] = (t0 + s + w0 + j <= t_len) ? v0[j] : lowest<TB>();
        }
        p += to_acc<TX, TB>((TX)(xl[s] - o));
        win[s % G] = win[(s + G - 1) % G] + to_acc<TX, TB>((TX)(xl[s + w0 + G - 1] - o));
        if (s + 1 < S) {
#pragma unroll
            for (int j = 0; j < G; ++j) {
                TB v = (TB)(win[(j + s + 1) % G] - p);
                if (!FULL) v = (t0 + s + 1 + w0 + j <= t_len) ? v : lowest<TB>();
                seg[j] = max3(seg[j], v0[j], v);
            }
            p += to_acc<TX, TB>((TX)(xl[s + 1] - o));
            win[(s + 1) % G] = win[(s + G) % G] + to_acc<TX, TB>((TX)(xl[s + w0 + G] - o));
        } else {
#pragma unroll
            for (int j = 0; j < G; ++j) seg[j] = max(seg[j], v0[j]);
        }
    }
}

// grid (CTAs of gpc width groups, trials).  The CTA's warps split into gpc groups of
// 8 / gpc warps; all of them scan the same staged chunk of 32 * (8 / gpc) * S samples,
// each group for its own 16 widths, so a row is read once per gpc groups.  Thread
// segments still start at multiples of S (chunks are whole segments).  fp32: three CTAs
// per SM (80 registers, 72 bytes spilled), 8 % faster than two with no spills on the
// CRAFT-like series (1.283 -> 1.185 ms with the normaliser).
template <typename TX, typename TB>
__global__ void __launch_bounds__(256, std::is_same<TB, float>::value ? 3 : 2) k_boxcar_run(BoxArgs a) {
    constexpr int S = kBoxS, G = kBoxG;
    using U = typename Acc<TB>::U;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ TB rb[8][G];
    __shared__ int rc[8][G];
    __shared__ int rt[8][G];
    const int d = blockIdx.y;
    if (a.narrow && (int)a.narrow[d] != a.narrow_sel) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gpc = a.gpc, wpg = 8 / gpc, tpg = 32 * wpg;  // groups per CTA, warps and threads per group
    const int ng = (a.nw + G - 1) / G;
    const int gi = warp / wpg, gt = tid - gi * tpg;      // this thread's group in the CTA, index in it
    const int g = blockIdx.x * gpc + gi;                  // its width group (>= ng: idle)
    const int g_first = blockIdx.x * gpc, g_last = min(ng, g_first + gpc) - 1;
    const bool active = g < ng;
    const int j0 = (active ? g : g_last) * G;
    const int cnt = min(G, a.nw - j0);
    const int w0 = a.widths[j0];
    const int w0_first = a.widths[g_first * G], w0_cta = a.widths[g_last * G];
    const int w0_last = a.widths[(ng - 1) * G];
    const int chunk = tpg * S;
    // two chunk buffers (sized for the launch's last width group): the next chunk's
    // copies are in flight while the current one is scanned
    const int bufl = (chunk + w0_last + G + 4 + 3) & ~3;
    TX* const xs0 = (TX*)smem_raw;
    TX* const xs1 = xs0 + bufl;
    const int wlast = w0 + cnt - 1;
    const TX o = (TX)a.off[d];
    const TX* xrow = (const TX*)a.x + (int64_t)d * a.ld;
    TB best[G];
    int bch[G];
#pragma unroll
    for (int j = 0; j < G; ++j) {
        best[j] = lowest<TB>();
        bch[j] = -1;
    }
    const int tvalid = a.t_len - w0 + 1;
    const int tvalid_cta = a.t_len - w0_first + 1;  // the CTA's longest scan
    const int stage = chunk + w0_cta + G;
    const int ls = gt * S;
    // 16-byte copies from the row's 16-byte boundaries: buffer element k holds series
    // element tc - mis + k (chunks start at multiples of 4 elements)
    const int mis = (int)(((uintptr_t)xrow >> 2) & 3);
    // the staged chunk fits its buffer and every width of the group fits the series
    if (!dbg_ok(stage + mis <= bufl && w0 >= 1 && wlast <= a.t_len && (chunk & 3) == 0, a.status)) return;
    // pieces past the end of the row are not copied (their buffer words keep older
    // values) and a piece that crosses it is zero-filled: only windows that run past the
    // series end read them, and those are excluded
    auto load = [&](int tc, TX* dst) {
        const int n16 = (stage + mis + 3) >> 2;
        for (int i = tid; i < n16; i += 256) {
            const int t = tc - mis + 4 * i;  // first element of the piece
            if (t < 0) {  // the row's first piece: nothing before the row is read
                for (int k = -t; k < 4; ++k) {
                    const bool ok = t + k < a.t_len;
                    cp_async4(dst + 4 * i + k, ok ? xrow + t + k : xrow, ok);
                }
            } else if (t < a.t_len) {
                cp_async16(dst + 4 * i, xrow + t, 4 * min(4, a.t_len - t));
            }
        }
        cp_async_commit();
    };
    load(0, xs0);
    for (int ci = 0, tc = 0; tc < tvalid_cta; ++ci, tc += chunk) {
        TX* const xs = (ci & 1) ? xs1 : xs0;
        if (tc + chunk < tvalid_cta) {
            load(tc + chunk, (ci & 1) ? xs0 : xs1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        TB seg[G];
#pragma unroll
        for (int j = 0; j < G; ++j) seg[j] = lowest<TB>();
        if (active && tc + chunk - 1 + wlast <= a.t_len)
            run_segment<TX, TB, true>(xs + mis + ls, o, w0, tc + ls, a.t_len, seg);
        else if (active && tc + ls < tvalid)
            run_segment<TX, TB, false>(xs + mis + ls, o, w0, tc + ls, a.t_len, seg);
#pragma unroll
        for (int j = 0; j < G; ++j) {
            if (seg[j] > best[j]) {
                best[j] = seg[j];
                bch[j] = ci;
            }
        }
        __syncthreads();  // this buffer is reloaded by the next iteration but one
    }
    // (max, earliest chunk, earliest thread) over each group's warps
#pragma unroll
    for (int j = 0; j < G; ++j) {
        TB b = best[j];
        int c = bch[j];
        int t = gt;
#pragma unroll
        for (int ofs = 16; ofs > 0; ofs >>= 1) {
            const TB ob = __shfl_xor_sync(0xffffffffu, b, ofs);
            const int oc = __shfl_xor_sync(0xffffffffu, c, ofs);
            const int ot = __shfl_xor_sync(0xffffffffu, t, ofs);
            if (oc >= 0 && (c < 0 || ob > b || (ob == b && (oc < c || (oc == c && ot < t))))) {
                b = ob;
                c = oc;
                t = ot;
            }
        }
        if (lane == 0) {
            rb[warp][j] = b;
            rc[warp][j] = c;
            rt[warp][j] = t;
        }
    }
    __syncthreads();
    if (active && gt < cnt) {
        const int j = gt;
        const int k0 = gi * wpg;
        TB b = rb[k0][j];
        int c = rc[k0][j], th = rt[k0][j];
        for (int k = k0 + 1; k < k0 + wpg; ++k) {
            const TB ob = rb[k][j];
            const int oc = rc[k][j], ot = rt[k][j];
            if (oc >= 0 && (c < 0 || ob > b || (ob == b && (oc < c || (oc == c && ot < th))))) {
                b = ob;
                c = oc;
                th = ot;
            }
        }
        int arg = -1;
        if (c >= 0) {
            // the winning segment again, with the hot loop's recurrence
            const int w = w0 + j;
            const int t0 = c * chunk + th * S;
            auto xv = [&](int t) -> U { return to_acc<TX, TB>(t < a.t_len ? (TX)(xrow[t] - o) : TX(0)); };
            U p = U(0), r = U(0);
            for (int k = 0; k < w0; ++k) r += xv(t0 + k);
            for (int k = w0; k < w; ++k) r += xv(t0 + k);
            for (int s = 0; s < S; ++s) {
                const int t = t0 + s;
                if (t + w > a.t_len) break;
                if ((TB)(r - p) == b) {
                    arg = t;
                    break;
                }
                p += xv(t);
                r += xv(t + w);
            }
        }
        const int64_t o2 = (int64_t)d * a.nw + j0 + j;
        if (!dbg_ok(d < a.ndm && j0 + j < a.nw, a.status)) return;
        const float snr = (float)(((double)b - (double)a.mu[o2]) * (double)a.isd[o2]);
        a.peak[o2] = snr;
        a.arg[o2] = arg;
        if (a.cands && snr > a.thresh) {
            const int k = atomicAdd(a.ncands, 1);
            if (k < a.cap) {
                dd_candidate cd;
                cd.dm_index = d;
                cd.width_index = j0 + j;
                cd.t = arg;
                cd.snr = snr;
                a.cands[k] = cd;
            }
        }
    }
}

// Width groups per CTA: up to eight (a row is read once per eight groups; measured on the
// large block's 16 groups: 0.208 s with four per CTA, 0.200 s with eight).
template <typename TX, typename TB>
dd_status run_boxcar_contig(const BoxArgs& a0, int w0_last, cudaStream_t s) {
    BoxArgs a = a0;
    const int ng = (a.nw + kBoxG - 1) / kBoxG;
    a.gpc = ng >= 8 ? 8 : (ng >= 4 ? 4 : (ng >= 2 ? 2 : 1));
    const int chunk = 32 * (8 / a.gpc) * kBoxS;
    const size_t smem = (size_t)2 * ((chunk + w0_last + kBoxG + 4 + 3) & ~3) * sizeof(TX);
    auto kern = k_boxcar_run<TX, TB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e);
    dim3 grid((unsigned)((ng + a.gpc - 1) / a.gpc), (unsigned)a.ndm);
    if (grid.y > 65535) return DD_ERR_UNSUPPORTED;
    kern<<<grid, 256, smem, s>>>(a);
    return cuda_status(cudaGetLastError());
}

template <typename TX, typename TB>
dd_status run_boxcar(const BoxArgs& a, int wmax_all, cudaStream_t s) {
    const size_t smem = (size_t)(256 * kBoxS + wmax_all + 2) * sizeof(TX);
    auto kern = k_boxcar<TX, TB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e);
    dim3 grid((unsigned)((a.nw + kBoxG - 1) / kBoxG), (unsigned)a.ndm);
    if (grid.y > 65535) return DD_ERR_UNSUPPORTED;
    kern<<<grid, 256, smem, s>>>(a);
    return cuda_status(cudaGetLastError());
}

}  // namespace

// Series type and sum type, and the contiguous-width kernel when w_j = w_0 + j.
// Per-row bound for integer series: narrow[d] = 1 when wmax * max_t |x[d][t] - o_d| < 2^31,
// i.e. when every boxcar sum of the row fits int32 (one read of the series).
__global__ void __launch_bounds__(256) k_row_narrow(const int* x, int64_t ld, int32_t t_len,
                                                    const double* off, int32_t wmax, uint8_t* narrow) {
    const int d = blockIdx.x;
    const int* row = x + (int64_t)d * ld;
    const long long o = (long long)off[d];
    long long m = 0;
    for (int t = threadIdx.x; t < t_len; t += blockDim.x) {
        const long long v = (long long)row[t] - o;
        m = max(m, v < 0 ? -v : v);
    }
#pragma unroll
    for (int ofs = 16; ofs > 0; ofs >>= 1) m = max(m, (long long)__shfl_xor_sync(0xffffffffu, m, ofs));
    __shared__ long long wm[8];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < 8; ++i) m = max(m, wm[i]);
        narrow[d] = (uint8_t)(m * (long long)wmax < (long long)INT_MAX ? 1 : 0);
    }
}

static dd_status dispatch_boxcar(const dd_plan_s* p, const BoxArgs& a, const int32_t* widths,
                                 int32_t nw, cudaStream_t s, bool split_rows) {
    const int wmax = widths[nw - 1];
    bool contig = true;
    for (int j = 1; j < nw; ++j) contig = contig && widths[j] == widths[0] + j;
    const int w0_last = widths[((nw - 1) / kBoxG) * kBoxG];
    if (!p->out_int)
        return contig ? run_boxcar_contig<float, float>(a, w0_last, s) : run_boxcar<float, float>(a, wmax, s);
    // exact integer sums around the per-trial offset: |x - o| <= 255 * N_S(d), so a
    // width-w sum fits int32 when wmax * 255 * max_d N_S(d) < 2^31
    const long long bound = (long long)wmax * p->max_abs_row;
    if (bound < (long long)INT_MAX)
        return contig ? run_boxcar_contig<int, int>(a, w0_last, s) : run_boxcar<int, int>(a, wmax, s);
    if (!contig || !split_rows || !p->dev.narrow)
        return contig ? run_boxcar_contig<int, long long>(a, w0_last, s) : run_boxcar<int, long long>(a, wmax, s);
    // the plan-wide bound needs int64, but rows of noise-like series rarely do: measure
    // each row, sum the narrow ones in int32 and only the rest in int64
    k_row_narrow<<<a.ndm, 256, 0, s>>>((const int*)a.x, a.ld, a.t_len, a.off, wmax, p->dev.narrow);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    BoxArgs a32 = a, a64 = a;
    a32.narrow = a64.narrow = p->dev.narrow;
    a32.narrow_sel = 1;
    a64.narrow_sel = 0;
    dd_status st = run_boxcar_contig<int, int>(a32, w0_last, s);
    if (st != DD_OK) return st;
    return run_boxcar_contig<int, long long>(a64, w0_last, s);
}

dd_status launch_channel_stats(dd_plan_s* p, const void* in, int64_t ld, int64_t t_offset,
                               int64_t nsamp, double* mean, double* sd, cudaStream_t s) {
    if (p->band.in_type == DD_U8)
        k_chan_stats<uint8_t><<<p->nchan, 256, 0, s>>>((const uint8_t*)in, ld, t_offset, nsamp, mean, sd);
    else
        k_chan_stats<float><<<p->nchan, 256, 0, s>>>((const float*)in, ld, t_offset, nsamp, mean, sd);
    return cuda_status(cudaGetLastError());
}

static dd_status ensure_norm_ws(dd_plan_s* p, int nw) {
    if (p->dev.ws_w >= nw && p->dev.mu) return DD_OK;
    cudaFree(p->dev.mu);
    cudaFree(p->dev.isd);
    cudaFree(p->dev.widths);
    cudaFree(p->dev.narrow);
    p->widths_on_dev.clear();
    p->dev.mu = nullptr;
    p->dev.isd = nullptr;
    p->dev.widths = nullptr;
    p->dev.narrow = nullptr;
    p->dev.ws_w = 0;
    cudaError_t e = cudaMalloc((void**)&p->dev.mu, (size_t)p->ndm * nw * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->dev.isd, (size_t)p->ndm * nw * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->dev.widths, (size_t)nw * sizeof(int32_t));
    if (e == cudaSuccess && p->out_int) e = cudaMalloc((void**)&p->dev.narrow, (size_t)p->ndm);
    if (e != cudaSuccess) return cuda_status(e);
    p->dev.ws_w = nw;
    return DD_OK;
}

// The normaliser's staged weight stride (0: weights read from global memory) and its
// dynamic shared memory.
static int norm_wstage(const dd_plan_s* p) {
    return (!p->unit && p->kpad > 0 && p->kpad <= kNormStageK) ? norm_stage_stride(p->kpad) : 0;
}
static size_t norm_smem(int wstage, int nw) { return ((size_t)8 * nw + (size_t)256 * wstage) * sizeof(float); }

dd_status launch_boxcar_scratch(dd_plan_s* p, const void* x, int64_t ld, int64_t t_len,
                                const int32_t* widths, int32_t nw, const int32_t* widths_dev,
                                const double* mean, const double* sd, double* off, float* mu,
                                float* isd, float* peak, int32_t* arg, float thresh,
                                dd_candidate* cands, int32_t cap, int32_t* ncands, cudaStream_t s) {
    const int wstage = norm_wstage(p);
    const size_t red = norm_smem(wstage, nw);
    cudaError_t e = cudaSuccess;
    if (red > 48 * 1024) {
        e = cudaFuncSetAttribute(k_norm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)red);
        if (e != cudaSuccess) return cuda_status(e);
    }
    k_norm<<<p->ndm, 256, red, s>>>(p->dev.taps, p->unit ? nullptr : p->dev.w, p->kpad, p->nchan,
                                    mean, sd, widths_dev, nw, p->out_int ? 1 : 0, wstage, off, mu, isd);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    BoxArgs a;
    a.x = x;
    a.ld = ld;
    a.t_len = (int32_t)t_len;
    a.ndm = p->ndm;
    a.widths = widths_dev;
    a.nw = nw;
    a.off = off;
    a.mu = mu;
    a.isd = isd;
    a.peak = peak;
    a.arg = arg;
    a.thresh = thresh;
    a.cands = cands;
    a.cap = cap;
    a.ncands = ncands;
    a.narrow = nullptr;
    a.narrow_sel = 0;
    a.status = p->dev.status;
    return dispatch_boxcar(p, a, widths, nw, s, false);
}

// Loads every kernel that launch_boxcar_scratch can launch onto the current device.
// Under lazy module loading a kernel's code is placed in device memory at its first
// launch; the allocation-free boxcar entry point must not be the call that does that.
dd_status preload_boxcar_kernels() {
    cudaFuncAttributes fa;
    const void* kerns[] = {
        (const void*)k_norm,
        (const void*)k_boxcar_run<float, float>, (const void*)k_boxcar<float, float>,
        (const void*)k_boxcar_run<int, int>, (const void*)k_boxcar<int, int>,
        (const void*)k_boxcar_run<int, long long>, (const void*)k_boxcar<int, long long>,
    };
    for (const void* k : kerns) {
        const cudaError_t e = cudaFuncGetAttributes(&fa, k);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return DD_OK;
}

// The normaliser of the plan's trials for a width list: dev.off, dev.mu, dev.isd.
dd_status launch_norm(dd_plan_s* p, const int32_t* widths, int32_t nw, const double* mean,
                      const double* sd, cudaStream_t s) {
    dd_status st = ensure_norm_ws(p, nw);
    if (st != DD_OK) return st;
    cudaError_t e = cudaSuccess;
    if (p->widths_on_dev.size() != (size_t)nw ||
        !std::equal(widths, widths + nw, p->widths_on_dev.begin())) {
        // a new width list: copy it synchronously (the host array may be a temporary)
        e = cudaMemcpyAsync(p->dev.widths, widths, (size_t)nw * sizeof(int32_t),
                            cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_status(e);
        p->widths_on_dev.assign(widths, widths + nw);
    }
    const int wstage = norm_wstage(p);
    const size_t red = norm_smem(wstage, nw);
    if (red > 48 * 1024) {
        e = cudaFuncSetAttribute(k_norm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)red);
        if (e != cudaSuccess) return cuda_status(e);
    }
    k_norm<<<p->ndm, 256, red, s>>>(p->dev.taps, p->unit ? nullptr : p->dev.w, p->kpad, p->nchan,
                                    mean, sd, p->dev.widths, nw, p->out_int ? 1 : 0, wstage, p->dev.off,
                                    p->dev.mu, p->dev.isd);
    return cuda_status(cudaGetLastError());
}

dd_status launch_boxcar(dd_plan_s* p, const void* x, int64_t ld, int64_t t_len,
                        const int32_t* widths, int32_t nw, const double* mean, const double* sd,
                        float* peak, int32_t* arg, float thresh, dd_candidate* cands, int32_t cap,
                        int32_t* ncands, cudaStream_t s) {
    const dd_status st = launch_norm(p, widths, nw, mean, sd, s);
    if (st != DD_OK) return st;
    BoxArgs a;
    a.x = x;
    a.ld = ld;
    a.t_len = (int32_t)t_len;
    a.ndm = p->ndm;
    a.widths = p->dev.widths;
    a.nw = nw;
    a.off = p->dev.off;
    a.mu = p->dev.mu;
    a.isd = p->dev.isd;
    a.peak = peak;
    a.arg = arg;
    a.thresh = thresh;
    a.cands = cands;
    a.cap = cap;
    a.ncands = ncands;
    a.narrow = nullptr;
    a.narrow_sel = 0;
    a.status = p->dev.status;
    return dispatch_boxcar(p, a, widths, nw, s, true);
}

}  // namespace dd
