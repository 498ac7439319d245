// Adjoint of the weighted dedispersion map (no counterpart in the paper; it is the
// transpose of eq. p_dedisp, needed to optimise profile weights by gradient ascent).
//
//   gw[d][c][k] = sum_t g[d][t] * I[c][t_offset + t + delta_dc + k]          (k < n_dc)
//   gI[c][tau]  = sum_d sum_{k < n_dc} w_dck * g[d][tau - t_offset - delta_dc - k]
//
// gI is itself a dedispersion with rows and columns swapped (see build_adjoint_plan):
// the output gradient is copied into a zero-padded buffer (k_pad_rows), the forward
// weights are transposed and reversed into the adjoint plan (k_transpose_w, then the
// adjoint plan's record repack), and the forward dedispersion kernel runs on it.
//
// gw is a correlation of each trial's gradient row with the shifted channel row, for
// the tap lags k: k_bwd_w gives each warp one (trial, channel) pair and its 32 lags in
// registers, as 16 packed lag pairs (k, k + 16) updated by fma.rn.f32x2; lanes own 33
// consecutive samples (odd, so lane-strided shared loads are conflict free) and slide a
// window of 16 sample pairs (x[p], x[p + 16]) along them; the lanes' partial sums are
// added in a fixed order at the end.  Both paths are deterministic.
#include <algorithm>
#include <cstdint>

#include "dd_async.cuh"
#include "dd_internal.h"
#include "dd_packed.cuh"

namespace dd {
namespace {

constexpr int kLags = 32;          // lags per pass of k_bwd_w
constexpr int kSeg = 33;           // samples per lane per tile
constexpr int kTileW = 32 * kSeg;  // samples per tile

__global__ void k_pad_rows(const float* g, int64_t gld, int32_t t_out, int32_t pad, float* gp,
                           int64_t gpld, int32_t rows) {
    const int d = blockIdx.y;
    if (d >= rows) return;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < gpld; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = v - pad;
        gp[(int64_t)d * gpld + v] = (u >= 0 && u < t_out) ? g[(int64_t)d * gld + u] : 0.f;
    }
}

// Wt[c][d][j] = w[d][c][n_dc - 1 - j] for j < n_dc, zero beyond.
__global__ void k_transpose_w(const float* w, const int32_t* taps, int32_t ndm, int32_t nchan,
                              int32_t kpad, float* wt) {
    const int64_t n = (int64_t)ndm * nchan;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(i / nchan), c = (int)(i - (int64_t)d * nchan);
        const int nt = taps[i];
        const float* src = w + i * kpad;
        float* dst = wt + ((int64_t)c * ndm + d) * kpad;
        for (int j = 0; j < kpad; ++j) dst[j] = j < nt ? src[nt - 1 - j] : 0.f;
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// grid (trial blocks of 8, channels).  Shared memory: two buffers, each the channel's
// window for the block's 8 trials and the 8 gradient rows of one tile of kTileW
// outputs; the next tile's copies (cp.async, zero-filled past the ends of the rows)
// are in flight while the current one is summed.
__global__ void __launch_bounds__(256, 2) k_bwd_w(const float* in, int64_t ld, int64_t t_offset,
                                               int32_t t_out, const float* g, int64_t gld,
                                               const int32_t* delay, const int32_t* taps,
                                               int32_t nchan, int32_t ndm, int32_t kpad,
                                               int32_t kout, int32_t span, float* gw) {
    extern __shared__ float sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.y;
    const int d = blockIdx.x * 8 + warp;
    const int xlen = kTileW + span + kpad + 1;
    const int xstride = (xlen + 3) & ~3;
    float* const buf0 = sm;                          // [xlen] then [8][kTileW]
    float* const buf1 = sm + xstride + 8 * kTileW;
    __shared__ int s_lo;
    __shared__ int s_del[8], s_tap[8];
    if (threadIdx.x < 8) {
        const int dd = blockIdx.x * 8 + threadIdx.x;
        s_del[threadIdx.x] = dd < ndm ? delay[(int64_t)dd * nchan + c] : INT32_MAX;
        s_tap[threadIdx.x] = dd < ndm ? taps[(int64_t)dd * nchan + c] : 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int lo = INT32_MAX;
        for (int i = 0; i < 8; ++i) lo = min(lo, s_del[i]);
        s_lo = lo;
    }
    __syncthreads();
    const int lo = s_lo;
    const bool active = d < ndm;
    const int off = active ? s_del[warp] - lo : 0;
    const int n = active ? s_tap[warp] : 0;
    const float* row = in + (int64_t)c * ld + t_offset + lo;
    const int64_t row_end = ld - t_offset - lo;  // columns available in the row
    const int ntile = (t_out + kTileW - 1) / kTileW;
    // the CTA stages the channel window shared by its 8 trials; each warp stages its own
    // trial's gradient segment (a full tile needs no bounds tests)
    auto stage = [&](int t0, float* B) {
        float* xs = B;
        for (int i = threadIdx.x; i < xlen; i += blockDim.x) {
            const int64_t col = (int64_t)t0 + i;
            const bool ok = col < row_end;
            cp_async4(xs + i, ok ? row + col : in, ok);
        }
        float* gs = B + xstride + warp * kTileW;
        if (active && t0 + kTileW <= t_out) {
            const float* grow = g + (int64_t)d * gld + t0 + lane;
#pragma unroll
            for (int j = 0; j < kSeg; ++j) cp_async4(gs + j * 32 + lane, grow + j * 32, true);
        } else {
            for (int j = 0; j < kSeg; ++j) {
                const int tt = j * 32 + lane;
                const bool ok = active && t0 + tt < t_out;
                cp_async4(gs + tt, ok ? g + (int64_t)d * gld + t0 + tt : g, ok);
            }
        }
        cp_async_commit();
    };
    for (int kc = 0; kc < kout; kc += kLags) {
        // lags in packed pairs (k, k + 16), k < 16
        constexpr int H = kLags / 2;
        uint64_t acc2[H];
#pragma unroll
        for (int k = 0; k < H; ++k) acc2[k] = 0ull;
        stage(0, buf0);
        for (int it = 0; it < ntile; ++it) {
            if (it + 1 < ntile) {
                stage((it + 1) * kTileW, (it & 1) ? buf0 : buf1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            if (active && kc < n) {
                const float* xs = (it & 1) ? buf1 : buf0;
                const float* x = xs + off + kc + lane * kSeg;
                const float* gv = xs + xstride + warp * kTileW + lane * kSeg;
                // window of sample pairs (x[p], x[p + 16]) for positions p = tt .. tt + 15,
                // position p in register p mod 16; lag pair k reads position tt + k
                uint64_t win[H];
#pragma unroll
                for (int k = 0; k < H; ++k) win[k] = pk2(x[k], x[k + H]);
#pragma unroll
                for (int tt = 0; tt < kSeg; ++tt) {
                    const uint64_t gt = pk_dup(gv[tt]);
#pragma unroll
                    for (int k = 0; k < H; ++k) fma2(acc2[k], gt, win[(k + tt) % H]);
                    win[tt % H] = pk2(x[tt + H], x[tt + kLags]);
                }
            }
            __syncthreads();  // this buffer is restaged by the next iteration but one
        }
        if (active) {
            float acc[kLags];
#pragma unroll
            for (int k = 0; k < H; ++k) unpk(acc2[k], acc[k], acc[k + H]);
#pragma unroll
            for (int k = 0; k < kLags; ++k) {
                const float v = warp_sum(acc[k]);
                if (lane == 0 && kc + k < kout) gw[((int64_t)d * nchan + c) * kout + kc + k] = (kc + k < n) ? v : 0.f;
            }
        }
    }
}

// gI[c][tau] = sum over splits of the partial sums (fixed order: deterministic).
__global__ void k_sum_splits(const float* part, int32_t nsplit, int64_t split_ld, int32_t rows,
                             int64_t n, int64_t pld, float* gin, int64_t gin_ld) {
    const int c = blockIdx.y;
    if (c >= rows) return;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        float v = 0.f;
        for (int z = 0; z < nsplit; ++z) v += part[z * split_ld + (int64_t)c * pld + t];
        gin[(int64_t)c * gin_ld + t] = v;
    }
}

}  // namespace

dd_status launch_backward(dd_plan_s* p, const float* in, int64_t ld, int64_t t_offset,
                          int64_t t_out, const float* g, int64_t gld, float* gw, float* gin,
                          int64_t gin_ld, cudaStream_t s) {
    if (p->unit) return DD_ERR_UNSUPPORTED;  // gradients need a weighted plan
    cudaError_t e;
    if (gw) {
        const int xlen = kTileW + p->bw_span + p->kpad + 1;
        const size_t smem = (size_t)2 * (((xlen + 3) & ~3) + 8 * kTileW) * sizeof(float);
        if (smem > 200 * 1024) return DD_ERR_UNSUPPORTED;
        e = cudaFuncSetAttribute(k_bwd_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_status(e);
        dim3 grid((unsigned)((p->ndm + 7) / 8), (unsigned)p->nchan);
        k_bwd_w<<<grid, 256, smem, s>>>(in, ld, t_offset, (int32_t)t_out, g, gld, p->dev.delay,
                                        p->dev.taps, p->nchan, p->ndm, p->kpad, p->kuser,
                                        p->bw_span, gw);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (gin) {
        dd_status st;
        if (!p->adj || p->adj_stale) {
            st = build_adjoint_plan(p);
            if (st != DD_OK) return st;
        }
        dd_plan_s* t = p->adj;
        st = upload_tables(t);
        if (st != DD_OK) return st;
        const int32_t P = p->dmax;
        const int64_t nsamp = t_out + P;
        // padded gradient rows: P zeros, t_out values, zeros up to a 16-byte multiple
        int64_t gpld = t_out + 2 * (int64_t)P + 1;
        gpld = (gpld + 3) & ~(int64_t)3;
        const int64_t need = gpld * p->ndm;
        if (need > p->gpad_elems) {
            cudaFree(p->d_gpad);
            p->d_gpad = nullptr;
            p->gpad_elems = 0;
            e = cudaMalloc((void**)&p->d_gpad, (size_t)need * sizeof(float));
            if (e != cudaSuccess) return cuda_status(e);
            p->gpad_elems = need;
        }
        dim3 pg((unsigned)std::min<int64_t>((gpld + 255) / 256, 64), (unsigned)p->ndm);
        k_pad_rows<<<pg, 256, 0, s>>>(g, gld, (int32_t)t_out, P, p->d_gpad, gpld, p->ndm);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_status(e);
        if (p->adj_w_stale) {
            k_transpose_w<<<1024, 256, 0, s>>>(p->dev.w, p->dev.taps, p->ndm, p->nchan, p->kpad, t->dev.w);
            e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_status(e);
            st = launch_repack(t, s);
            if (st != DD_OK) return st;
            p->adj_w_stale = false;
        }
        // gI[c][t_offset + tau] for tau in [0, nsamp): the adjoint plan's outputs.  Its
        // few output rows (channels) give few CTAs; when they would not fill the GPU
        // about four times over, the sum over its input rows (trials) is split across
        // grid z into partial sums that k_sum_splits adds in a fixed order.
        int sms = 0, dev = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_status(e);
        const int64_t tile = (int64_t)chunk_t(true) * t->nch;
        const int64_t db = (int64_t)2 * (kWarps / t->nch);
        const int64_t ctas = ((nsamp + tile - 1) / tile) * ((t->ndm + db - 1) / db);
        const int nst = (t->nchan + t->cs - 1) / t->cs;
        int nsplit = (int)std::min<int64_t>(std::min<int64_t>(8, nst), (4LL * 2 * sms + ctas - 1) / ctas);
        if (nsplit <= 1) {
            st = launch_dedisperse(t, p->d_gpad, gpld, 0, nsamp, gin + t_offset, gin_ld, s);
            if (st != DD_OK) return st;
        } else {
            const int64_t pld = (nsamp + 3) & ~(int64_t)3;
            const int64_t split_ld = pld * t->ndm;
            if (split_ld * nsplit > p->gsplit_elems) {
                cudaFree(p->d_gsplit);
                p->d_gsplit = nullptr;
                p->gsplit_elems = 0;
                e = cudaMalloc((void**)&p->d_gsplit, (size_t)(split_ld * nsplit) * sizeof(float));
                if (e != cudaSuccess) return cuda_status(e);
                p->gsplit_elems = split_ld * nsplit;
            }
            st = launch_dedisperse(t, p->d_gpad, gpld, 0, nsamp, p->d_gsplit, pld, s, nsplit, split_ld);
            if (st != DD_OK) return st;
            dim3 sg((unsigned)std::min<int64_t>((nsamp + 255) / 256, 64), (unsigned)t->ndm);
            k_sum_splits<<<sg, 256, 0, s>>>(p->d_gsplit, nsplit, split_ld, t->ndm, nsamp, pld,
                                            gin + t_offset, gin_ld);
            e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_status(e);
        }
    }
    return DD_OK;
}

}  // namespace dd
