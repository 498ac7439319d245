// Adjoint of the weighted dedispersion map (no counterpart in the paper; it is the
// transpose of eq. p_dedisp, needed to optimise profile weights by gradient ascent).
//
//   gw[d][c][k] = sum_t g[d][t] * I[c][t_offset + t + delta_dc + k]          (k < n_dc)
//   gI[c][tau]  = sum_d sum_{k < n_dc} w_dck * g[d][tau - t_offset - delta_dc - k]
//
// k_bwd_w: one CTA per (trial, channel); threads stride over t with a register
// accumulator per tap (32 taps per pass), then a fixed-order CTA reduction.
// k_bwd_in: one thread per input column; the sum runs over trials, then taps, in
// ascending order, as a gather (no atomics), so it is deterministic.
#include <cstdint>

#include "dd_internal.h"

namespace dd {
namespace {

constexpr int kKc = 32;

__global__ void __launch_bounds__(256) k_bwd_w(const float* in, int64_t ld, int64_t t_offset,
                                               int32_t t_out, const float* g, int64_t gld,
                                               const int32_t* delay, const int32_t* taps,
                                               int32_t nchan, int32_t kpad, int32_t kout, float* gw) {
    const int c = blockIdx.x, d = blockIdx.y;
    const int64_t dc = (int64_t)d * nchan + c;
    const int n = taps[dc];
    const float* src = in + (int64_t)c * ld + t_offset + delay[dc];
    const float* gd = g + (int64_t)d * gld;
    __shared__ float red[8][kKc];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int kc = 0; kc < kpad; kc += kKc) {
        float acc[kKc];
#pragma unroll
        for (int k = 0; k < kKc; ++k) acc[k] = 0.f;
        const int kn = min(kKc, n - kc);
        if (kn > 0) {
            for (int t = threadIdx.x; t < t_out; t += blockDim.x) {
                const float gv = gd[t];
                const float* s = src + t + kc;
#pragma unroll
                for (int k = 0; k < kKc; ++k)
                    if (k < kn) acc[k] = fmaf(gv, s[k], acc[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < kKc; ++k) {
            float v = acc[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][k] = v;
        }
        __syncthreads();
        if (threadIdx.x < kKc && kc + (int)threadIdx.x < kout) {
            float v = 0.f;
            for (int i = 0; i < 8; ++i) v += red[i][threadIdx.x];
            gw[dc * kout + kc + threadIdx.x] = (kc + (int)threadIdx.x < n) ? v : 0.f;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_bwd_in(int64_t nsamp, int32_t t_out, const float* g,
                                                int64_t gld, const int32_t* delay,
                                                const int32_t* taps, const float* w, int32_t kpad,
                                                int32_t nchan, int32_t ndm, float* gin,
                                                int64_t gin_ld, int64_t t_offset) {
    const int c = blockIdx.y;
    const int64_t tau = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tau >= nsamp) return;
    float acc = 0.f;
    for (int d = 0; d < ndm; ++d) {
        const int64_t dc = (int64_t)d * nchan + c;
        const int n = taps[dc];
        const int64_t base = tau - delay[dc];
        const float* gd = g + (int64_t)d * gld;
        const float* wk = w + dc * kpad;
        for (int k = 0; k < n; ++k) {
            const int64_t t = base - k;
            if (t >= 0 && t < t_out) acc = fmaf(wk[k], gd[t], acc);
        }
    }
    gin[(int64_t)c * gin_ld + t_offset + tau] = acc;
}

}  // namespace

dd_status launch_backward(dd_plan_s* p, const float* in, int64_t ld, int64_t t_offset,
                          int64_t t_out, const float* g, int64_t gld, float* gw, float* gin,
                          int64_t gin_ld, cudaStream_t s) {
    if (p->unit) return DD_ERR_UNSUPPORTED;  // gradients need a weighted plan
    if (gw) {
        dim3 grid((unsigned)p->nchan, (unsigned)p->ndm);
        if (grid.y > 65535) return DD_ERR_UNSUPPORTED;
        k_bwd_w<<<grid, 256, 0, s>>>(in, ld, t_offset, (int32_t)t_out, g, gld, p->dev.delay,
                                     p->dev.taps, p->nchan, p->kpad, p->kuser, gw);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (gin) {
        const int64_t nsamp = t_out + p->dmax;
        dim3 grid((unsigned)((nsamp + 255) / 256), (unsigned)p->nchan);
        k_bwd_in<<<grid, 256, 0, s>>>(nsamp, (int32_t)t_out, g, gld, p->dev.delay, p->dev.taps,
                                      p->dev.w, p->kpad, p->nchan, p->ndm, gin, gin_ld, t_offset);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_status(e);
    }
    return DD_OK;
}

}  // namespace dd
