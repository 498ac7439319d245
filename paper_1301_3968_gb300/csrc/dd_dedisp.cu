// Profiled dedispersion, eq. p_dedisp (Sec. 2.1):
//
//   out[d][t] = sum_c sum_{k < n_dc} w_dck * I[c][t_offset + t + delta_dc + k]
//
// Work decomposition (sm_103a):
//   * A CTA has kWarps = 8 warps covering db consecutive trials x nch time chunks
//     (db * nch = 8); a chunk is 32 * kR outputs and lane l owns outputs
//     chunk_start + l*kR + r, r < kR.  The plan picks the largest db whose staged
//     window fits in shared memory (db = 8 whenever neighbouring trials have close
//     delays, as every trial list of eq. trial DMs does).
//   * Channels are streamed in stages of cs rows.  For each channel the CTA stages
//     the window that all its trials read -- [T0 + min delta, T0 + tile + max(delta + n))
//     rounded to 16-byte chunks -- into shared memory with cp.async, NBUF stages deep,
//     so every staged sample is reused by db trials x up to n_dc taps.
//   * Inner loop: a register window of kR samples slides along the taps; each tap
//     costs one shared-memory load, one weight broadcast and kR FMAs (or integer
//     adds).  kR is odd, so the lane-strided loads hit 32 distinct banks.
//   * fp32 sums accumulate each stage's channels in a fresh partial that is then
//     added to the running total (two-level summation); uint8 unit-weight sums are
//     exact int32.
//   * Results are transposed through shared memory so that global stores coalesce.
#include <cstdint>

#include "dd_internal.h"

namespace dd {
namespace {

struct DedispArgs {
    const void* in;
    int64_t ld;
    int64_t t_offset;
    void* out;
    int64_t out_ld;
    int32_t t_out;
    const int32_t* delay;
    const int32_t* taps;
    const float* w;
    int32_t kpad;
    const int32_t* blk_lo;
    int32_t nchan;
    int32_t ndm;
    int32_t lcap;
    int32_t cs;   // channels per stage
    int32_t nch;  // time chunks per CTA (trials per CTA = kWarps / nch)
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
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

template <typename TACC, typename TIN>
__device__ __forceinline__ TACC cvt(TIN v) {
    return (TACC)v;
}

template <typename TIN, bool UNIT>
struct StageLayout : StageBytes {
    __host__ __device__ StageLayout(int lcap, int kpad, int cs)
        : StageBytes((int)sizeof(TIN), UNIT, lcap, kpad, cs) {}
};

template <typename TIN, bool UNIT>
__device__ __forceinline__ void load_stage(const DedispArgs& a, unsigned char* buf,
                                           const StageLayout<TIN, UNIT>& L, int stage,
                                           int blk, int64_t t0) {
    constexpr int Q = Elem<TIN>::Q;
    const int CS = a.cs;
    const int db = kWarps / a.nch;
    const int tid = threadIdx.x;
    const int c0 = stage * CS;
    const int csn = min(CS, a.nchan - c0);
    const int nq = a.lcap / Q;
    const TIN* in = (const TIN*)a.in;
    const int64_t base = a.t_offset + t0;
    // staged rows: chunk j of channel ci holds global columns a0 + j*Q .. +Q-1
    for (int idx = tid; idx < csn * nq; idx += blockDim.x) {
        const int ci = idx / nq;
        const int j = idx - ci * nq;
        const int c = c0 + ci;
        const int64_t a0 = (base + a.blk_lo[(int64_t)blk * a.nchan + c]) / Q * Q;
        const int64_t g = a0 + (int64_t)j * Q;
        unsigned char* dst = buf + ((int64_t)ci * a.lcap + (int64_t)j * Q) * sizeof(TIN);
        if (g + Q <= a.ld) {
            cp_async16(dst, in + (int64_t)c * a.ld + g);
        } else {
            *(uint4*)dst = make_uint4(0, 0, 0, 0);
        }
    }
    int* e = (int*)(buf + L.e_off);
    int* dl = (int*)(buf + L.dl_off);
    int* tp = (int*)(buf + L.tp_off);
    for (int i = tid; i < CS; i += blockDim.x) {
        const int c = c0 + i;
        int ev = 0;
        if (i < csn) {
            const int64_t a0 = (base + a.blk_lo[(int64_t)blk * a.nchan + c]) / Q * Q;
            ev = (int)(base - a0);
        }
        e[i] = ev;
    }
    for (int idx = tid; idx < db * CS; idx += blockDim.x) {
        const int wi = idx / CS, ci = idx - wi * CS;
        const int d = blk * db + wi;
        int dv = 0, tv = 0;
        if (ci < csn && d < a.ndm) {
            dv = a.delay[(int64_t)d * a.nchan + c0 + ci];
            tv = a.taps[(int64_t)d * a.nchan + c0 + ci];
        }
        dl[idx] = dv;
        tp[idx] = tv;
    }
    if (!UNIT) {
        // weights [d][c0 .. c0+csn)[kpad] are contiguous for each trial d
        const int nchunk = csn * a.kpad / 4;
        float* wdst = (float*)(buf + L.w_off);
        for (int idx = tid; idx < db * nchunk; idx += blockDim.x) {
            const int wi = idx / nchunk, j = idx - wi * nchunk;
            const int d = blk * db + wi;
            float* dst = wdst + (int64_t)wi * CS * a.kpad + j * 4;
            if (d < a.ndm)
                cp_async16(dst, a.w + ((int64_t)d * a.nchan + c0) * a.kpad + j * 4);
            else
                *(float4*)dst = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

template <typename TIN, typename TACC, bool UNIT, int NBUF>
__global__ void __launch_bounds__(kWarps * 32, 2) k_dedisp(DedispArgs a) {
    constexpr int R = kR;
    extern __shared__ __align__(128) unsigned char smem[];
    const int CS = a.cs;
    const StageLayout<TIN, UNIT> L(a.lcap, a.kpad, CS);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int blk = blockIdx.y;
    const int dmi = warp / a.nch, chunk = warp - dmi * a.nch;
    const int d = blk * (kWarps / a.nch) + dmi;
    const int64_t t0 = (int64_t)blockIdx.x * kTileT * a.nch;   // CTA time start
    const int64_t tw = t0 + (int64_t)chunk * kTileT;            // warp time start
    const int nst = (a.nchan + CS - 1) / CS;

    TACC acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = TACC(0);

#pragma unroll
    for (int s = 0; s < NBUF - 1; ++s) {
        if (s < nst) load_stage<TIN, UNIT>(a, smem + s * L.bytes, L, s, blk, t0);
        cp_commit();
    }

    for (int s = 0; s < nst; ++s) {
        const int sn = s + NBUF - 1;
        if (sn < nst) load_stage<TIN, UNIT>(a, smem + (sn % NBUF) * L.bytes, L, sn, blk, t0);
        cp_commit();
        cp_wait<NBUF - 1>();
        __syncthreads();

        if (d < a.ndm) {
            const unsigned char* buf = smem + (s % NBUF) * L.bytes;
            const TIN* rows = (const TIN*)buf;
            const int* e = (const int*)(buf + L.e_off);
            const int* dl = (const int*)(buf + L.dl_off) + dmi * CS;
            const int* tp = (const int*)(buf + L.tp_off) + dmi * CS;
            const float* wts = (const float*)(buf + L.w_off) + dmi * CS * a.kpad;
            const int csn = min(CS, a.nchan - s * CS);
            TACC part[R];
#pragma unroll
            for (int r = 0; r < R; ++r) part[r] = TACC(0);
            for (int ci = 0; ci < csn; ++ci) {
                const int n = tp[ci];
                const TIN* p = rows + ci * a.lcap + e[ci] + dl[ci] + chunk * kTileT + lane * R;
                const float* wk = wts + ci * a.kpad;
                TACC win[R];
#pragma unroll
                for (int j = 0; j < R; ++j) win[j] = cvt<TACC>(p[j]);
                for (int k0 = 0; k0 < n; k0 += R) {
#pragma unroll
                    for (int kk = 0; kk < R; ++kk) {
                        if (k0 + kk >= n) break;
                        if (UNIT) {
#pragma unroll
                            for (int r = 0; r < R; ++r) part[r] += win[(r + kk) % R];
                        } else {
                            const float wv = wk[k0 + kk];
#pragma unroll
                            for (int r = 0; r < R; ++r) part[r] = fmaf(wv, (float)win[(r + kk) % R], (float)part[r]);
                        }
                        win[kk] = cvt<TACC>(p[R + k0 + kk]);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] += part[r];
        }
        __syncthreads();
    }

    // transpose through shared memory and store coalesced
    TACC* st = (TACC*)smem + warp * (32 * R);
#pragma unroll
    for (int r = 0; r < R; ++r) st[lane * R + r] = acc[r];
    __syncwarp();
    if (d < a.ndm) {
        TACC* out = (TACC*)a.out + (int64_t)d * a.out_ld;
#pragma unroll 4
        for (int j = 0; j < R; ++j) {
            const int64_t t = tw + j * 32 + lane;
            if (t < a.t_out) out[t] = st[j * 32 + lane];
        }
    }
}

template <typename TIN, typename TACC, bool UNIT, int NBUF>
dd_status run(const DedispArgs& a, cudaStream_t s) {
    const StageLayout<TIN, UNIT> L(a.lcap, a.kpad, a.cs);
    size_t smem = (size_t)NBUF * L.bytes;
    const size_t st_bytes = (size_t)kWarps * 32 * kR * sizeof(TACC);
    if (smem < st_bytes) smem = st_bytes;
    auto kern = k_dedisp<TIN, TACC, UNIT, NBUF>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e);
    const int64_t tile = (int64_t)kTileT * a.nch;
    const int db = kWarps / a.nch;
    dim3 grid((unsigned)((a.t_out + tile - 1) / tile), (unsigned)((a.ndm + db - 1) / db));
    if (grid.y > 65535) return DD_ERR_UNSUPPORTED;
    kern<<<grid, kWarps * 32, smem, s>>>(a);
    return cuda_status(cudaGetLastError());
}

}  // namespace

dd_status launch_dedisperse(dd_plan_s* p, const void* in, int64_t ld, int64_t t_offset,
                            int64_t t_out, void* out, int64_t out_ld, cudaStream_t s) {
    DedispArgs a;
    a.in = in;
    a.ld = ld;
    a.t_offset = t_offset;
    a.out = out;
    a.out_ld = out_ld;
    a.t_out = (int32_t)t_out;
    a.delay = p->dev.delay;
    a.taps = p->dev.taps;
    a.w = p->dev.w;
    a.kpad = p->kpad;
    a.blk_lo = p->dev.blk_lo;
    a.nchan = p->nchan;
    a.ndm = p->ndm;
    a.lcap = p->lcap;
    a.cs = p->cs;
    a.nch = p->nch;
    const bool u8 = p->band.in_type == DD_U8;
    if (u8 && p->unit) return run<uint8_t, int, true, kStages>(a, s);
    if (u8) return run<uint8_t, float, false, kStages>(a, s);
    if (p->unit) return run<float, float, true, kStages>(a, s);
    return run<float, float, false, kStages>(a, s);
}

}  // namespace dd
