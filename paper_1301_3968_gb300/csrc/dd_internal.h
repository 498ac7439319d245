// Internal definitions shared by the host plan code and the CUDA launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "dd.h"

namespace dd {

// Dedispersion kernel geometry (see dd_dedisp.cu): a CTA has kWarps warps; a warp
// unit sums two adjacent trials (fp32 path) or one trial (exact integer and run-length
// paths), and each lane owns R consecutive output samples: kRPair on the pair path
// (packed accumulators and a duplicated window take 4 R registers), kRInt otherwise.
// R is odd so that lane-strided shared-memory reads hit distinct banks.  A warp's time
// chunk is 32 R outputs.
constexpr int kWarps = 8;
constexpr int kRPair = 27;
constexpr int kRInt = 31;
constexpr int kRMax = 31;
__host__ __device__ constexpr int lane_r(bool pair) { return pair ? kRPair : kRInt; }
__host__ __device__ constexpr int chunk_t(bool pair) { return 32 * lane_r(pair); }
// Start times per thread segment of the contiguous-width boxcar scan (k_boxcar_run):
// each segment's prefix chain starts at a multiple of kBoxSeg (odd: lane-strided shared
// loads are conflict-free).  The fused fp32 scan forms the same chains.
constexpr int kBoxSeg = 31;
constexpr int kRlUnits = 3;                // trials per warp on the run-length path
constexpr int kRlMinMeanTaps = 12;         // automatic run-length choice (uint8, unit weights)
// Bulk-copy pipeline depth (buffers in the ring) per path: the pair and run-length paths
// do more work per staged channel and gain more from large stages (up to kCsMax channels)
// than from depth; the integer path's stages are small and it keeps four in flight.
constexpr int kStagesPair = 2;
constexpr int kStagesRl = 2;
constexpr int kStagesInt = 4;
constexpr int kCsMax = 12;
constexpr int kStagesMax = 8;
constexpr int kSmemBudget = 110 * 1024;    // dynamic shared memory per CTA (two per SM)
constexpr int kSmemBudgetOne = 220 * 1024; // fallback: one CTA per SM
constexpr long long kWaitNs = 2000000000;  // bound on any device-side barrier wait

// Byte layout of one dedispersion pipeline stage in shared memory: cs staged input
// rows of lcap elements, then the stage's profile record.  The record holds, for each
// of the CTA's nu warp units and each of the stage's channels, an entry (window start
// relative to the block's minimum delay for the channel, taps) and, for fp32 plans,
// the per-tap weights of the unit's two trials as (w0, w1) pairs, packed one entry
// after another (kw pairs per record, the most any record needs).  An fp32 (pair)
// entry is 16 bytes: (trial 0's start, the larger of the two tap counts, trial 1's
// start minus trial 0's, offset of its weight pairs); tap k of the pair reads sample k
// of each trial's own run, so the pair sums max(n0, n1) taps.
// With shared difference rows (run-length path, `brow`) an entry is (run start, index of
// its tap count in the channel's list) and the record ends with, per channel, its at
// most two tap counts and the length of each one's difference row (n0, n1, len0, len1).
// The CTA then also holds two halves (stage i uses half i & 1), each with cs x 2
// difference rows of blen words and a copy of the stage's nu x cs entries (`bbytes`,
// outside the ring).  Records are stored in this layout in global memory
// ([block][stage][rec_bytes]) and staged by one bulk copy.
struct StageGeom {
    int rows_bytes, rec_off, rec_bytes, w_off, bytes, bbytes, bhalf_words;
    __host__ __device__ StageGeom(int esz, bool has_w, int lcap, int kw, int cs, int nu,
                                  bool brow = false, int blen = 0) {
        rows_bytes = (cs * lcap * esz + 15) & ~15;
        rec_off = rows_bytes;
        w_off = (has_w ? 16 : 8) * nu * cs;
        rec_bytes = (w_off + (has_w ? 8 * kw : 0) + (brow ? 16 * cs : 0) + 15) & ~15;
        bytes = (rec_off + rec_bytes + 127) & ~127;
        bhalf_words = brow ? ((cs * 2 * blen + 2 * nu * cs + 3) & ~3) : 0;
        bbytes = 2 * bhalf_words * 4;
    }
};

// Shared memory of a dedispersion CTA beyond its stages: the block's per-channel
// minimum delays and the pipeline's barriers and counters.
__host__ __device__ inline int dedisp_smem_bytes(const StageGeom& g, int nbuf, int nchan) {
    return nbuf * g.bytes + ((4 * nchan + 15) & ~15) + g.bbytes + nbuf * 8 + 2 * nbuf * 4;
}
// The output transpose reuses the stage buffers: one row of 32 * R values per warp.
constexpr int kStoreBytes = kWarps * 32 * kRMax * 4;

// Arguments of one dedispersion launch (one plan, one input block); the batched
// kernel keeps one per beam in device memory.
struct DedispArgs {
    const void* in;
    int64_t ld;
    int64_t t_offset;
    void* out;
    int64_t out_ld;
    int32_t t_out;
    const unsigned char* rec;  // [nblk][nst][rec_bytes]
    const int32_t* blk_lo;     // [nblk][nchan]
    int32_t nchan;
    int32_t ndm;
    int32_t lcap;
    int32_t blen;  // difference-row stride (run-length path with shared rows)
    int32_t cs;   // channels per stage
    int32_t nch;  // time chunks per CTA (trials per CTA = kWarps / nch)
    int32_t kpad;  // weight pairs per stage record (pair path)
    int32_t nsplit;    // channel-sum splits (grid z); split z writes out + z * split_ld
    int64_t split_ld;
    int32_t* status;
    int32_t skip_stage;
    int64_t wait_ns;
    uint32_t smem_bytes;  // dynamic shared memory of the launch
};

// The boxcar scan fused into the dedispersion CTAs (contiguous widths w0 .. w0 + nw - 1;
// dd_fused.cu).  The launch's items (trial block, time tile), block-major, are cut into
// nparts contiguous parts, one CTA each.  A CTA walks its part's items in order and
// scans each finished tile in shared memory, with the last C outputs of the previous tile of the same block carried
// in front of it (through `carry`, a per-part global buffer).
// Windows that a part boundary inside a trial block separates from their data are
// scanned afterwards from `seam`, which holds C outputs on each side of such a boundary.
// Maxima are merged in `key` as (value, earliest start) packed into one 64-bit word.
// Integer plans: C = wmax - 1 and exact sums.  fp32 plans: the sums of the unfused fp32
// scan, whose prefix chains start at multiples of kBoxSeg outputs, so C = wmax +
// kBoxSeg - 2 reaches back to the chain start of every window a tile owns.
struct FusedArgs {
    int32_t w0, nw;
    int32_t C;          // carried outputs: wmax - 1 (integer), wmax + kBoxSeg - 2 (fp32)
    int32_t rowlen;     // shared-memory row stride (4-byte words)
    int32_t nparts;
    int32_t tiles;      // time tiles per trial block; item = block * tiles + tile
    int32_t mlim;       // largest |x - o| for which every width-wmax sum fits int32
    const int64_t* starts;    // [nparts + 1] first item of each part
    const int64_t* order;     // [nparts] part taken by CTA i: parts sorted by their first
                              // time tile, so that CTAs resident together read the same
                              // input columns (shared in L2)
    const double* off;        // [ndm] per-trial offsets (integer valued on integer plans)
    unsigned long long* key;  // [ndm][nw]
    int32_t* carry;     // [nparts][trials per CTA][C] (fp32 plans: float bits)
    int32_t* seam;      // [nparts][trials per CTA][2 C]; entry s: boundary between parts s-1, s
};

// Shared-memory rows of the fused scan: nrow rows of `rowlen` ints (C carried outputs,
// the tile, 32 spare), then C + 48 ints that the last row's reads may run into; the
// run-length path's other trials' sums follow (fused_smem_for).
__host__ __device__ inline int fused_rows_ints(int nrow, int rowlen, int C) { return nrow * rowlen + C + 48; }

// Packs a boxcar sum and its start so that the larger sum, then the earlier start,
// compares larger; 0 stands for "no window".
__host__ __device__ inline unsigned long long fused_key(int v, int t) {
    return ((unsigned long long)((uint32_t)v ^ 0x80000000u) << 32) | (unsigned long long)(0xffffffffu - (uint32_t)t);
}

// The fp32 form: the float's bits mapped to an unsigned order (negative values with every
// bit flipped, others with the sign bit set) after -0 is made +0, so that equal sums
// compare equal and the earlier start wins, as in the unfused scan's comparisons.
#ifdef __CUDACC__
// max(a, b, c): one three-input max.f32 for fp32 (maxima are exact, so any grouping
// gives the same value), pairwise for the integer types.
__device__ __forceinline__ float max3(float a, float b, float c) {
    float m;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(m) : "f"(a), "f"(b), "f"(c));
    return m;
}
__device__ __forceinline__ int max3(int a, int b, int c) { return max(max(a, b), c); }
__device__ __forceinline__ long long max3(long long a, long long b, long long c) { return max(max(a, b), c); }

__device__ __forceinline__ unsigned long long fused_key_f32(float v, int t) {
    const uint32_t u = __float_as_uint(v == 0.f ? 0.f : v);
    const uint32_t o = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)o << 32) | (unsigned long long)(0xffffffffu - (uint32_t)t);
}
__device__ __forceinline__ float fused_key_value_f32(unsigned long long k) {
    const uint32_t o = (uint32_t)(k >> 32);
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}
#endif

// One work item of the batched dedispersion kernel: a CTA tile of one beam.
struct BatchItem {
    int32_t beam;
    int32_t blk;   // trial block
    int32_t tx;    // time tile
    int32_t pad;
};

struct DevTables {
    int device = -1;
    int32_t* delay = nullptr;   // [ndm][nchan]
    int32_t* taps = nullptr;    // [ndm][nchan]
    float* w = nullptr;         // [ndm][nchan][kpad]  (weighted plans)
    int32_t* blk_lo = nullptr;  // [nblk][nchan] minimum delay over the CTA's trials
    unsigned char* rec = nullptr;  // [nblk][nstage][rec_bytes] staged profile records
    int32_t* status = nullptr;  // device status word (0 = ok)
    // boxcar normaliser workspace
    double* off = nullptr;      // [ndm]  per-trial offset subtracted before summing
    float* mu = nullptr;        // [ndm][ws_w] mean of B_w minus w*off
    float* isd = nullptr;       // [ndm][ws_w] 1/sigma_dw
    int32_t* widths = nullptr;  // [ws_w]
    int32_t ws_w = 0;
    uint8_t* narrow = nullptr;  // [ndm] 1 where a row's boxcar sums fit int32
};

}  // namespace dd

struct dd_plan_s {
    dd_band band{};
    int32_t nchan = 0, ndm = 0;
    std::vector<double> dms;
    std::vector<int32_t> delay, taps;  // [ndm][nchan]
    std::vector<float> w;              // [ndm][nchan][kpad], empty for unit weights
    int32_t kpad = 0;                  // weight row stride (multiple of 4) or 0
    int32_t kuser = 0;                 // caller's weight row length (kmax argument)
    bool unit = true;
    int32_t kmax = 1, dmax = 0;
    int64_t ns_total = 0;
    bool out_int = true;               // int32 sums (uint8 input, unit weights)
    int64_t max_abs_row = 0;           // bound on |out| for integer plans
    // dedispersion schedule
    int32_t nblk = 0;
    std::vector<int32_t> blk_lo;       // [nblk][nchan] minimum delay over the block's trials
    int32_t lcap = 0;                  // staged row length (elements)
    int32_t cs = 4;                    // channels per pipeline stage
    int32_t nch = 1;                   // time chunks per CTA
    int32_t rec_bytes = 0;             // bytes of one stage's profile record
    bool pair = true;                  // fp32 path: each warp sums two adjacent trials
    int32_t kw = 0;                    // weight pairs per stage record (pair path)
    int32_t umax = 0;                  // most taps of a pair unit, max(n0, n1) (pair path)
    std::vector<unsigned char> rec;    // host copy of the records
    bool rec_from_dev_w = false;       // records' weights come from dev.w (device weights)
    int32_t debug_skip_stage = -1;     // test hook: a stage whose bulk copies are never issued
    int64_t wait_ns = dd::kWaitNs;
    bool dev_dirty = true;
    dd::DevTables dev;
    std::vector<int32_t> widths_on_dev;  // widths last copied to dev.widths
    // adjoint workspace, built on the first dd_backward: the transposed plan (output rows
    // = channels, input rows = trials) whose dedispersion is the input gradient, and the
    // zero-padded copy of the output gradient it reads
    dd_plan_s* adj = nullptr;
    bool adj_stale = true;             // forward delays or taps changed since it was built
    bool adj_w_stale = true;           // forward weights changed since they were transposed
    float* d_gpad = nullptr;
    int64_t gpad_elems = 0;
    int32_t bw_span = 0;               // widest delay spread of 8 consecutive trials
    float* d_gsplit = nullptr;         // partial input gradients of a split adjoint sum
    int64_t gsplit_elems = 0;
    // tap sums: direct multiply-adds, or differences of per-channel prefix sums
    // (run-length path; uint8 unit weights), and that path's prefix scratch
    int32_t method = DD_METHOD_AUTO;   // requested
    bool rl = false;                   // in use
    bool rl_b = false;                 // run-length with difference rows shared by the CTA
    int32_t blen = 0;                  // their stride (words)
    uint32_t* d_prefix = nullptr;
    int64_t prefix_elems = 0;
    // fused dedispersion + boxcar scratch: merged maxima, per-CTA carries, strip seams
    unsigned long long* d_fkey = nullptr;
    int64_t fkey_elems = 0;
    int32_t* d_fcarry = nullptr;
    int64_t fcarry_elems = 0;
    int32_t* d_fseam = nullptr;
    int64_t fseam_elems = 0;
    int64_t* d_fstarts = nullptr;
    std::vector<int64_t> fstarts;      // the parts of the last fused launch (host copy)
    int32_t debug_fused_parts = 0;     // test hook: parts of a fused launch (0 = automatic)
};

namespace dd {

dd_status upload_tables(dd_plan_s* p);  // (re)creates the device tables if dirty
dd_status build_adjoint_plan(dd_plan_s* p);  // (re)builds p->adj on the host
void destroy_plan(dd_plan_s* p);
dd_status launch_repack(dd_plan_s* p, cudaStream_t s);  // dev.w -> records' weights
void fill_dedisp_args(const dd_plan_s* p, const void* in, int64_t ld, int64_t t_offset,
                      int64_t t_out, void* out, int64_t out_ld, DedispArgs* a);
size_t dedisp_smem_for(const dd_plan_s* p);
dd_status launch_dedisperse_rl(dd_plan_s* p, const void* in, int64_t ld, int64_t t_offset,
                               int64_t nsamp, void* out, int64_t out_ld, cudaStream_t s);
dd_status launch_dedisperse_batched(bool u8, bool pair, bool short_taps, const DedispArgs* d_args,
                                    const BatchItem* d_items, int32_t nitems, size_t smem, cudaStream_t s,
                                    bool rl = false);
int dedisp_batched_blocks_per_sm(bool u8, bool pair, bool short_taps, size_t smem, bool rl = false);
dd_status launch_prefix_into(const dd_plan_s* p, const void* in, int64_t ld, int64_t t_offset,
                             int64_t nsamp, uint32_t* P, int64_t ldp, cudaStream_t s);
dd_status cuda_status(cudaError_t e);

// launchers (stream = cudaStream_t)
dd_status launch_dedisperse(dd_plan_s* p, const void* in, int64_t ld, int64_t t_offset,
                            int64_t t_out, void* out, int64_t out_ld, cudaStream_t s,
                            int nsplit = 1, int64_t split_ld = 0);
dd_status launch_channel_stats(dd_plan_s* p, const void* in, int64_t ld, int64_t t_offset,
                               int64_t nsamp, double* mean, double* sd, cudaStream_t s);
dd_status launch_boxcar(dd_plan_s* p, const void* x, int64_t ld, int64_t t_len,
                        const int32_t* widths, int32_t nw, const double* mean,
                        const double* sd, float* peak, int32_t* arg, float thresh,
                        dd_candidate* cands, int32_t cap, int32_t* ncands, cudaStream_t s);
dd_status launch_boxcar_scratch(dd_plan_s* p, const void* x, int64_t ld, int64_t t_len,
                                const int32_t* widths, int32_t nw, const int32_t* widths_dev,
                                const double* mean, const double* sd, double* off, float* mu,
                                float* isd, float* peak, int32_t* arg, float thresh,
                                dd_candidate* cands, int32_t cap, int32_t* ncands, cudaStream_t s);
dd_status launch_prefix(dd_plan_s* p, const void* in, int64_t ld, int64_t t_offset, int64_t nsamp,
                        int64_t* ldp, cudaStream_t s);
dd_status launch_norm(dd_plan_s* p, const int32_t* widths, int32_t nw, const double* mean,
                      const double* sd, cudaStream_t s);
// fused dedispersion + boxcar: dynamic shared memory of the launch (stages, or the scan
// rows plus the pipeline barriers, whichever is larger), its CTAs per SM, and the launch
size_t fused_smem_for(const dd_plan_s* p, int rowlen, int C);
int fused_blocks_per_sm(const dd_plan_s* p, size_t smem);
dd_status launch_dedisperse_fused(const dd_plan_s* p, DedispArgs a, const FusedArgs& f, size_t smem,
                                  cudaStream_t s);
// allocation-free boxcar path: loads its kernels and its static scratch array onto the
// current device (once per device; called when a plan's tables are uploaded)
dd_status preload_boxcar_kernels();
dd_status noalloc_preload();
dd_status launch_backward(dd_plan_s* p, const float* in, int64_t ld, int64_t t_offset,
                          int64_t t_out, const float* g, int64_t gld, float* gw, float* gin,
                          int64_t gin_ld, cudaStream_t s);

}  // namespace dd
