/*
 * dd.h -- C ABI of the GB300 profiled-dedispersion library (libdd.so).
 *
 * The library computes, for every trial dispersion measure d, the profiled
 * dedispersion sum of eq. p_dedisp (Sec. 2.1)
 *
 *     out[d][t] = sum_c sum_{k < n_dc} w_dck * I[c][t_offset + t + delta_dc + k]
 *
 * over a channelised filterbank I[c][t], followed by boxcar S/N detection over a
 * list of widths (eq. snr, Sec. 2.1, and the boxcar detector of Sec. 5).  Each trial
 * d has a programmable per-channel profile: a start delay delta_dc (Sec. 3, t_A), a
 * tap count n_dc covering the intra-channel smear (Sec. 3, Delta tau_c) and per-tap
 * weights w_dck.
 *
 * Conventions
 *   - Frequencies in MHz, times in ms, DM in pc cm^-3.  k_dm = 1/kappa in ms GHz^2.
 *   - Channel c has low edge f_lo_mhz + c*df_mhz (descending = 0) or the mirror image
 *     (descending = 1).  nu_c is the channel's highest frequency (Sec. 3).
 *   - Arrays are row-major.  "d_" pointers are CUDA device pointers; all others are
 *     host pointers.  The caller owns every data buffer and stream; the plan owns its
 *     tables and workspace.  `stream` is a cudaStream_t (NULL = legacy default stream).
 *   - Device calls are asynchronous and stream-ordered.  Argument and plan errors are
 *     reported synchronously by the return value; CUDA launch errors as DD_ERR_CUDA.
 *   - A plan may be used from one stream at a time (its workspace is shared).
 *   - Input rows are `in_ld` elements apart; in_ld * element size must be a multiple of
 *     16 bytes and the input base pointer 16-byte aligned (rows are staged in 16-byte
 *     chunks).  Violations return DD_ERR_ARG.
 *   - Tracing and logging: every device call opens an NVTX range named after it (shown by
 *     timeline tools; a no-op without one), and the environment variable DD_LOG (read once)
 *     makes the library log to stderr: 1 = plan decisions (tap-sum method, CTA shape, stage
 *     size, row lengths, shared memory), autotuner results, batch bindings; 2 = also every
 *     device call with its sizes.
 *   - No call here allocates device memory except dd_plan_create / dd_set_profiles /
 *     the first device call on a plan (tables; on a device's first plan also the 8 MiB
 *     array of dd_boxcar_snr_noalloc), dd_boxcar_snr when the width count
 *     grows (normaliser workspace), dd_dedisperse on a run-length plan when nsamp
 *     grows (prefix scratch), dd_dedisperse_boxcar when its scratch grows, and the
 *     first dd_backward (adjoint workspace).
 */
#ifndef DD_H
#define DD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dd_plan_s* dd_plan_t;

typedef enum {
    DD_OK = 0,
    DD_ERR_ARG = 1,         /* bad argument (null pointer, size, alignment, range)      */
    DD_ERR_OVERFLOW = 2,    /* a size or sum would overflow the integer type used       */
    DD_ERR_OOM = 3,         /* host or device allocation failed                         */
    DD_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed              */
    DD_ERR_STATE = 5,       /* call not valid in the plan's current state               */
    DD_ERR_TIMEOUT = 6,     /* a bounded device wait gave up                            */
    DD_ERR_CAPACITY = 7,    /* more results than the caller's buffer holds (truncated)  */
    DD_ERR_UNSUPPORTED = 8  /* valid request outside what the kernels implement         */
} dd_status;

typedef enum { DD_U8 = 0, DD_F32 = 1 } dd_dtype;

/* Band and sampling of the filterbank (Sec. 2.1, Sec. 3). */
typedef struct {
    int32_t nchan;       /* C > 0                                                  */
    double f_lo_mhz;     /* lower edge of the band, > 0                            */
    double df_mhz;       /* channel width Delta nu, > 0                            */
    int32_t descending;  /* 0: channel 0 is the lowest frequency                   */
    double dt_ms;        /* sampling time Delta t, > 0                             */
    int64_t nsamp;       /* default samples per dedispersion call                  */
    int32_t in_type;     /* dd_dtype of I                                          */
    double k_dm;         /* 1/kappa in ms GHz^2; <= 0 selects 4.15                 */
} dd_band;

/* One detection: trial d, width index, first sample t of the boxcar, and S/N. */
typedef struct {
    int32_t dm_index;
    int32_t width_index;
    int32_t t;
    float snr;
} dd_candidate;

/* Trial DM list of eq. trial DMs (Sec. 6.3):
 *   DM_n = DM_0 + (2 eps / C) sum_{i<n} sqrt(DM_i^2 + DM_diag^2 + DM_tau^2),
 * with DM_diag and DM_tau of Sec. 6.2 (tau_av_ms = average scattered pulse width
 * tau'_av) and eps found by bisection so that DM_{n-1} = dm_max.  smear_terms = 2
 * keeps both smear terms as printed; 1 keeps DM_diag only.  Host only; writes n
 * doubles to dms_out and the DM error factor to *eps_out (may be NULL).
 * Errors: DD_ERR_ARG for n < 2, dm_max <= dm0, bad band or null output. */
dd_status dd_trial_dms(const dd_band* band, double dm0, double dm_max, int32_t n,
                       double tau_av_ms, int32_t smear_terms, double* dms_out,
                       double* eps_out);

/* Creates a plan for `ndm` trial DMs (host array, copied).  Builds the default
 * profile tables on the host (no device work):
 *   delta_dc = floor(k_dm * DM_d * (nu_c^-2 - nu_top^-2) / dt)        (Sec. 3, t_A)
 *   n_dc     = max(1, ceil(k_dm * DM_d * ((nu_c - dnu)^-2 - nu_c^-2) / dt))
 * with unit weights.  Errors: DD_ERR_ARG (null, ndm < 1, bad band, DM < 0),
 * DD_ERR_OOM. */
dd_status dd_plan_create(dd_plan_t* plan, const dd_band* band, const double* dms,
                         int32_t ndm);

/* Replaces the profiles (host arrays, copied).  delay [ndm][nchan] (NULL keeps the
 * formula), ntaps [ndm][nchan] (NULL keeps the formula), w [ndm][nchan][kmax] fp32
 * (NULL = unit weights; taps beyond n_dc are ignored).  Requires delay >= 0,
 * 1 <= n_dc, and n_dc <= kmax when w is given.  Unit-weight uint8 plans produce
 * int32 sums; all other plans produce fp32 sums.  Errors: DD_ERR_ARG,
 * DD_ERR_OVERFLOW (int32 sums could overflow), DD_ERR_UNSUPPORTED (profile too wide
 * for the kernels' shared-memory staging). */
dd_status dd_set_profiles(dd_plan_t plan, const int32_t* delay, const int32_t* ntaps,
                          const float* w, int32_t kmax);

/* Replaces the per-tap weights from device memory (stream-ordered copy; no host
 * round trip).  d_w is [ndm][nchan][kmax] fp32; the delay and tap tables are kept and
 * every n_dc must be <= kmax.  A unit-weight plan becomes a weighted one (fp32 sums).
 * Meant for training loops (the autograd binding calls it before each forward and
 * backward).  Errors: DD_ERR_ARG, DD_ERR_OOM, DD_ERR_CUDA. */
dd_status dd_set_weights_device(dd_plan_t plan, const float* d_w, int32_t kmax, void* stream);

/* Plan facts: t_out = nsamp - d_max for the default nsamp, d_max = max(delta + n - 1),
 * kmax = max n_dc, ns_total = sum_{d,c} n_dc, out_is_int = 1 when sums are int32.
 * Any output pointer may be NULL. */
dd_status dd_plan_info(dd_plan_t plan, int64_t* t_out, int32_t* d_max, int32_t* kmax,
                       int64_t* ns_total, int32_t* out_is_int);

/* Copies the plan's delay and tap tables ([ndm][nchan] int32, host) out. */
dd_status dd_get_tables(dd_plan_t plan, int32_t* delay, int32_t* ntaps);

/* eq. p_dedisp.  d_in: [nchan][in_ld] uint8 or fp32 (band.in_type); d_out: [ndm][out_ld]
 * int32 or fp32 (see dd_set_profiles).  Computes out[d][t] for 0 <= t < nsamp - d_max,
 * reading columns t_offset .. t_offset + nsamp - 1 of every row (nsamp <= 0 uses the
 * band's).  Chunked calls with t_offset advancing by L reproduce the one-shot result.
 * Errors: DD_ERR_ARG (null, alignment, t_offset + nsamp > in_ld, out_ld too small,
 * nsamp <= d_max), DD_ERR_UNSUPPORTED (run-length plan and nsamp > 2^24), DD_ERR_OOM,
 * DD_ERR_CUDA. */
dd_status dd_dedisperse(dd_plan_t plan, const void* d_in, int64_t in_ld, int64_t t_offset,
                        int64_t nsamp, void* d_out, int64_t out_ld, void* stream);

/* Per-channel noise statistics of the input over columns t_offset .. t_offset+nsamp-1:
 * mean and population standard deviation (fp64, device arrays of nchan), the cell
 * noise sigma_n of Sec. 2.1 as measured.  Errors: DD_ERR_ARG, DD_ERR_CUDA. */
dd_status dd_channel_stats(dd_plan_t plan, const void* d_in, int64_t in_ld,
                           int64_t t_offset, int64_t nsamp, double* d_mean, double* d_std,
                           void* stream);

/* Boxcar S/N of every trial and width (eq. snr; Sec. 5 boxcar detector).
 * d_series: the dedisperse output ([ndm][ld], int32 or fp32 as the plan produces),
 * t_len valid samples per row.  widths: host array of nw strictly increasing widths,
 * 1 <= w <= t_len.  For each (d, w):
 *   B_w[t] = sum_{j<w} x[d][t+j],  0 <= t <= t_len - w,
 *   snr    = (B_w - mu_dw) / sigma_dw,
 * where mu_dw and sigma_dw are the mean and deviation of B_w on noise with the given
 * per-channel mean and std (device fp64 [nchan]):
 *   mu_dw = sum_c mu_c sum_m v_dcm,  sigma_dw^2 = sum_c sigma_c^2 sum_m v_dcm^2,
 *   v_dc = w_dc (*) 1_w   (eq. P_N_dedisp generalised to weighted boxcar sums).
 * Writes d_peak_snr [ndm][nw] (fp32) and d_peak_t [ndm][nw] (earliest t of the
 * maximum).  If d_cands != NULL, every (d, w) whose peak exceeds thresh is appended
 * to d_cands (capacity cap, order unspecified) and *d_ncands counts them all (it must
 * be zeroed by the caller); overflow is visible as *d_ncands > cap.  Integer series
 * are summed exactly (int32 or int64 around a per-trial integer offset).
 * Errors: DD_ERR_ARG, DD_ERR_OOM, DD_ERR_CUDA. */
dd_status dd_boxcar_snr(dd_plan_t plan, const void* d_series, int64_t ld, int64_t t_len,
                        const int32_t* widths, int32_t nw, const double* d_chan_mean,
                        const double* d_chan_std, float* d_peak_snr, int32_t* d_peak_t,
                        float thresh, dd_candidate* d_cands, int32_t cap,
                        int32_t* d_ncands, void* stream);

/* dd_boxcar_snr for callers that may not allocate device memory while running -- a
 * real-time pipeline that fixes its device-memory footprint at start-up, or a host
 * that gives the library a fixed device budget.  The paper has no counterpart; this is
 * a deployment variant.  Same arguments, results and errors as dd_boxcar_snr, but the
 * normaliser tables live in an 8 MiB array in device global memory that is part of the
 * library image, so the call allocates nothing.  Limits and rules:
 *   - ndm * 8 + 2 * ndm * nw * 4 + nw * 4 bytes (each part rounded up to 256) must fit
 *     in 8 MiB (about ndm * nw <= 1,000,000); larger requests return DD_ERR_CAPACITY.
 *   - The plan's tables must already be on the current device (any earlier device call
 *     on the plan, e.g. dd_dedisperse, puts them there); otherwise DD_ERR_STATE, since
 *     uploading them would allocate.  Putting a plan's tables on a device for the first
 *     time also loads the 8 MiB array and the boxcar kernels there (CUDA would otherwise
 *     load them lazily, at this call) and looks up the array's device address; that
 *     device then holds the array until the process exits.
 *   - Every call shares the one array, and it keeps the last call's contents: calls on
 *     one stream are ordered, but calls that overlap on the GPU (different streams or
 *     host threads) race.  Nothing in it needs clearing: each call writes every value
 *     it reads.
 *   - The widths are sent with a stream-ordered copy from the caller's host array.  From
 *     pageable memory the copy has read them when the call returns; from pinned memory
 *     the array must stay unchanged until the stream reaches the call. */
dd_status dd_boxcar_snr_noalloc(dd_plan_t plan, const void* d_series, int64_t ld, int64_t t_len,
                                const int32_t* widths, int32_t nw, const double* d_chan_mean,
                                const double* d_chan_std, float* d_peak_snr, int32_t* d_peak_t,
                                float thresh, dd_candidate* d_cands, int32_t cap,
                                int32_t* d_ncands, void* stream);

/* eq. p_dedisp fused with the boxcar S/N of dd_boxcar_snr (eq. snr; Sec. 5): the same
 * results as dd_dedisperse(plan, d_in, in_ld, t_offset, nsamp, x, ...) followed by
 * dd_boxcar_snr(plan, x, ..., nsamp - d_max, widths, ...), bit for bit, but the
 * dedispersed series x is never written to device memory: the dedispersion CTAs scan
 * their finished tiles in shared memory (C outputs per tile and trial are carried to
 * the CTA's next tile, and 2C per part boundary go to a seam pass, through plan-owned
 * scratch).  For a caller that only needs the detections.
 * Every plan kind is taken:
 *   - integer plans (uint8 input, unit weights; both tap-sum methods): C = wmax - 1.
 *     Every boxcar sum of x - o_d (o_d the normaliser's per-trial integer offset) must
 *     fit int32: the kernel checks wmax * |x - o_d| < 2^31 per output and otherwise
 *     records DD_ERR_OVERFLOW in the plan's device status word (dd_get_device_status),
 *     the results of that call being undefined; dd_boxcar_snr on the stored series
 *     handles that case with 64-bit sums.
 *   - fp32 plans (fp32 input, or weighted uint8): the fp32 sums of dd_boxcar_snr, whose
 *     prefix chains start every 31 outputs, formed the same way; C = wmax + 29.
 * Limits (DD_ERR_UNSUPPORTED otherwise): contiguous widths (w_j = w_0 + j), C <= the
 * schedule's tile (992 * nch outputs on the integer paths, 864 * nch on fp32 plans), and
 * nsamp <= 2^24 on the run-length path.
 * Other arguments, outputs and errors as dd_dedisperse and dd_boxcar_snr.  Allocates
 * plan-owned device scratch when the sizes grow: the merged maxima (8 bytes per trial
 * and width) and, per part, its carried outputs and seams (12 C bytes per trial of a
 * CTA's block).  A call with a new width list or a new launch geometry copies small
 * host tables to the device synchronously, so make one such call before capturing the
 * stream in a CUDA graph.  Calls on one plan share its scratch: order them on one
 * stream. */
dd_status dd_dedisperse_boxcar(dd_plan_t plan, const void* d_in, int64_t in_ld, int64_t t_offset,
                               int64_t nsamp, const int32_t* widths, int32_t nw,
                               const double* d_chan_mean, const double* d_chan_std,
                               float* d_peak_snr, int32_t* d_peak_t, float thresh,
                               dd_candidate* d_cands, int32_t cap, int32_t* d_ncands, void* stream);

/* Test hook: the number of parts (CTAs, each a contiguous run of the launch's (trial
 * block, time tile) items) of the next dd_dedisperse_boxcar calls, capped at the number
 * of items; 0 restores the automatic choice (one to eight per CTA resident on the device,
 * parts of at least ~16 tiles).
 * Errors: DD_ERR_ARG. */
dd_status dd_test_set_fused_parts(dd_plan_t plan, int32_t nparts);

/* Adjoint of the weighted map of eq. p_dedisp (no counterpart in the paper): given
 * g = d(loss)/d(out) (d_gout [ndm][gout_ld] fp32, nsamp - d_max valid columns),
 *   d_gw [ndm][nchan][kmax] : gw_dck   = sum_t g[d][t] I[c][t_offset + t + delta + k]
 *                             (zero for k >= n_dc), NULL to skip;
 *   d_gin [nchan][gin_ld]   : gI[c][tau] += sum_{d,k} w_dck g[d][tau - t_offset - delta - k]
 *                             for every column, NULL to skip.  Columns outside
 *                             t_offset .. t_offset + nsamp - 1 are left unchanged; the
 *                             columns inside are overwritten.
 * fp32 plans only (fp32 input).  Errors: DD_ERR_ARG, DD_ERR_UNSUPPORTED, DD_ERR_CUDA. */
dd_status dd_backward(dd_plan_t plan, const float* d_in, int64_t in_ld, int64_t t_offset,
                      int64_t nsamp, const float* d_gout, int64_t gout_ld, float* d_gw,
                      float* d_gin, int64_t gin_ld, void* stream);

/* Kernel schedule of the plan: nch time chunks per CTA (the CTA sums 16/nch trials on
 * the fp32 path, 8/nch on the exact integer path, 24/nch on the run-length path) and cs
 * channels per pipeline stage.
 * dd_plan_create and dd_set_profiles pick a default; dd_plan_set_schedule overrides it
 * (DD_ERR_UNSUPPORTED if it does not fit in shared memory, the old one is then kept). */
dd_status dd_plan_set_schedule(dd_plan_t plan, int32_t nch, int32_t cs);
dd_status dd_plan_get_schedule(dd_plan_t plan, int32_t* nch, int32_t* cs, int32_t* trials_per_cta);

/* How a plan forms the tap sums of eq. p_dedisp.
 *   DD_METHOD_DIRECT:    every tap is one multiply-add (any weights).
 *   DD_METHOD_RUNLENGTH: uint8 unit-weight plans only.  A run of n unit taps is a
 *     difference of per-channel prefix sums, sum_{k<n} I[c][s+k] = P_c[s+n] - P_c[s]
 *     with P_c[i] = sum_{j<i} I[c][t_offset+j], so each (trial, channel) costs two
 *     loads and one add per output whatever its tap count.  dd_dedisperse first writes
 *     P for the requested samples into plan-owned device scratch (4 bytes per channel
 *     and sample, uint32; exact since the differences are taken modulo 2^32), then sums.
 *     Results are bit-identical to DD_METHOD_DIRECT.  nsamp is limited to 2^24.
 *   DD_METHOD_AUTO (default): RUNLENGTH for uint8 unit-weight plans whose mean tap count
 *     is at least 12, DIRECT otherwise.
 * dd_plan_set_method rebuilds the schedule (DD_ERR_UNSUPPORTED: RUNLENGTH on a weighted
 * or fp32 plan; the method is then unchanged).  A run-length plan that later gets weights
 * sums directly.  dd_plan_get_method reports the method in use (never AUTO).  A batch
 * (below) takes plans of one method. */
typedef enum {
    DD_METHOD_AUTO = 0,
    DD_METHOD_DIRECT = 1,
    DD_METHOD_RUNLENGTH = 2
} dd_method;
dd_status dd_plan_set_method(dd_plan_t plan, int32_t method);
dd_status dd_plan_get_method(dd_plan_t plan, int32_t* method);

/* Autotuner: times the plan's dedispersion on the given buffers (as dd_dedisperse with
 * t_offset 0 and the band's nsamp) for each CTA shape (nch 1, 2) and stage size (fp32 and
 * run-length: 2, 3, 4, 6, 8 channels; uint8: 4, 8, 12, 16) that fits, keeps the fastest,
 * and appends
 * it to the text cache at cache_path (may be NULL) under a key of channel count, input
 * type, path, and the powers of two of the trial-block delay spread and the widest tap
 * run.  A cached key is applied without timing (*best_ms = -1).  Synchronises the
 * stream; overwrites d_out.  Errors: DD_ERR_ARG, DD_ERR_CUDA. */
dd_status dd_plan_autotune(dd_plan_t plan, const void* d_in, int64_t in_ld, void* d_out,
                           int64_t out_ld, const char* cache_path, float* best_ms, void* stream);

/* Many beams in one launch (uneven lengths and trial lists; no counterpart in
 * the paper, which describes one beam).  Each beam has its own plan (the same input type
 * and tap-sum path for all: DD_ERR_ARG for mixed input types, DD_ERR_UNSUPPORTED for mixed
 * methods, or run-length beams longer than 2^24 samples; the plans must outlive the
 * batch); a beam's block is the band's nsamp samples from column 0.  The work list has
 * one item per CTA tile (beam, trial block, time tile), and the launch one CTA per item in
 * list order: beams by decreasing estimated cost, each beam's tiles in the order of its
 * own launch (dd_dedisperse).
 * Run-length beams first get their per-channel prefix sums (one small launch per beam,
 * into device memory the batch owns: 4 bytes per channel and sample, allocated by
 * dd_batch_bind), then the batched launch sums them. */
typedef struct dd_batch_s* dd_batch_t;
dd_status dd_batch_create(dd_batch_t* batch, const dd_plan_t* plans, int32_t nbeams);
/* Binds each beam's device input [nchan][in_ld] and output [ndm][out_ld] (host arrays of
 * nbeams pointers / leading dimensions), uploads the plans' tables and the work list
 * (allocates; synchronous).  Rebinding invalidates a captured graph. */
dd_status dd_batch_bind(dd_batch_t batch, const void* const* d_in, const int64_t* in_ld,
                        void* const* d_out, const int64_t* out_ld);
/* The batched dedispersion launch for all bound beams (on run-length beams the prefix
 * passes before it). */
dd_status dd_batch_dedisperse(dd_batch_t batch, void* stream);
/* Binds, per beam, the outputs of the detection stage (boxcar widths shared by all beams;
 * device channel mean/std [nchan], peak S/N and peak time [ndm][nw]). */
dd_status dd_batch_bind_boxcar(dd_batch_t batch, const int32_t* widths, int32_t nw,
                               double* const* d_mean, double* const* d_std, float* const* d_peak,
                               int32_t* const* d_arg);
/* One block of every beam: dd_batch_dedisperse, then (if bound) each beam's channel
 * statistics and boxcar S/N. */
dd_status dd_batch_run(dd_batch_t batch, void* stream);
/* Runs dd_batch_run once eagerly (creating all workspace), then captures it on `stream`
 * (a non-default stream) into a CUDA graph owned by the batch; dd_batch_replay launches
 * the graph. */
dd_status dd_batch_capture(dd_batch_t batch, void* stream);
dd_status dd_batch_replay(dd_batch_t batch, void* stream);
/* Work items, CTAs per launch (one per item), and total trial x output samples of one
 * block. */
dd_status dd_batch_info(dd_batch_t batch, int32_t* nitems, int32_t* grid, int64_t* units);
dd_status dd_batch_destroy(dd_batch_t batch);

/* Device-side errors: synchronises `stream`, then returns in *code the first error a
 * kernel of this plan recorded since the last call (0 = none; DD_ERR_TIMEOUT when a
 * bounded wait on a bulk-copy barrier ran out) and clears it.  Errors: DD_ERR_ARG,
 * DD_ERR_CUDA. */
dd_status dd_get_device_status(dd_plan_t plan, int32_t* code, void* stream);

/* Test hook for the failure path of the dedispersion pipeline: the bulk copies of
 * channel stage `skip_stage` (-1: none) are never issued, and every barrier wait gives
 * up after wait_ns (0 restores the default of 2 s).  The kernel then records
 * DD_ERR_TIMEOUT, drains the copies it did issue and returns; no GPU fault is involved.
 * Errors: DD_ERR_ARG. */
dd_status dd_test_set_wait(dd_plan_t plan, int32_t skip_stage, int64_t wait_ns);

/* Profile construction (host only).
 *
 * dd_predict_rect: the cell-averaged power of eq. Pavg for the rectangular scattered pulse
 * of eq. profile_sb, P(t, nu) = p0 (nu/nu0)^-alpha tau/tau' on [t_d, t_d + tau'), with
 * t_d(nu) = t0_ms + k_dm DM (nu^-2 - nu_top^-2) (arrival t0_ms at the top of the band):
 *   pbar[c][j] = (1/dt) int_{channel c} dnu int_{j dt}^{(j+1) dt} dt' P(t', nu),
 * nu in GHz, for 0 <= j < nt (cells before t = 0 or from nt on are left out).  The time
 * integral is the exact overlap; the frequency integral is a midpoint rule on at least 64
 * sub-channels per channel, more where one sub-channel's own sweep would exceed tau'/16.
 * pbar is a host array [nchan][nt].  Errors: DD_ERR_ARG.
 *
 * dd_select_samples: the sample selection of Sec. 2.2 on one trial's predicted powers
 * pbar [nchan][nt]: samples are taken in order of decreasing power (equal powers in
 * channel-major order) while eq. sel_criterion holds, P > (sqrt((N+1)/N) - 1) * sum of
 * the N already taken.  Each channel's selected samples become a tap run from the first
 * to the last of them with weight 1 on selected samples and 0 on gaps (delay[c] = first
 * sample, ntaps[c] = run length, w [nchan][kmax]); a channel with none gets one tap of
 * weight 0.  *nsel = samples taken, *gain = (S/N of the selection)/(S/N of every sample
 * with P > 0), S/N = sum P / sqrt(N) (equal noise per sample, eq. snr).  Either output
 * may be NULL.  Errors: DD_ERR_ARG, DD_ERR_CAPACITY (a run longer than kmax).
 *
 * dd_exact_profiles: the tap rule of eq. num_samples with the pulse width,
 * delay = floor(t_A/dt) and ntaps = ceil(t_B/dt) - floor(t_A/dt), t_A = k_dm DM
 * (nu_c^-2 - nu_top^-2) and t_B = t_A + tau' + the exact sweep across the channel, for
 * every trial of the plan (host arrays [ndm][nchan]; pass them to dd_set_profiles).
 * Errors: DD_ERR_ARG, DD_ERR_OVERFLOW. */
dd_status dd_predict_rect(const dd_band* band, double dm, double t0_ms, double tau_ms,
                          double tau_prime_ms, double alpha, double nu0_ghz, double p0,
                          int32_t nt, double* pbar);
dd_status dd_select_samples(const double* pbar, int32_t nchan, int32_t nt, int32_t kmax,
                            int32_t* delay, int32_t* ntaps, float* w, int32_t* nsel, double* gain);
dd_status dd_exact_profiles(dd_plan_t plan, double tau_prime_ms, int32_t* delay, int32_t* ntaps);

/* dd_select_profiles: the Sec. 2.2 sample selection for every trial of the plan, on the
 * eq. Pavg cell powers of the rectangular scattered pulse of eq. profile_sb (dd_predict_rect
 * with p0 = 1, spectral index alpha about nu0_ghz, scattering tau_ms, width tau_prime_ms) at
 * the trial's own DM, arriving `phase` samples (>= 0) into output sample 0 at the top of the
 * band.  Each trial's cells run from there to the end of its sweep across the whole band,
 * plus tau' and two samples.  Writes delay and ntaps [ndm][nchan], the weights w
 * [ndm][nchan][kmax] (0/1, as dd_select_samples; may be NULL), each trial's S/N gain over
 * taking every sample with pulse power (gains [ndm], may be NULL) and the longest run in
 * *kused (may be NULL).  Call with w = NULL to learn kused, then with kmax >= kused.  Host
 * only.  Errors: DD_ERR_ARG, DD_ERR_CAPACITY (a run longer than kmax), DD_ERR_OVERFLOW. */
dd_status dd_select_profiles(dd_plan_t plan, double tau_ms, double tau_prime_ms, double alpha,
                             double nu0_ghz, double phase, int32_t kmax, int32_t* delay,
                             int32_t* ntaps, float* w, double* gains, int32_t* kused);

/* The comparison detectors of Sec. 5 as profiles for the same dedispersion kernel, from one
 * trial's predicted powers pbar [nchan][nt] (host):
 *   kind 0, dynamic-spectrum matched filter: every cell with power, weighted by its power
 *     (scaled to a maximum of 1); *snr = sqrt(sum pbar^2).
 *   kind 1, time-series matched filter: the channels aligned by align[c] (the trial's integer
 *     delays) and summed into T[m] = sum_c pbar[c][align[c] + m]; every channel gets the tap
 *     run of T's window with weights T (scaled to a maximum of 1); *snr = sqrt(sum T^2 / C).
 *   kind 2, time-series boxcar matched in width: the same window with unit weights;
 *     *snr = sum T / sqrt(C * window length).
 * S/N assumes unit noise per cell (divide by the cell noise for physical units).  Outputs as
 * dd_select_samples (delay/ntaps [nchan], w [nchan][kmax]); snr may be NULL.
 * Errors: DD_ERR_ARG (no power, align NULL for kinds 1-2, a window before sample 0),
 * DD_ERR_CAPACITY (a run longer than kmax). */
dd_status dd_detector_profile(const double* pbar, int32_t nchan, int32_t nt, const int32_t* align,
                              int32_t kind, int32_t kmax, int32_t* delay, int32_t* ntaps, float* w,
                              double* snr);

/* Measured ALU throughput of the current device (no counterpart in the paper; the
 * denominator of the roofline fraction of the ALU-bound kernels).  kind 0: FP32 fused
 * multiply-adds, reported as flops/s (2 per FMA); kind 1: INT32 three-input adds,
 * reported as additions/s (2 per instruction); kind 2: packed FP32 pairs (fma.rn.f32x2,
 * the instruction of the fp32 dedispersion kernels), flops/s (4 per instruction).  Dependency-free loops over every SM;
 * one warm-up launch, one timed launch (about 0.1 s); synchronises the stream.
 * Errors: DD_ERR_ARG, DD_ERR_OOM, DD_ERR_CUDA. */
dd_status dd_alu_peak(int32_t kind, double* ops_per_s, void* stream);

/* Releases the plan's host and device memory (after its work has finished). */
dd_status dd_plan_destroy(dd_plan_t plan);

/* Static, human-readable name of a status code. */
const char* dd_status_str(dd_status s);

/* Library version, as major*10000 + minor*100 + patch. */
int32_t dd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DD_H */
