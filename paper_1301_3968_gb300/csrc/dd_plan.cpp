// Host side of the C ABI: band geometry, the default profile tables (Sec. 3), the
// trial-DM rule (eq. trial DMs, Sec. 6.3), argument checking and the dedispersion
// schedule (trial blocks and staged window lengths).
#include <algorithm>
#include <cstdlib>
#include <cstdio>
#include <cstdarg>
#include <cmath>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <new>
#include <sstream>
#include <string>

#include "dd_internal.h"
#include "dd_trace.h"

namespace {

constexpr double kDefaultKdm = 4.15;

double kdm_of(const dd_band& b) { return b.k_dm > 0 ? b.k_dm : kDefaultKdm; }

bool band_ok(const dd_band* b) {
    return b && b->nchan > 0 && b->f_lo_mhz > 0 && b->df_mhz > 0 && b->dt_ms > 0 &&
           b->nsamp >= 0 && (b->in_type == DD_U8 || b->in_type == DD_F32) &&
           b->f_lo_mhz > 0;
}

// nu_c: highest frequency of channel c in GHz (Sec. 3).
double chan_top_ghz(const dd_band& b, int c) {
    int j = b.descending ? (b.nchan - 1 - c) : c;
    return (b.f_lo_mhz + (j + 1) * b.df_mhz) / 1000.0;
}

double band_top_ghz(const dd_band& b) { return (b.f_lo_mhz + b.nchan * b.df_mhz) / 1000.0; }

// Sec. 6.2: [(1/C) sum_c nu_c^-3]^-1 (channel order does not matter).
double inv_mean_inv_cube(const dd_band& b) {
    double s = 0.0;
    for (int c = 0; c < b.nchan; ++c) {
        double nu = (b.f_lo_mhz + (c + 1) * b.df_mhz) / 1000.0;
        s += 1.0 / (nu * nu * nu);
    }
    return 1.0 / (s / b.nchan);
}

void build_trials(const dd_band& b, double dm0, double eps, int n, double extra2, double* out) {
    out[0] = dm0;
    double acc = 0.0;
    for (int i = 1; i < n; ++i) {
        acc += std::sqrt(out[i - 1] * out[i - 1] + extra2);
        out[i] = dm0 + 2.0 * eps / b.nchan * acc;
    }
}

// Span of the staged window when `db` consecutive trials share a CTA: the largest
// max(delta + n) - min(delta) over blocks and channels.
int64_t block_span(const dd_plan_s* p, int db, std::vector<int32_t>* lo_out) {
    const int C = p->nchan;
    const int nblk = (p->ndm + db - 1) / db;
    if (lo_out) lo_out->assign((size_t)nblk * C, 0);
    int64_t span = 0;
    for (int b = 0; b < nblk; ++b) {
        for (int c = 0; c < C; ++c) {
            int64_t lo = INT64_MAX, hi = 0;
            for (int i = 0; i < db; ++i) {
                const int d = b * db + i;
                if (d >= p->ndm) break;
                const int64_t dl = p->delay[(size_t)d * C + c];
                lo = std::min(lo, dl);
                hi = std::max(hi, dl + p->taps[(size_t)d * C + c]);
            }
            if (lo_out) (*lo_out)[(size_t)b * C + c] = (int32_t)lo;
            span = std::max(span, hi - lo);
        }
    }
    return span;
}

// Trials per warp unit: two adjacent trials share one register window on the fp32
// path; the exact integer path sums one trial per unit.
int trials_per_unit(const dd_plan_s* p) { return p->pair ? 2 : 1; }

// Warp units per warp: a run-length warp keeps kRlUnits trials' sums (it needs no
// register window, so more trials share each staged prefix row).
int units_per_warp(const dd_plan_s* p) { return p->rl ? dd::kRlUnits : 1; }

// Buffers in the staging ring of the plan's path.
int stages_of(const dd_plan_s* p) {
    return p->rl ? dd::kStagesRl : (p->pair ? dd::kStagesPair : dd::kStagesInt);
}

// Staged element size and elements per 16-byte chunk: uint8 samples, fp32 samples, or
// uint32 prefix sums on the run-length path.
int stage_esz(const dd_plan_s* p) { return p->rl ? 4 : (p->band.in_type == DD_U8 ? 1 : 4); }

// Elements a CTA stages per channel: its outputs, the block's delay spread plus taps
// (plus the run's end point P[delta + n] on the run-length path), 16 bytes of
// alignment slack and the element that the register pipeline reads ahead.
int64_t staged_len(const dd_plan_s* p, int nch, int64_t span) {
    const int64_t q = 16 / stage_esz(p);
    int64_t need = (int64_t)nch * dd::chunk_t(p->pair) + span + (p->rl ? 1 : 0) + q + 2;
    return (need + q - 1) / q * q;
}

// Weight pairs per record entry on the pair path: the most taps of any warp unit on
// any channel, max(n0, n1) (each trial's tap k reads sample k of its own run).
int32_t pair_taps(const dd_plan_s* p) {
    const int C = p->nchan, tpw = trials_per_unit(p);
    int64_t u = 0;
    for (int d0 = 0; d0 < p->ndm; d0 += tpw)
        for (int c = 0; c < C; ++c)
            for (int i = 0; i < tpw && d0 + i < p->ndm; ++i)
                u = std::max<int64_t>(u, p->taps[(size_t)(d0 + i) * C + c]);
    return (int32_t)std::min<int64_t>(u, INT32_MAX);
}

// Weight pairs of the fullest stage record on the pair path for stages of cs channels:
// each entry holds max(n0, n1) pairs.
int32_t pair_record_pairs(const dd_plan_s* p, int db, int cs) {
    const int C = p->nchan;
    const int nblk = (p->ndm + db - 1) / db;
    int64_t most = 0;
    for (int b = 0; b < nblk; ++b)
        for (int c0 = 0; c0 < C; c0 += cs) {
            int64_t tot = 0;
            for (int d0 = b * db; d0 < std::min(p->ndm, (b + 1) * db); d0 += 2)
                for (int c = c0; c < std::min(C, c0 + cs); ++c) {
                    const size_t a = (size_t)d0 * C + c;
                    int64_t n = p->taps[a];
                    if (d0 + 1 < p->ndm) n = std::max<int64_t>(n, p->taps[a + C]);
                    tot += n;
                }
            most = std::max(most, tot);
        }
    return (int32_t)std::min<int64_t>((most + 1) & ~(int64_t)1, INT32_MAX);
}

// Samples past the block minimum that a pair unit's register window reaches: each
// trial reads max(n0, n1) samples from its own start, so the shorter run's trial reads
// past its own window by |n0 - n1| (with zero weights).  The staged window must hold
// them.
int64_t pair_read_span(const dd_plan_s* p, int db) {
    const int C = p->nchan;
    const int nblk = (p->ndm + db - 1) / db;
    int64_t span = 0;
    for (int b = 0; b < nblk; ++b)
        for (int c = 0; c < C; ++c) {
            int64_t lo = INT64_MAX;
            for (int d = b * db; d < std::min(p->ndm, (b + 1) * db); ++d)
                lo = std::min<int64_t>(lo, p->delay[(size_t)d * C + c]);
            for (int d0 = b * db; d0 < std::min(p->ndm, (b + 1) * db); d0 += 2) {
                const size_t a = (size_t)d0 * C + c;
                int64_t st = p->delay[a], n = p->taps[a];
                if (d0 + 1 < p->ndm) {
                    const size_t bb = (size_t)(d0 + 1) * C + c;
                    st = std::max<int64_t>(st, p->delay[bb]);
                    n = std::max<int64_t>(n, p->taps[bb]);
                }
                span = std::max(span, st + n - lo);
            }
        }
    return span;
}

// Most distinct tap counts among one trial block's trials on any channel (run-length
// path): the CTA builds one difference row per distinct count, so at most two fit.
int max_distinct_taps(const dd_plan_s* p, int db) {
    const int C = p->nchan;
    int most = 0;
    for (int d0 = 0; d0 < p->ndm; d0 += db)
        for (int c = 0; c < C; ++c) {
            int a = -1, b = -1, n = 0;
            for (int d = d0; d < std::min(p->ndm, d0 + db); ++d) {
                const int t = p->taps[(size_t)d * C + c];
                if (t == a || t == b) continue;
                if (a < 0) a = t;
                else if (b < 0) b = t;
                ++n;
                if (n > 2) return n;
            }
            most = std::max(most, n);
        }
    return most;
}

// Length of one difference row (run-length path with shared rows) for tap count n on
// channel c of block b: its words are read up to the largest run start of the block's
// trials with that count (relative to the block minimum), plus the CTA's outputs, plus
// three words of 16-byte alignment slack.
int32_t brow_row_len(const dd_plan_s* p, int db, int nch, const std::vector<int32_t>& blk_lo, int b,
                     int c, int n) {
    const int C = p->nchan;
    const int64_t lo = blk_lo[(size_t)b * C + c];
    int64_t x = 0;
    for (int d = b * db; d < std::min(p->ndm, (b + 1) * db); ++d)
        if (p->taps[(size_t)d * C + c] == n) x = std::max<int64_t>(x, p->delay[(size_t)d * C + c] - lo);
    return (int32_t)(x + (int64_t)nch * dd::chunk_t(false) + 4);
}

// The stride of the difference rows: the longest row of any block and channel.
int32_t brow_stride(const dd_plan_s* p, int db, int nch) {
    const int C = p->nchan;
    const int nblk = (p->ndm + db - 1) / db;
    std::vector<int32_t> lo;
    block_span(p, db, &lo);
    int32_t len = 0;
    for (int b = 0; b < nblk; ++b)
        for (int c = 0; c < C; ++c) {
            int n0 = 0, n1 = 0;
            for (int d = b * db; d < std::min(p->ndm, (b + 1) * db); ++d) {
                const int t = p->taps[(size_t)d * C + c];
                if (n0 == 0) n0 = t;
                else if (t != n0 && n1 == 0) n1 = t;
            }
            len = std::max(len, brow_row_len(p, db, nch, lo, b, c, n0));
            if (n1) len = std::max(len, brow_row_len(p, db, nch, lo, b, c, n1));
        }
    return (len + 3) & ~3;
}

// Lays the profile tables out as the kernel stages them: one record per (trial block,
// channel stage).  Entry (unit j, channel ci) = (window start - block minimum, taps);
// on the pair path it is (trial 0's start - block minimum, max(n0, n1), trial 1's start
// - trial 0's, 0) and the weights are (w0, w1) pairs, zero past a trial's own taps.
void build_records(dd_plan_s* p) {
    const int C = p->nchan;
    const int tpw = trials_per_unit(p);
    const int nu = dd::kWarps / p->nch * units_per_warp(p);
    const int db = tpw * nu;
    const int nst = (C + p->cs - 1) / p->cs;
    const int kw = p->pair ? p->kw : 0;
    const dd::StageGeom g(stage_esz(p), p->pair, p->lcap, kw, p->cs, nu, p->rl_b, p->blen);
    p->rec_bytes = g.rec_bytes;
    p->rec.assign((size_t)p->nblk * nst * g.rec_bytes, 0);
    for (int b = 0; b < p->nblk; ++b)
        for (int st = 0; st < nst; ++st) {
            unsigned char* r = p->rec.data() + ((size_t)b * nst + st) * g.rec_bytes;
            int32_t* ent = (int32_t*)r;
            float* w = (float*)(r + g.w_off);
            // difference rows: (n0, n1, len0, len1) per channel
            int32_t* nlist = (int32_t*)(r + g.w_off);
            int32_t woff = 0;  // pair path: weight pairs used so far in this record
            if (p->rl_b)
                for (int ci = 0; ci < p->cs; ++ci) {
                    const int c = st * p->cs + ci;
                    if (c >= C) continue;
                    int a = 0, bb = 0;
                    for (int d = b * db; d < std::min(p->ndm, (b + 1) * db); ++d) {
                        const int t = p->taps[(size_t)d * C + c];
                        if (a == 0) a = t;
                        else if (t != a && bb == 0) bb = t;
                    }
                    nlist[4 * ci] = a;
                    nlist[4 * ci + 1] = bb;
                    nlist[4 * ci + 2] = a ? brow_row_len(p, db, p->nch, p->blk_lo, b, c, a) : 0;
                    nlist[4 * ci + 3] = bb ? brow_row_len(p, db, p->nch, p->blk_lo, b, c, bb) : 0;
                }
            for (int j = 0; j < nu; ++j)
                for (int ci = 0; ci < p->cs; ++ci) {
                    const int c = st * p->cs + ci;
                    const int d0 = b * db + j * tpw;
                    if (d0 >= p->ndm || c >= C) continue;
                    if (p->pair) {
                        // (trial 0's start, max(n0, n1), trial 1's start - trial 0's, offset of
                        // the entry's weights) and per tap k the pair (w0[k], w1[k]), zero past
                        // a trial's own taps; entries' weights follow one another
                        const int e = j * p->cs + ci;
                        const int64_t blo = p->blk_lo[(size_t)b * C + c];
                        const size_t a0 = (size_t)d0 * C + c;
                        const bool two = d0 + 1 < p->ndm;
                        const size_t a1 = two ? a0 + C : a0;
                        const int n = std::max(p->taps[a0], two ? p->taps[a1] : 0);
                        ent[4 * e] = (int32_t)(p->delay[a0] - blo);
                        ent[4 * e + 1] = n;
                        ent[4 * e + 2] = two ? p->delay[a1] - p->delay[a0] : 0;
                        ent[4 * e + 3] = woff;
                        for (int i = 0; i < 2; ++i) {
                            if (i == 1 && !two) break;
                            const size_t dc = i ? a1 : a0;
                            for (int k = 0; k < p->taps[dc]; ++k)
                                w[((size_t)woff + k) * 2 + i] = p->unit ? 1.0f : p->w[dc * p->kpad + k];
                        }
                        woff += n;
                        continue;
                    }
                    int64_t lo = INT64_MAX, hi = 0;
                    for (int i = 0; i < tpw && d0 + i < p->ndm; ++i) {
                        const size_t dc = (size_t)(d0 + i) * C + c;
                        lo = std::min<int64_t>(lo, p->delay[dc]);
                        hi = std::max<int64_t>(hi, (int64_t)p->delay[dc] + p->taps[dc]);
                    }
                    const int e = j * p->cs + ci;
                    ent[2 * e] = (int32_t)(lo - p->blk_lo[(size_t)b * C + c]);
                    ent[2 * e + 1] = (int32_t)(hi - lo);
                    if (p->rl_b) ent[2 * e + 1] = (hi - lo) == nlist[4 * ci] ? 0 : 1;
                }
        }
}

// Chooses the CTA shape of the dedispersion kernel (warp units x time chunks), the
// staged window length and the channels per pipeline stage.  The most trials per CTA
// (the most reuse of each staged sample) whose window still fits is taken.
dd_status build_schedule(dd_plan_s* p) {
    const bool u8 = p->band.in_type == DD_U8;
    p->pair = !(u8 && p->unit);
    const double mean_taps = (double)p->ns_total / ((double)p->ndm * p->nchan);
    p->rl = u8 && p->unit &&
            (p->method == DD_METHOD_RUNLENGTH ||
             (p->method == DD_METHOD_AUTO && mean_taps >= dd::kRlMinMeanTaps));
    const int esz = stage_esz(p);
    const int cs_want = dd::kCsMax;
    const int nbuf = stages_of(p);
    const int tpw = trials_per_unit(p);
    // first pass: shared memory for two CTAs per SM and at least two channels per
    // stage; second pass: one CTA per SM, any stage size
    const int budgets[2] = {dd::kSmemBudget, dd::kSmemBudgetOne};
    const int min_cs[2] = {2, 1};
    for (int pass = 0; pass < 2; ++pass) {
        for (int nch = 1; nch <= dd::kWarps; nch *= 2) {
            const int nu = dd::kWarps / nch * units_per_warp(p);
            const int db = tpw * nu;
            int64_t span = block_span(p, db, nullptr);
            if (p->pair) span = std::max(span, pair_read_span(p, db));
            p->umax = p->pair ? pair_taps(p) : 0;
            p->rl_b = p->rl && max_distinct_taps(p, db) <= 2;
            const int64_t need = staged_len(p, nch, span);
            if (need > (1 << 22)) continue;
            p->blen = p->rl_b ? brow_stride(p, db, nch) : 0;
            int cs = cs_want;
            int32_t kw = p->pair ? pair_record_pairs(p, db, cs) : 0;
            while (cs >= min_cs[pass] &&
                   dd::dedisp_smem_bytes(dd::StageGeom(esz, p->pair, (int)need, kw, cs, nu, p->rl_b, p->blen),
                                         nbuf, p->nchan) > budgets[pass]) {
                --cs;
                if (p->pair && cs >= 1) kw = pair_record_pairs(p, db, cs);
            }
            if (cs < min_cs[pass]) continue;
            p->nch = nch;
            p->cs = cs;
            p->kw = kw;
            p->lcap = (int32_t)need;
            p->nblk = (p->ndm + db - 1) / db;
            block_span(p, db, &p->blk_lo);
            build_records(p);
            p->dev_dirty = true;
            dd::log_msg(1, "plan %d trials x %d channels: %s, %d trials per CTA, %d channels per stage, "
                        "staged rows of %d elements, difference rows of %d, record %d bytes, %zu bytes "
                        "of shared memory",
                     p->ndm, p->nchan,
                     p->rl ? (p->rl_b ? "run-length sums with shared difference rows" : "run-length sums")
                           : (p->pair ? "fp32 pair units" : "exact integer sums"),
                     db, p->cs, p->lcap, p->blen, p->rec_bytes, dd::dedisp_smem_for(p));
            return DD_OK;
        }
    }
    dd::log_msg(1, "plan %d trials x %d channels: no CTA shape fits in shared memory", p->ndm, p->nchan);
    return DD_ERR_UNSUPPORTED;
}

// Fixed CTA shape (nch time chunks) and stage size (cs channels), if it fits.
dd_status build_schedule_fixed(dd_plan_s* p, int nch, int cs) {
    if (nch < 1 || nch > dd::kWarps || (dd::kWarps % nch) != 0 || cs < 1 || cs > 32) return DD_ERR_ARG;
    const int esz = stage_esz(p);
    const int nu = dd::kWarps / nch * units_per_warp(p);
    const int db = trials_per_unit(p) * nu;
    int64_t span = block_span(p, db, nullptr);
    if (p->pair) span = std::max(span, pair_read_span(p, db));
    p->umax = p->pair ? pair_taps(p) : 0;
    const bool rl_b = p->rl && max_distinct_taps(p, db) <= 2;
    const int32_t kw = p->pair ? pair_record_pairs(p, db, cs) : 0;
    const int64_t need = staged_len(p, nch, span);
    if (need > (1 << 22)) return DD_ERR_UNSUPPORTED;
    const int32_t blen = rl_b ? brow_stride(p, db, nch) : 0;
    if (dd::dedisp_smem_bytes(dd::StageGeom(esz, p->pair, (int)need, kw, cs, nu, rl_b, blen), stages_of(p),
                              p->nchan) > dd::kSmemBudgetOne)
        return DD_ERR_UNSUPPORTED;
    p->blen = blen;
    p->rl_b = rl_b;
    p->nch = nch;
    p->cs = cs;
    p->kw = kw;
    p->lcap = (int32_t)need;
    p->nblk = (p->ndm + db - 1) / db;
    block_span(p, db, &p->blk_lo);
    build_records(p);
    p->dev_dirty = true;
    return DD_OK;
}

dd_status finish_profiles(dd_plan_s* p) {
    const size_t n = (size_t)p->ndm * p->nchan;
    int32_t kmax = 1, dmax = 0;
    int64_t ns = 0, row_max = 0;
    for (int d = 0; d < p->ndm; ++d) {
        int64_t row = 0;
        for (int c = 0; c < p->nchan; ++c) {
            size_t i = (size_t)d * p->nchan + c;
            kmax = std::max(kmax, p->taps[i]);
            int64_t e = (int64_t)p->delay[i] + p->taps[i] - 1;
            if (e > INT32_MAX) return DD_ERR_OVERFLOW;
            dmax = std::max<int32_t>(dmax, (int32_t)e);
            ns += p->taps[i];
            row += p->taps[i];
        }
        row_max = std::max(row_max, row);
    }
    (void)n;
    p->kmax = kmax;
    p->dmax = dmax;
    p->ns_total = ns;
    p->out_int = p->unit && p->band.in_type == DD_U8;
    p->max_abs_row = row_max * 255;
    if (p->out_int && p->max_abs_row > INT32_MAX) return DD_ERR_OVERFLOW;
    p->adj_stale = true;
    p->adj_w_stale = true;
    int64_t bws = 0;
    for (int d0 = 0; d0 < p->ndm; d0 += 8)
        for (int c = 0; c < p->nchan; ++c) {
            int32_t lo = INT32_MAX, hi = 0;
            for (int d = d0; d < std::min(p->ndm, d0 + 8); ++d) {
                lo = std::min(lo, p->delay[(size_t)d * p->nchan + c]);
                hi = std::max(hi, p->delay[(size_t)d * p->nchan + c]);
            }
            bws = std::max<int64_t>(bws, (int64_t)hi - lo);
        }
    p->bw_span = (int32_t)std::min<int64_t>(bws, INT32_MAX);
    return build_schedule(p);
}

}  // namespace

namespace dd {

// The input gradient gI[c][tau] = sum_{d,k} w_dck g[d][tau - delta_dc - k] is a
// dedispersion with the roles swapped: output rows are channels, input rows are the
// trials' output gradients zero-padded by P = d_max on both sides, delays
// P - delta_dc - n_dc + 1 and the taps' weights reversed.  This builds that plan's
// tables on the host (its weights are filled on the device from the forward plan's).
dd_status build_adjoint_plan(dd_plan_s* p) {
    const int D = p->ndm, C = p->nchan;
    const int32_t P = p->dmax;
    if (p->adj) {
        destroy_plan(p->adj);
        p->adj = nullptr;
    }
    dd_plan_s* t = new (std::nothrow) dd_plan_s;
    if (!t) return DD_ERR_OOM;
    t->band = p->band;
    t->band.nchan = D;
    t->band.in_type = DD_F32;
    t->band.descending = 0;
    t->band.nsamp = 0;
    t->nchan = D;
    t->ndm = C;
    t->dms.assign(C, 0.0);
    t->delay.resize((size_t)C * D);
    t->taps.resize((size_t)C * D);
    for (int d = 0; d < D; ++d)
        for (int c = 0; c < C; ++c) {
            const size_t dc = (size_t)d * C + c, cd = (size_t)c * D + d;
            t->delay[cd] = P - p->delay[dc] - p->taps[dc] + 1;
            t->taps[cd] = p->taps[dc];
        }
    t->unit = false;
    t->kpad = p->kpad;
    t->kuser = p->kuser;
    t->w.assign((size_t)C * D * t->kpad, 0.0f);
    dd_status st = finish_profiles(t);
    if (st != DD_OK) {
        delete t;
        return st;
    }
    p->adj = t;
    p->adj_stale = false;
    p->adj_w_stale = true;
    return DD_OK;
}

int log_level() {
    static const int level = [] {
        const char* v = std::getenv("DD_LOG");
        return v ? std::atoi(v) : 0;
    }();
    return level;
}

void log_msg(int level, const char* fmt, ...) {
    if (log_level() < level) return;
    char line[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(line, sizeof line, fmt, ap);
    va_end(ap);
    std::fprintf(stderr, "[dd] %s\n", line);
}

dd_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return DD_OK;
    return e == cudaErrorMemoryAllocation ? DD_ERR_OOM : DD_ERR_CUDA;
}

static void free_dev(dd_plan_s* p) {
    if (p->dev.device < 0) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != p->dev.device) cudaSetDevice(p->dev.device);
    cudaFree(p->dev.delay);
    cudaFree(p->dev.taps);
    cudaFree(p->dev.w);
    cudaFree(p->dev.blk_lo);
    cudaFree(p->dev.rec);
    cudaFree(p->dev.status);
    cudaFree(p->dev.off);
    cudaFree(p->dev.mu);
    cudaFree(p->dev.isd);
    cudaFree(p->dev.widths);
    cudaFree(p->dev.narrow);
    if (cur >= 0 && cur != p->dev.device) cudaSetDevice(cur);
    p->dev = DevTables{};
    p->widths_on_dev.clear();
}

template <typename T>
static dd_status put(T** dst, const T* src, size_t n) {
    cudaError_t e = cudaMalloc((void**)dst, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) return cuda_status(e);
    if (n) e = cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
    return cuda_status(e);
}

void destroy_plan(dd_plan_s* p) {
    if (p->adj) destroy_plan(p->adj);
    if (p->d_gpad) cudaFree(p->d_gpad);
    if (p->d_gsplit) cudaFree(p->d_gsplit);
    if (p->d_prefix) cudaFree(p->d_prefix);
    if (p->d_fkey) cudaFree(p->d_fkey);
    if (p->d_fcarry) cudaFree(p->d_fcarry);
    if (p->d_fseam) cudaFree(p->d_fseam);
    if (p->d_fstarts) cudaFree(p->d_fstarts);
    free_dev(p);
    delete p;
}

dd_status upload_tables(dd_plan_s* p) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (!p->dev_dirty && p->dev.device == dev) return DD_OK;
    free_dev(p);
    p->dev.device = dev;
    const size_t n = (size_t)p->ndm * p->nchan;
    dd_status st;
    if ((st = put(&p->dev.delay, p->delay.data(), n)) != DD_OK) return st;
    if ((st = put(&p->dev.taps, p->taps.data(), n)) != DD_OK) return st;
    if (!p->unit && (st = put(&p->dev.w, p->w.data(), p->w.size())) != DD_OK) return st;
    if ((st = put(&p->dev.blk_lo, p->blk_lo.data(), p->blk_lo.size())) != DD_OK) return st;
    if ((st = put(&p->dev.rec, p->rec.data(), p->rec.size())) != DD_OK) return st;
    const int32_t zero = 0;
    if ((st = put(&p->dev.status, &zero, 1)) != DD_OK) return st;
    e = cudaMalloc((void**)&p->dev.off, (size_t)p->ndm * sizeof(double));
    if (e != cudaSuccess) return cuda_status(e);
    // place dd_boxcar_snr_noalloc's scratch array and kernels on this device now, so
    // that its calls allocate nothing (lazy module loading would do it at its first call)
    if ((st = noalloc_preload()) != DD_OK) return st;
    p->dev_dirty = false;
    return DD_OK;
}

}  // namespace dd

extern "C" {

const char* dd_status_str(dd_status s) {
    switch (s) {
        case DD_OK: return "ok";
        case DD_ERR_ARG: return "invalid argument";
        case DD_ERR_OVERFLOW: return "integer overflow";
        case DD_ERR_OOM: return "out of memory";
        case DD_ERR_CUDA: return "CUDA error";
        case DD_ERR_STATE: return "invalid state";
        case DD_ERR_TIMEOUT: return "device wait timed out";
        case DD_ERR_CAPACITY: return "capacity exceeded";
        case DD_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

int32_t dd_version(void) { return 100; }

dd_status dd_trial_dms(const dd_band* band, double dm0, double dm_max, int32_t n,
                       double tau_av_ms, int32_t smear_terms, double* dms_out,
                       double* eps_out) {
    if (!band_ok(band) || !dms_out || n < 2 || !(dm_max > dm0) || dm0 < 0 ||
        tau_av_ms < 0 || (smear_terms != 1 && smear_terms != 2))
        return DD_ERR_ARG;
    const dd_band& b = *band;
    const double k = kdm_of(b);
    const double dnu = b.df_mhz / 1000.0;
    const double geo = inv_mean_inv_cube(b);
    const double dm_diag = b.dt_ms / (2.0 * k * dnu) * geo;   // Sec. 6.2, kappa = 1/k
    const double dm_tau = tau_av_ms / (2.0 * k * dnu) * geo;  // eq. DM_tau
    const double extra2 = dm_diag * dm_diag + (smear_terms == 2 ? dm_tau * dm_tau : 0.0);
    std::vector<double> tmp(n);
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 200; ++it) {
        build_trials(b, dm0, hi, n, extra2, tmp.data());
        if (tmp[n - 1] >= dm_max) break;
        hi *= 2.0;
    }
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        build_trials(b, dm0, mid, n, extra2, tmp.data());
        if (tmp[n - 1] < dm_max) lo = mid; else hi = mid;
    }
    const double eps = 0.5 * (lo + hi);
    build_trials(b, dm0, eps, n, extra2, dms_out);
    if (eps_out) *eps_out = eps;
    return DD_OK;
}

dd_status dd_plan_create(dd_plan_t* out, const dd_band* band, const double* dms, int32_t ndm) {
    if (!out || !band_ok(band) || !dms || ndm < 1) return DD_ERR_ARG;
    *out = nullptr;
    for (int d = 0; d < ndm; ++d)
        if (!(dms[d] >= 0.0) || !std::isfinite(dms[d])) return DD_ERR_ARG;
    dd_plan_s* p = new (std::nothrow) dd_plan_s;
    if (!p) return DD_ERR_OOM;
    p->band = *band;
    p->nchan = band->nchan;
    p->ndm = ndm;
    p->dms.assign(dms, dms + ndm);
    const size_t n = (size_t)ndm * band->nchan;
    p->delay.resize(n);
    p->taps.resize(n);
    const double k = kdm_of(*band);
    const double top = band_top_ghz(*band);
    const double dnu = band->df_mhz / 1000.0;
    for (int d = 0; d < ndm; ++d) {
        for (int c = 0; c < band->nchan; ++c) {
            const double nu = chan_top_ghz(*band, c);
            const double lo = nu - dnu;
            const double raw_d = k * dms[d] * (1.0 / (nu * nu) - 1.0 / (top * top)) / band->dt_ms;
            const double raw_n = k * dms[d] * (1.0 / (lo * lo) - 1.0 / (nu * nu)) / band->dt_ms;
            if (!(raw_d < 2.0e9) || !(raw_n < 2.0e9)) {
                delete p;
                return DD_ERR_OVERFLOW;
            }
            p->delay[(size_t)d * band->nchan + c] = (int32_t)std::floor(raw_d);
            p->taps[(size_t)d * band->nchan + c] = std::max(1, (int32_t)std::ceil(raw_n));
        }
    }
    dd_status st = finish_profiles(p);
    if (st != DD_OK) {
        delete p;
        return st;
    }
    *out = p;
    return DD_OK;
}

dd_status dd_set_profiles(dd_plan_t p, const int32_t* delay, const int32_t* ntaps,
                          const float* w, int32_t kmax) {
    if (!p) return DD_ERR_ARG;
    const size_t n = (size_t)p->ndm * p->nchan;
    if (w && kmax < 1) return DD_ERR_ARG;
    if (delay)
        for (size_t i = 0; i < n; ++i)
            if (delay[i] < 0) return DD_ERR_ARG;
    if (ntaps)
        for (size_t i = 0; i < n; ++i)
            if (ntaps[i] < 1) return DD_ERR_ARG;
    // keep the old state so that a rejected profile leaves the plan usable
    std::vector<int32_t> old_d = p->delay, old_t = p->taps;
    std::vector<float> old_w = p->w;
    int32_t old_kpad = p->kpad, old_kuser = p->kuser;
    bool old_unit = p->unit;
    if (delay) std::memcpy(p->delay.data(), delay, n * sizeof(int32_t));
    if (ntaps) std::memcpy(p->taps.data(), ntaps, n * sizeof(int32_t));
    if (w) {
        for (size_t i = 0; i < n; ++i)
            if (p->taps[i] > kmax) {
                p->delay = old_d;
                p->taps = old_t;
                return DD_ERR_ARG;
            }
        p->kpad = (kmax + 3) / 4 * 4;
        p->kuser = kmax;
        p->w.assign(n * (size_t)p->kpad, 0.0f);
        for (size_t i = 0; i < n; ++i)
            for (int k = 0; k < p->taps[i]; ++k) p->w[i * p->kpad + k] = w[i * (size_t)kmax + k];
        p->unit = false;
    } else {
        p->w.clear();
        p->kpad = 0;
        p->kuser = 0;
        p->unit = true;
    }
    dd_status st = finish_profiles(p);
    if (st != DD_OK) {
        p->delay = old_d;
        p->taps = old_t;
        p->w = old_w;
        p->kpad = old_kpad;
        p->kuser = old_kuser;
        p->unit = old_unit;
        finish_profiles(p);
        return st;
    }
    p->dev_dirty = true;
    return DD_OK;
}

dd_status dd_set_weights_device(dd_plan_t p, const float* d_w, int32_t kmax, void* stream) {
    if (!p || !d_w || kmax < 1) return DD_ERR_ARG;
    if (p->kmax > kmax) return DD_ERR_ARG;
    const int32_t kpad = (kmax + 3) / 4 * 4;
    if (p->unit || p->kpad != kpad || p->kuser != kmax) {
        // switch the plan to weighted with this row length; host weights start at zero
        const size_t n = (size_t)p->ndm * p->nchan;
        p->w.assign(n * (size_t)kpad, 0.0f);
        p->kpad = kpad;
        p->kuser = kmax;
        p->unit = false;
        dd_status st = finish_profiles(p);
        if (st != DD_OK) return st;
    }
    dd_status st = dd::upload_tables(p);
    if (st != DD_OK) return st;
    cudaError_t e = cudaMemcpy2DAsync(p->dev.w, (size_t)kpad * sizeof(float), d_w,
                                      (size_t)kmax * sizeof(float), (size_t)kmax * sizeof(float),
                                      (size_t)p->ndm * p->nchan, cudaMemcpyDeviceToDevice,
                                      (cudaStream_t)stream);
    if (e != cudaSuccess) return dd::cuda_status(e);
    p->adj_w_stale = true;
    return dd::launch_repack(p, (cudaStream_t)stream);
}

dd_status dd_plan_info(dd_plan_t p, int64_t* t_out, int32_t* d_max, int32_t* kmax,
                       int64_t* ns_total, int32_t* out_is_int) {
    if (!p) return DD_ERR_ARG;
    if (t_out) *t_out = std::max<int64_t>(0, p->band.nsamp - p->dmax);
    if (d_max) *d_max = p->dmax;
    if (kmax) *kmax = p->kmax;
    if (ns_total) *ns_total = p->ns_total;
    if (out_is_int) *out_is_int = p->out_int ? 1 : 0;
    return DD_OK;
}

dd_status dd_get_tables(dd_plan_t p, int32_t* delay, int32_t* ntaps) {
    if (!p) return DD_ERR_ARG;
    const size_t n = (size_t)p->ndm * p->nchan;
    if (delay) std::memcpy(delay, p->delay.data(), n * sizeof(int32_t));
    if (ntaps) std::memcpy(ntaps, p->taps.data(), n * sizeof(int32_t));
    return DD_OK;
}

static bool aligned16(const void* ptr) { return ((uintptr_t)ptr & 15u) == 0; }

dd_status dd_dedisperse(dd_plan_t p, const void* in, int64_t in_ld, int64_t t_offset,
                        int64_t nsamp, void* out, int64_t out_ld, void* stream) {
    DD_TRACE("dd_dedisperse");
    dd::log_msg(2, "dd_dedisperse: %d trials, t_offset %lld, nsamp %lld", p ? p->ndm : 0, (long long)t_offset, (long long)nsamp);
    if (!p || !in || !out) return DD_ERR_ARG;
    const int64_t esz = p->band.in_type == DD_U8 ? 1 : 4;
    if (nsamp <= 0) nsamp = p->band.nsamp;
    if (t_offset < 0 || nsamp <= p->dmax || t_offset + nsamp > in_ld) return DD_ERR_ARG;
    if (!aligned16(in) || (in_ld * esz) % 16 != 0) return DD_ERR_ARG;
    const int64_t t_out = nsamp - p->dmax;
    if (out_ld < t_out) return DD_ERR_ARG;
    if (t_out > INT32_MAX - dd::chunk_t(false) * dd::kWarps || in_ld > (int64_t)1 << 40) return DD_ERR_OVERFLOW;
    if (p->rl && nsamp > ((int64_t)1 << 24)) return DD_ERR_UNSUPPORTED;
    dd_status st = dd::upload_tables(p);
    if (st != DD_OK) return st;
    if (p->rl) return dd::launch_dedisperse_rl(p, in, in_ld, t_offset, nsamp, out, out_ld, (cudaStream_t)stream);
    return dd::launch_dedisperse(p, in, in_ld, t_offset, t_out, out, out_ld, (cudaStream_t)stream);
}

dd_status dd_channel_stats(dd_plan_t p, const void* in, int64_t in_ld, int64_t t_offset,
                           int64_t nsamp, double* mean, double* sd, void* stream) {
    DD_TRACE("dd_channel_stats");
    if (!p || !in || !mean || !sd) return DD_ERR_ARG;
    if (nsamp <= 0) nsamp = p->band.nsamp;
    if (t_offset < 0 || nsamp < 1 || t_offset + nsamp > in_ld) return DD_ERR_ARG;
    dd_status st = dd::upload_tables(p);
    if (st != DD_OK) return st;
    return dd::launch_channel_stats(p, in, in_ld, t_offset, nsamp, mean, sd, (cudaStream_t)stream);
}

dd_status dd_boxcar_snr(dd_plan_t p, const void* x, int64_t ld, int64_t t_len,
                        const int32_t* widths, int32_t nw, const double* mean,
                        const double* sd, float* peak, int32_t* arg, float thresh,
                        dd_candidate* cands, int32_t cap, int32_t* ncands, void* stream) {
    DD_TRACE("dd_boxcar_snr");
    dd::log_msg(2, "dd_boxcar_snr: %d trials, %lld samples, %d widths", p ? p->ndm : 0, (long long)t_len, nw);
    if (!p || !x || !widths || nw < 1 || !mean || !sd || !peak || !arg) return DD_ERR_ARG;
    if (t_len < 1 || ld < t_len || t_len > INT32_MAX) return DD_ERR_ARG;
    if (cands && (!ncands || cap < 0)) return DD_ERR_ARG;
    for (int i = 0; i < nw; ++i) {
        if (widths[i] < 1 || widths[i] > t_len) return DD_ERR_ARG;
        if (i && widths[i] <= widths[i - 1]) return DD_ERR_ARG;
    }
    dd_status st = dd::upload_tables(p);
    if (st != DD_OK) return st;
    return dd::launch_boxcar(p, x, ld, t_len, widths, nw, mean, sd, peak, arg, thresh, cands,
                             cap, ncands, (cudaStream_t)stream);
}

dd_status dd_backward(dd_plan_t p, const float* in, int64_t in_ld, int64_t t_offset,
                      int64_t nsamp, const float* g, int64_t gld, float* gw, float* gin,
                      int64_t gin_ld, void* stream) {
    DD_TRACE("dd_backward");
    dd::log_msg(2, "dd_backward: %d trials, nsamp %lld, weight gradient %s, input gradient %s", p ? p->ndm : 0,
             (long long)nsamp, gw ? "yes" : "no", gin ? "yes" : "no");
    if (!p || !in || !g) return DD_ERR_ARG;
    if (p->band.in_type != DD_F32) return DD_ERR_UNSUPPORTED;
    if (nsamp <= 0) nsamp = p->band.nsamp;
    if (t_offset < 0 || nsamp <= p->dmax || t_offset + nsamp > in_ld) return DD_ERR_ARG;
    const int64_t t_out = nsamp - p->dmax;
    if (gld < t_out) return DD_ERR_ARG;
    if (gin && (gin_ld < t_offset + nsamp || (gin_ld * 4) % 16 != 0 || !aligned16(gin)))
        return DD_ERR_ARG;
    if (!aligned16(in) || (in_ld * 4) % 16 != 0) return DD_ERR_ARG;
    dd_status st = dd::upload_tables(p);
    if (st != DD_OK) return st;
    return dd::launch_backward(p, in, in_ld, t_offset, t_out, g, gld, gw, gin, gin_ld,
                               (cudaStream_t)stream);
}

dd_status dd_plan_set_schedule(dd_plan_t p, int32_t nch, int32_t cs) {
    if (!p) return DD_ERR_ARG;
    const int old_nch = p->nch, old_cs = p->cs;
    dd_status st = build_schedule_fixed(p, nch, cs);
    if (st != DD_OK && (p->nch != old_nch || p->cs != old_cs)) build_schedule_fixed(p, old_nch, old_cs);
    return st;
}

dd_status dd_plan_get_schedule(dd_plan_t p, int32_t* nch, int32_t* cs, int32_t* trials_per_cta) {
    if (!p) return DD_ERR_ARG;
    if (nch) *nch = p->nch;
    if (cs) *cs = p->cs;
    if (trials_per_cta) *trials_per_cta = trials_per_unit(p) * units_per_warp(p) * dd::kWarps / p->nch;
    return DD_OK;
}

dd_status dd_plan_set_method(dd_plan_t p, int32_t method) {
    if (!p || method < DD_METHOD_AUTO || method > DD_METHOD_RUNLENGTH) return DD_ERR_ARG;
    if (method == DD_METHOD_RUNLENGTH && !(p->unit && p->band.in_type == DD_U8)) return DD_ERR_UNSUPPORTED;
    const int32_t old = p->method;
    p->method = method;
    dd_status st = build_schedule(p);
    if (st != DD_OK) {
        p->method = old;
        build_schedule(p);
    }
    return st;
}

dd_status dd_plan_get_method(dd_plan_t p, int32_t* method) {
    if (!p || !method) return DD_ERR_ARG;
    *method = p->rl ? DD_METHOD_RUNLENGTH : DD_METHOD_DIRECT;
    return DD_OK;
}

namespace {

std::mutex g_tune_mu;

// Schedule cache key: channel count, input type, path, and the trial-block delay
// spread and widest tap run in powers of two -- the quantities that decide which CTA
// shape and stage size fit and run best.
std::string tune_key(const dd_plan_s* p) {
    const int64_t span8 = block_span(p, 8, nullptr);
    const int sb = (int)std::floor(std::log2((double)span8 + 1.0));
    const int kb = (int)std::floor(std::log2((double)p->kmax + 1.0));
    std::ostringstream o;
    o << "C" << p->nchan << "_" << (p->band.in_type == DD_U8 ? "u8" : "f32") << "_"
      << (p->pair ? "pair" : (p->rl ? "rl" : "int")) << "_s" << sb << "_k" << kb;
    return o.str();
}

std::map<std::string, std::pair<int, int>> read_cache(const char* path) {
    std::map<std::string, std::pair<int, int>> m;
    if (!path) return m;
    std::ifstream f(path);
    std::string key;
    int nch, cs;
    double ms;
    while (f >> key >> nch >> cs >> ms) m[key] = {nch, cs};
    return m;
}

}  // namespace

dd_status dd_plan_autotune(dd_plan_t p, const void* d_in, int64_t in_ld, void* d_out,
                           int64_t out_ld, const char* cache_path, float* best_ms, void* stream) {
    DD_TRACE("dd_plan_autotune");
    if (!p || !d_in || !d_out) return DD_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const std::string key = tune_key(p);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto cache = read_cache(cache_path);
    auto hit = cache.find(key);
    if (hit != cache.end() && dd_plan_set_schedule(p, hit->second.first, hit->second.second) == DD_OK) {
        if (best_ms) *best_ms = -1.0f;
        dd::log_msg(1, "autotune %s: cached schedule (%d time chunks, %d channels per stage)", key.c_str(),
                 hit->second.first, hit->second.second);
        return DD_OK;
    }
    const bool u8 = stage_esz(p) == 1;
    const int cs_list_f[] = {2, 3, 4, 6, 8};
    const int cs_list_u[] = {4, 8, 12, 16};
    const int* cs_list = u8 ? cs_list_u : cs_list_f;
    const int ncs = u8 ? 4 : 5;
    const int orig_nch = p->nch, orig_cs = p->cs;
    int best_nch = orig_nch, best_cs = orig_cs;
    float best = 1e30f;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) return dd::cuda_status(ce);
    dd_status st = DD_OK;
    for (int nch = 1; nch <= 2 && st == DD_OK; nch *= 2) {
        for (int i = 0; i < ncs; ++i) {
            if (build_schedule_fixed(p, nch, cs_list[i]) != DD_OK) continue;
            st = dd_dedisperse(p, d_in, in_ld, 0, p->band.nsamp, d_out, out_ld, stream);
            if (st != DD_OK) break;
            float t = 1e30f;
            for (int rep = 0; rep < 2; ++rep) {
                cudaEventRecord(e0, s);
                st = dd_dedisperse(p, d_in, in_ld, 0, p->band.nsamp, d_out, out_ld, stream);
                cudaEventRecord(e1, s);
                if (st != DD_OK) break;
                ce = cudaEventSynchronize(e1);
                if (ce != cudaSuccess) {
                    st = dd::cuda_status(ce);
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                t = std::min(t, ms);
            }
            if (st != DD_OK) break;
            if (t < best) {
                best = t;
                best_nch = nch;
                best_cs = cs_list[i];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (build_schedule_fixed(p, best_nch, best_cs) != DD_OK) build_schedule_fixed(p, orig_nch, orig_cs);
    if (st != DD_OK) return st;
    if (best_ms) *best_ms = best;
    dd::log_msg(1, "autotune %s: %d time chunks, %d channels per stage, %.3f ms (default %d, %d)", key.c_str(),
             best_nch, best_cs, best, orig_nch, orig_cs);
    if (cache_path) {
        std::ofstream f(cache_path, std::ios::app);
        if (f) f << key << " " << best_nch << " " << best_cs << " " << best << "\n";
    }
    return DD_OK;
}

dd_status dd_get_device_status(dd_plan_t p, int32_t* code, void* stream) {
    if (!p || !code) return DD_ERR_ARG;
    *code = 0;
    if (p->dev.device < 0 || !p->dev.status) return DD_OK;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    int32_t v = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&v, p->dev.status, sizeof(v), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && v != 0) e = cudaMemset(p->dev.status, 0, sizeof(int32_t));
    if (e != cudaSuccess) return dd::cuda_status(e);
    *code = v;
    return DD_OK;
}

dd_status dd_test_set_wait(dd_plan_t p, int32_t skip_stage, int64_t wait_ns) {
    if (!p || wait_ns < 0) return DD_ERR_ARG;
    p->debug_skip_stage = skip_stage;
    p->wait_ns = wait_ns > 0 ? wait_ns : dd::kWaitNs;
    return DD_OK;
}

dd_status dd_plan_destroy(dd_plan_t p) {
    if (!p) return DD_ERR_ARG;
    dd::destroy_plan(p);
    return DD_OK;
}

}  // extern "C"
