// Profile construction on the host: the cell-averaged power of a model pulse (eq. Pavg
// for the rectangular scattered pulse of eq. profile_sb), the greedy sample selection
// for maximum S/N (Sec. 2.2, eq. sel_criterion) and the comparison detectors of Sec. 5,
// each of which turns a predicted power map into one trial's (delay, taps, weights)
// profile for the dedispersion kernel.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "dd_internal.h"

namespace {

constexpr double kDefaultKdm = 4.15;

double chan_lo_ghz(const dd_band& b, int c) {
    const int j = b.descending ? (b.nchan - 1 - c) : c;
    return (b.f_lo_mhz + j * b.df_mhz) / 1000.0;
}

}  // namespace

extern "C" {

dd_status dd_predict_rect(const dd_band* band, double dm, double t0_ms, double tau_ms,
                          double tau_prime_ms, double alpha, double nu0_ghz, double p0,
                          int32_t nt, double* pbar) {
    if (!band || !pbar || nt < 1 || band->nchan < 1 || !(band->dt_ms > 0) || !(band->df_mhz > 0) ||
        !(band->f_lo_mhz > 0) || dm < 0 || !(tau_prime_ms > 0) || tau_ms < 0 || !(nu0_ghz > 0))
        return DD_ERR_ARG;
    const dd_band& b = *band;
    const double k = b.k_dm > 0 ? b.k_dm : kDefaultKdm;
    const double dt = b.dt_ms;
    const double dnu = b.df_mhz / 1000.0;
    const double top = (b.f_lo_mhz + b.nchan * b.df_mhz) / 1000.0;
    const double amp = p0 * tau_ms / tau_prime_ms;   // fluence-conserving height
    std::fill(pbar, pbar + (size_t)b.nchan * nt, 0.0);
    for (int c = 0; c < b.nchan; ++c) {
        const double lo = chan_lo_ghz(b, c);
        // sub-channels: at least 64, and fine enough that one sub-channel's own sweep is
        // below tau'/16 (midpoint rule on the frequency integral)
        const double sweep = k * dm * (1.0 / (lo * lo) - 1.0 / ((lo + dnu) * (lo + dnu)));
        const int nf = std::max(64, (int)std::ceil(16.0 * sweep / tau_prime_ms));
        const double h = dnu / nf;
        double* row = pbar + (size_t)c * nt;
        for (int f = 0; f < nf; ++f) {
            const double nu = lo + (f + 0.5) * h;
            const double ta = t0_ms + k * dm * (1.0 / (nu * nu) - 1.0 / (top * top));
            const double tb = ta + tau_prime_ms;
            const double wgt = amp * std::pow(nu / nu0_ghz, -alpha) * h / dt;
            const int64_t j0 = std::max<int64_t>(0, (int64_t)std::floor(ta / dt));
            const int64_t j1 = std::min<int64_t>(nt - 1, (int64_t)std::floor(tb / dt));
            for (int64_t j = j0; j <= j1; ++j) {
                const double ov = std::min((j + 1) * dt, tb) - std::max(j * dt, ta);
                if (ov > 0) row[j] += wgt * ov;
            }
        }
    }
    return DD_OK;
}

dd_status dd_select_samples(const double* pbar, int32_t nchan, int32_t nt, int32_t kmax,
                            int32_t* delay, int32_t* ntaps, float* w, int32_t* nsel, double* gain) {
    if (!pbar || nchan < 1 || nt < 1 || kmax < 1 || !delay || !ntaps || !w) return DD_ERR_ARG;
    const size_t n = (size_t)nchan * nt;
    std::vector<int64_t> idx;
    double all_sum = 0.0;
    for (size_t i = 0; i < n; ++i)
        if (pbar[i] > 0) {
            idx.push_back((int64_t)i);
            all_sum += pbar[i];
        }
    // highest predicted power first; equal powers in (channel, sample) order
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return pbar[a] > pbar[b]; });
    std::vector<char> sel(n, 0);
    double sum = 0.0;
    int64_t cnt = 0;
    for (int64_t i : idx) {
        // eq. sel_criterion: add while P > (sqrt((N+1)/N) - 1) * (sum of the set)
        if (cnt > 0 && !(pbar[i] > (std::sqrt((double)(cnt + 1) / (double)cnt) - 1.0) * sum)) break;
        sel[(size_t)i] = 1;
        sum += pbar[i];
        ++cnt;
    }
    std::fill(w, w + (size_t)nchan * kmax, 0.0f);
    for (int c = 0; c < nchan; ++c) {
        int lo = -1, hi = -1;
        for (int j = 0; j < nt; ++j)
            if (sel[(size_t)c * nt + j]) {
                if (lo < 0) lo = j;
                hi = j;
            }
        if (lo < 0) {  // no sample of this channel: one tap of zero weight
            delay[c] = 0;
            ntaps[c] = 1;
            continue;
        }
        if (hi - lo + 1 > kmax) return DD_ERR_CAPACITY;
        delay[c] = lo;
        ntaps[c] = hi - lo + 1;
        for (int j = lo; j <= hi; ++j) w[(size_t)c * kmax + (j - lo)] = sel[(size_t)c * nt + j] ? 1.0f : 0.0f;
    }
    if (nsel) *nsel = (int32_t)cnt;
    if (gain) {
        const double snr_sel = cnt ? sum / std::sqrt((double)cnt) : 0.0;
        const double snr_all = idx.empty() ? 0.0 : all_sum / std::sqrt((double)idx.size());
        *gain = snr_all > 0 ? snr_sel / snr_all : 0.0;
    }
    return DD_OK;
}

dd_status dd_detector_profile(const double* pbar, int32_t nchan, int32_t nt, const int32_t* align,
                              int32_t kind, int32_t kmax, int32_t* delay, int32_t* ntaps, float* w,
                              double* snr) {
    if (!pbar || nchan < 1 || nt < 1 || kmax < 1 || !delay || !ntaps || !w || kind < 0 || kind > 2)
        return DD_ERR_ARG;
    if (kind > 0 && !align) return DD_ERR_ARG;
    std::fill(w, w + (size_t)nchan * kmax, 0.0f);
    double pmax = 0.0;
    for (size_t i = 0; i < (size_t)nchan * nt; ++i) pmax = std::max(pmax, pbar[i]);
    if (!(pmax > 0)) return DD_ERR_ARG;
    if (kind == 0) {
        // dynamic-spectrum matched filter: every cell weighted by its expected power
        double q = 0.0;
        for (int c = 0; c < nchan; ++c) {
            const double* row = pbar + (size_t)c * nt;
            int lo = -1, hi = -1;
            for (int j = 0; j < nt; ++j)
                if (row[j] > 0) {
                    if (lo < 0) lo = j;
                    hi = j;
                    q += row[j] * row[j];
                }
            if (lo < 0) {
                delay[c] = 0;
                ntaps[c] = 1;
                continue;
            }
            if (hi - lo + 1 > kmax) return DD_ERR_CAPACITY;
            delay[c] = lo;
            ntaps[c] = hi - lo + 1;
            for (int j = lo; j <= hi; ++j) w[(size_t)c * kmax + (j - lo)] = (float)(row[j] / pmax);
        }
        if (snr) *snr = std::sqrt(q);
        return DD_OK;
    }
    // time-series detectors: the channels aligned by `align` and summed into one series
    // T[m] = sum_c pbar[c][align[c] + m] over the window of m holding pulse power
    int64_t mlo = INT64_MAX, mhi = INT64_MIN;
    for (int c = 0; c < nchan; ++c)
        for (int j = 0; j < nt; ++j)
            if (pbar[(size_t)c * nt + j] > 0) {
                mlo = std::min<int64_t>(mlo, (int64_t)j - align[c]);
                mhi = std::max<int64_t>(mhi, (int64_t)j - align[c]);
            }
    const int64_t len = mhi - mlo + 1;
    if (len > kmax) return DD_ERR_CAPACITY;
    std::vector<double> T((size_t)len, 0.0);
    for (int c = 0; c < nchan; ++c) {
        if ((int64_t)align[c] + mlo < 0) return DD_ERR_ARG;
        for (int64_t m = 0; m < len; ++m) {
            const int64_t j = align[c] + mlo + m;
            if (j >= 0 && j < nt) T[(size_t)m] += pbar[(size_t)c * nt + j];
        }
    }
    double s1 = 0.0, s2 = 0.0, tmax = 0.0;
    for (double v : T) {
        s1 += v;
        s2 += v * v;
        tmax = std::max(tmax, v);
    }
    for (int c = 0; c < nchan; ++c) {
        delay[c] = (int32_t)(align[c] + mlo);
        ntaps[c] = (int32_t)len;
        for (int64_t m = 0; m < len; ++m)
            w[(size_t)c * kmax + m] = kind == 1 ? (float)(T[(size_t)m] / tmax) : 1.0f;
    }
    // unit noise per cell: the matched filter's S/N is sqrt(sum T^2 / C), the boxcar's
    // sum T / sqrt(C * len)
    if (snr) *snr = kind == 1 ? std::sqrt(s2 / nchan) : s1 / std::sqrt((double)nchan * (double)len);
    return DD_OK;
}

dd_status dd_select_profiles(dd_plan_t plan, double tau_ms, double tau_prime_ms, double alpha,
                             double nu0_ghz, double phase, int32_t kmax, int32_t* delay,
                             int32_t* ntaps, float* w, double* gains, int32_t* kused) {
    if (!plan || !delay || !ntaps || (w && kmax < 1) || !(phase >= 0) || !(tau_prime_ms > 0))
        return DD_ERR_ARG;
    const dd_band& b = plan->band;
    const double k = b.k_dm > 0 ? b.k_dm : kDefaultKdm;
    const double lo = b.f_lo_mhz / 1000.0;
    const double top = (b.f_lo_mhz + b.nchan * b.df_mhz) / 1000.0;
    const int C = b.nchan;
    int32_t kmx = 1;
    std::vector<double> pbar;
    std::vector<float> wrow;
    for (int d = 0; d < plan->ndm; ++d) {
        // cells from the arrival at the top of the band to the end of the sweep across the
        // whole band, the pulse width and two samples' margin
        const double span = k * plan->dms[d] * (1.0 / (lo * lo) - 1.0 / (top * top)) + tau_prime_ms +
                            2.0 * b.dt_ms;
        const double ntd = std::ceil(span / b.dt_ms) + 2.0;
        if (!(ntd < 1.0e8)) return DD_ERR_OVERFLOW;
        const int32_t nt = (int32_t)ntd;
        pbar.assign((size_t)C * nt, 0.0);
        dd_status st = dd_predict_rect(&b, plan->dms[d], phase * b.dt_ms, tau_ms, tau_prime_ms, alpha,
                                       nu0_ghz, 1.0, nt, pbar.data());
        if (st != DD_OK) return st;
        wrow.assign((size_t)C * nt, 0.0f);
        double g = 0.0;
        st = dd_select_samples(pbar.data(), C, nt, nt, delay + (size_t)d * C, ntaps + (size_t)d * C,
                               wrow.data(), nullptr, &g);
        if (st != DD_OK) return st;
        if (gains) gains[d] = g;
        for (int c = 0; c < C; ++c) {
            const int32_t n = ntaps[(size_t)d * C + c];
            kmx = std::max(kmx, n);
            if (!w) continue;
            if (n > kmax) return DD_ERR_CAPACITY;
            float* dst = w + ((size_t)d * C + c) * kmax;
            std::fill(dst, dst + kmax, 0.0f);
            std::copy(wrow.data() + (size_t)c * nt, wrow.data() + (size_t)c * nt + n, dst);
        }
    }
    if (kused) *kused = kmx;
    return DD_OK;
}

dd_status dd_exact_profiles(dd_plan_t plan, double tau_prime_ms, int32_t* delay, int32_t* ntaps) {
    if (!plan || !delay || !ntaps || tau_prime_ms < 0) return DD_ERR_ARG;
    const dd_band& b = plan->band;
    const double k = b.k_dm > 0 ? b.k_dm : kDefaultKdm;
    const double dnu = b.df_mhz / 1000.0;
    const double top = (b.f_lo_mhz + b.nchan * b.df_mhz) / 1000.0;
    for (int d = 0; d < plan->ndm; ++d)
        for (int c = 0; c < b.nchan; ++c) {
            const double nu = chan_lo_ghz(b, c) + dnu;  // the channel's top edge
            const double ta = k * plan->dms[d] * (1.0 / (nu * nu) - 1.0 / (top * top));
            const double smear = k * plan->dms[d] * (1.0 / ((nu - dnu) * (nu - dnu)) - 1.0 / (nu * nu));
            const double tb = ta + tau_prime_ms + smear;
            const double fa = std::floor(ta / b.dt_ms), cb = std::ceil(tb / b.dt_ms);
            if (!(cb - fa < 2.0e9)) return DD_ERR_OVERFLOW;
            delay[(size_t)d * b.nchan + c] = (int32_t)fa;
            ntaps[(size_t)d * b.nchan + c] = std::max<int32_t>(1, (int32_t)(cb - fa));
        }
    return DD_OK;
}

}  // extern "C"
