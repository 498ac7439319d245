/*
 * Brute-force CPU oracle for eq. p_dedisp (Sec. 2.1) -- test infrastructure only.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg load this
 * library; the product path never does.  It shares no code with the CUDA library.
 *
 *   out[d][t] = sum_c sum_{k < n_dc} w_dck * I[c][t_offset + t + delta_dc + k]
 *
 * for the trial rows listed in `rows` (all rows when rows == NULL) and
 * 0 <= t < t_out.  uint8 input with unit weights accumulates in int64 (exact);
 * float32 input accumulates float32*float32 products (exact in double) in double.
 * The summation runs over c, then k, in ascending order.  OpenMP splits the rows.
 */
#include <stdint.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_dedisperse_u8(const uint8_t* in, int64_t ld, int32_t nchan, int64_t t_offset,
                       const int32_t* delay, const int32_t* taps, int32_t ndm, int64_t t_out,
                       const int32_t* rows, int32_t nrows, int64_t* out) {
    int32_t n = rows ? nrows : ndm;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int32_t i = 0; i < n; ++i) {
        int32_t d = rows ? rows[i] : i;
        int64_t* o = out + (int64_t)i * t_out;
        memset(o, 0, sizeof(int64_t) * (size_t)t_out);
        for (int32_t c = 0; c < nchan; ++c) {
            int64_t del = delay[(int64_t)d * nchan + c];
            int32_t nt = taps[(int64_t)d * nchan + c];
            for (int32_t k = 0; k < nt; ++k) {
                const uint8_t* src = in + (int64_t)c * ld + t_offset + del + k;
                for (int64_t t = 0; t < t_out; ++t) o[t] += (int64_t)src[t];
            }
        }
    }
}

void orc_dedisperse_f32(const float* in, int64_t ld, int32_t nchan, int64_t t_offset,
                        const int32_t* delay, const int32_t* taps, const float* w, int32_t kmax,
                        int32_t ndm, int64_t t_out, const int32_t* rows, int32_t nrows,
                        double* out) {
    int32_t n = rows ? nrows : ndm;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int32_t i = 0; i < n; ++i) {
        int32_t d = rows ? rows[i] : i;
        double* o = out + (int64_t)i * t_out;
        memset(o, 0, sizeof(double) * (size_t)t_out);
        for (int32_t c = 0; c < nchan; ++c) {
            int64_t del = delay[(int64_t)d * nchan + c];
            int32_t nt = taps[(int64_t)d * nchan + c];
            const float* wd = w ? w + ((int64_t)d * nchan + c) * kmax : 0;
            for (int32_t k = 0; k < nt; ++k) {
                double wk = wd ? (double)wd[k] : 1.0;
                const float* src = in + (int64_t)c * ld + t_offset + del + k;
                for (int64_t t = 0; t < t_out; ++t) o[t] += wk * (double)src[t];
            }
        }
    }
}

/* Absolute-value twin of orc_dedisperse_f32: sum_c sum_k |w| * |I|, the scale that
 * bounds the rounding error of any summation order of the same terms. */
void orc_abs_scale_f32(const float* in, int64_t ld, int32_t nchan, int64_t t_offset,
                       const int32_t* delay, const int32_t* taps, const float* w, int32_t kmax,
                       int32_t ndm, int64_t t_out, const int32_t* rows, int32_t nrows,
                       double* out) {
    int32_t n = rows ? nrows : ndm;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int32_t i = 0; i < n; ++i) {
        int32_t d = rows ? rows[i] : i;
        double* o = out + (int64_t)i * t_out;
        memset(o, 0, sizeof(double) * (size_t)t_out);
        for (int32_t c = 0; c < nchan; ++c) {
            int64_t del = delay[(int64_t)d * nchan + c];
            int32_t nt = taps[(int64_t)d * nchan + c];
            const float* wd = w ? w + ((int64_t)d * nchan + c) * kmax : 0;
            for (int32_t k = 0; k < nt; ++k) {
                double wk = wd ? (double)wd[k] : 1.0;
                if (wk < 0) wk = -wk;
                const float* src = in + (int64_t)c * ld + t_offset + del + k;
                for (int64_t t = 0; t < t_out; ++t) {
                    double v = (double)src[t];
                    o[t] += wk * (v < 0 ? -v : v);
                }
            }
        }
    }
}

/* Transpose of the weighted map: gw[d][c][k] = sum_t g[d][t] I[c][t_offset+t+delta+k]
 * and gin[c][tau] = sum_d sum_k w_dck g[d][tau - t_offset - delta - k].  gin has
 * nchan rows of length ld and must be zeroed by the caller. */
void orc_adjoint_f32(const float* in, int64_t ld, int32_t nchan, int64_t t_offset,
                     const int32_t* delay, const int32_t* taps, const float* w, int32_t kmax,
                     int32_t ndm, int64_t t_out, const float* g, double* gw, double* gin) {
    #pragma omp parallel for schedule(dynamic, 1)
    for (int32_t d = 0; d < ndm; ++d) {
        const float* gd = g + (int64_t)d * t_out;
        for (int32_t c = 0; c < nchan; ++c) {
            int64_t del = delay[(int64_t)d * nchan + c];
            int32_t nt = taps[(int64_t)d * nchan + c];
            for (int32_t k = 0; k < nt; ++k) {
                const float* src = in + (int64_t)c * ld + t_offset + del + k;
                double s = 0.0;
                for (int64_t t = 0; t < t_out; ++t) s += (double)gd[t] * (double)src[t];
                gw[((int64_t)d * nchan + c) * kmax + k] = s;
            }
        }
    }
    #pragma omp parallel for schedule(dynamic, 1)
    for (int32_t c = 0; c < nchan; ++c) {
        double* gc = gin + (int64_t)c * ld;
        for (int32_t d = 0; d < ndm; ++d) {
            const float* gd = g + (int64_t)d * t_out;
            int64_t del = delay[(int64_t)d * nchan + c];
            int32_t nt = taps[(int64_t)d * nchan + c];
            for (int32_t k = 0; k < nt; ++k) {
                double wk = (double)w[((int64_t)d * nchan + c) * kmax + k];
                double* dst = gc + t_offset + del + k;
                for (int64_t t = 0; t < t_out; ++t) dst[t] += wk * (double)gd[t];
            }
        }
    }
}
