"""CPU oracle for profiled incoherent dedispersion and boxcar S/N (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this module.
The product path never imports it.  Everything here is written from the paper's
definitions in plain numpy, in float64 for floating point and int64 for integers,
with no blocking, fusion or reordering beyond what each definition states.

Notation follows the paper: C channels, Δt sampling time, Δν channel width, ν_c the
highest frequency in channel c (Sec. 3), 1/κ = k_dm in ms·GHz² (Sec. 2.1).

Functions and the passages they follow:
  channel_top_ghz, delay_table   Sec. 2.1 delay law and Sec. 3 t_A = DM/(κ ν_c²)
  taps_table                     Sec. 3 intra-channel smear Δτ_c, eq. num_samples
  dm_diag, dm_tau, trial_dms     Sec. 6.2–6.3, eq. trial DMs
  dedisperse                     eq. p_dedisp (Sec. 2.1), sample set S = {(c, δ+k)}
  channel_stats                  Sec. 2.1 radiometer noise per cell
  boxcar_norm                    eq. P_N_dedisp generalised to weighted, boxcar sums
  boxcar_snr                     eq. snr and the time-series boxcar detector (Sec. 5)
  adjoint                        transpose of eq. p_dedisp (no counterpart in the paper)
  snr_b_over_snr_i, dropout      eq. snrb/snri_approx and the trial-spacing limit
  dsmf_snr                       dynamic-spectrum matched filter S/N (Sec. 5)
"""
from __future__ import annotations

import math

import numpy as np

K_DM_DEFAULT = 4.15


# ----------------------------------------------------------------------------- band


def channel_top_ghz(nchan: int, f_lo_mhz: float, df_mhz: float, descending: bool = False) -> np.ndarray:
    """ν_c: the highest frequency of channel c in GHz (Sec. 3)."""
    out = np.empty(nchan, dtype=np.float64)
    for c in range(nchan):
        j = (nchan - 1 - c) if descending else c
        out[c] = (f_lo_mhz + (j + 1) * df_mhz) / 1000.0
    return out


def _top_of_band_ghz(nchan: int, f_lo_mhz: float, df_mhz: float) -> float:
    return (f_lo_mhz + nchan * df_mhz) / 1000.0


# ----------------------------------------------------------------------------- profiles


def delay_table(dms, nchan, f_lo_mhz, df_mhz, dt_ms, descending=False, k_dm=K_DM_DEFAULT):
    """δ_dc = ⌊k_dm·DM_d·(ν_c⁻² − ν_top⁻²)/Δt⌋, int32 [D][C].

    t_A = DM/(κ ν_c²) is where the pulse enters channel c (Sec. 3); subtracting the
    top-of-band delay makes the top channel start at sample 0.  Returns the table
    and the pre-floor values (for the near-integer report).
    """
    nu = channel_top_ghz(nchan, f_lo_mhz, df_mhz, descending)
    top = _top_of_band_ghz(nchan, f_lo_mhz, df_mhz)
    D = len(dms)
    raw = np.empty((D, nchan), dtype=np.float64)
    for d in range(D):
        for c in range(nchan):
            raw[d, c] = k_dm * float(dms[d]) * (1.0 / (nu[c] * nu[c]) - 1.0 / (top * top)) / dt_ms
    return np.floor(raw).astype(np.int32), raw


def taps_table(dms, nchan, f_lo_mhz, df_mhz, dt_ms, descending=False, k_dm=K_DM_DEFAULT):
    """n_dc = max(1, ⌈Δτ_dc/Δt⌉) with Δτ_dc the exact sweep across channel c.

    Δτ_c is the dispersion smear across the channel (Sec. 3); it is evaluated here
    as the difference of the delay law at the channel's two edges,
    k_dm·DM·((ν_c − Δν)⁻² − ν_c⁻²), rather than its first-order form 2·DM·Δν/(κν³).
    """
    nu = channel_top_ghz(nchan, f_lo_mhz, df_mhz, descending)
    dnu = df_mhz / 1000.0
    D = len(dms)
    raw = np.empty((D, nchan), dtype=np.float64)
    for d in range(D):
        for c in range(nchan):
            lo = nu[c] - dnu
            raw[d, c] = k_dm * float(dms[d]) * (1.0 / (lo * lo) - 1.0 / (nu[c] * nu[c])) / dt_ms
    return np.maximum(1, np.ceil(raw)).astype(np.int32), raw


# ----------------------------------------------------------------------------- trial DMs


def _mean_inv_cube(nu_ghz: np.ndarray) -> float:
    return float(np.mean(1.0 / nu_ghz ** 3))


def dm_diag(nchan, f_lo_mhz, df_mhz, dt_ms, k_dm=K_DM_DEFAULT):
    """Diagonal DM: average per-channel smear equals Δt (Sec. 6.2).

    DM_diag = Δt κ/(2Δν) · [(1/C) Σ ν_c⁻³]⁻¹ with κ = 1/k_dm.
    """
    nu = channel_top_ghz(nchan, f_lo_mhz, df_mhz)
    return dt_ms / (2.0 * k_dm * (df_mhz / 1000.0)) / _mean_inv_cube(nu)


def dm_tau(nchan, f_lo_mhz, df_mhz, tau_av_ms, k_dm=K_DM_DEFAULT):
    """DM_τ: average per-channel smear equals τ'_av (eq. DM_tau, Sec. 4 and 6.2)."""
    nu = channel_top_ghz(nchan, f_lo_mhz, df_mhz)
    return tau_av_ms / (2.0 * k_dm * (df_mhz / 1000.0)) / _mean_inv_cube(nu)


def trial_dms_for_eps(eps, n, dm0, nchan, f_lo_mhz, df_mhz, dt_ms, tau_av_ms,
                      smear_terms=2, k_dm=K_DM_DEFAULT):
    """eq. trial DMs: DM_n = DM_0 + (2ε/C) Σ_{i<n} √(DM_i² + DM_diag² + DM_τ²).

    smear_terms = 2 uses both DM_diag and DM_τ as printed; 1 keeps only DM_diag.
    """
    dd = dm_diag(nchan, f_lo_mhz, df_mhz, dt_ms, k_dm)
    dt_ = dm_tau(nchan, f_lo_mhz, df_mhz, tau_av_ms, k_dm)
    extra = dd * dd + (dt_ * dt_ if smear_terms == 2 else 0.0)
    out = np.empty(n, dtype=np.float64)
    out[0] = dm0
    acc = 0.0
    for i in range(1, n):
        acc += math.sqrt(out[i - 1] ** 2 + extra)
        out[i] = dm0 + 2.0 * eps / nchan * acc
    return out


def trial_dms(dm0, dm_max, n, nchan, f_lo_mhz, df_mhz, dt_ms, tau_av_ms,
              smear_terms=2, k_dm=K_DM_DEFAULT):
    """Trial list of eq. trial DMs with ε found by bisection so that DM_{N-1} = dm_max."""
    lo, hi = 0.0, 1.0
    while trial_dms_for_eps(hi, n, dm0, nchan, f_lo_mhz, df_mhz, dt_ms, tau_av_ms,
                            smear_terms, k_dm)[-1] < dm_max:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        last = trial_dms_for_eps(mid, n, dm0, nchan, f_lo_mhz, df_mhz, dt_ms, tau_av_ms,
                                 smear_terms, k_dm)[-1]
        if last < dm_max:
            lo = mid
        else:
            hi = mid
    eps = 0.5 * (lo + hi)
    dms = trial_dms_for_eps(eps, n, dm0, nchan, f_lo_mhz, df_mhz, dt_ms, tau_av_ms,
                            smear_terms, k_dm)
    return dms, eps


def dropout(eps):
    """Relative S/N floor between trials, (ε² + 1)^(-1/4) (Sec. 6.3)."""
    return (eps * eps + 1.0) ** -0.25


def snr_b_over_snr_i(ddm, dm, nchan, dm_diag_, dm_tau_):
    """eq. snrb/snri_approx: (C²δDM²/(DM² + DM_diag² + DM_τ²) + 1)^(-1/4)."""
    return (nchan * nchan * ddm * ddm / (dm * dm + dm_diag_ ** 2 + dm_tau_ ** 2) + 1.0) ** -0.25


# ----------------------------------------------------------------------------- dedispersion


def d_max(delays, taps):
    """Largest sample offset any output reads: max_{d,c} (δ_dc + n_dc − 1)."""
    return int((np.asarray(delays, np.int64) + np.asarray(taps, np.int64) - 1).max())


def dedisperse(I, delays, taps, w=None, t_offset=0, nsamp=None):
    """eq. p_dedisp with the trial's sample set S_d = {(c, δ_dc + k) : k < n_dc}.

    out[d][t] = Σ_c Σ_{k<n_dc} w_dck · I[c][t_offset + t + δ_dc + k],  0 ≤ t < T_out,
    T_out = nsamp − D_max.  uint8 input with w=None accumulates in int64 (exact);
    otherwise products and sums are float64.
    """
    I = np.asarray(I)
    delays = np.asarray(delays, np.int64)
    taps = np.asarray(taps, np.int64)
    D, C = delays.shape
    nsamp = I.shape[1] - t_offset if nsamp is None else nsamp
    t_out = nsamp - d_max(delays, taps)
    if t_out <= 0:
        return np.zeros((D, 0), np.int64 if w is None else np.float64)
    integer = w is None and np.issubdtype(I.dtype, np.integer)
    X = I.astype(np.int64 if integer else np.float64)
    out = np.zeros((D, t_out), dtype=np.int64 if integer else np.float64)
    for d in range(D):
        for c in range(C):
            for k in range(int(taps[d, c])):
                s = t_offset + int(delays[d, c]) + k
                seg = X[c, s:s + t_out]
                if w is None:
                    out[d] += seg
                else:
                    out[d] += np.float64(np.float32(w[d, c, k])) * seg
    return out


def channel_stats(I, t_offset=0, nsamp=None):
    """Per-channel mean and population standard deviation over the call's samples."""
    I = np.asarray(I)
    nsamp = I.shape[1] - t_offset if nsamp is None else nsamp
    X = I[:, t_offset:t_offset + nsamp].astype(np.float64)
    mu = X.mean(axis=1)
    sd = np.sqrt(((X - mu[:, None]) ** 2).mean(axis=1))
    return mu, sd


def boxcar_norm(taps, widths, mu_c, sigma_c, w=None):
    """Mean μ_dw and standard deviation σ_dw of a width-w boxcar of trial d on noise.

    With independent cells of mean μ_c and deviation σ_c, the boxcar sum
    B_w[t] = Σ_{j<w} out[d][t+j] weights cell (c, s) by v_dc = w_dc ⊛ 1_w, so
    E[B] = Σ_c μ_c Σ_m v_dcm and Var[B] = Σ_c σ_c² Σ_m v_dcm².  For unit weights and
    w = 1 this is σ√N_S of eq. P_N_dedisp.
    """
    taps = np.asarray(taps, np.int64)
    D, C = taps.shape
    W = len(widths)
    mu = np.zeros((D, W))
    var = np.zeros((D, W))
    for d in range(D):
        for c in range(C):
            n = int(taps[d, c])
            wv = np.ones(n) if w is None else np.asarray(w[d, c, :n], np.float32).astype(np.float64)
            for i, wd in enumerate(widths):
                v = np.convolve(wv, np.ones(int(wd)))
                mu[d, i] += mu_c[c] * v.sum()
                var[d, i] += sigma_c[c] ** 2 * (v * v).sum()
    return mu, np.sqrt(var)


def boxcar_snr(x, widths, mu_dw, sigma_dw):
    """Boxcar S/N of every trial and width (eq. snr with a boxcar in time, Sec. 5).

    B_w[t] = Σ_{j<w} x[d][t+j] for 0 ≤ t ≤ T_out − w; snr = (B_w − μ_dw)/σ_dw.
    Returns (peak_snr [D][W] float64, peak_t [D][W] int64, peak_B [D][W]); the
    earliest t wins a tie.  Integer series are summed in int64.
    """
    x = np.asarray(x)
    D, T = x.shape
    W = len(widths)
    integer = np.issubdtype(x.dtype, np.integer)
    peak = np.full((D, W), -np.inf)
    arg = np.full((D, W), -1, dtype=np.int64)
    best = np.zeros((D, W), dtype=np.int64 if integer else np.float64)
    for d in range(D):
        row = x[d].astype(np.int64 if integer else np.float64)
        P = np.concatenate([[0], np.cumsum(row)])
        for i, wd in enumerate(widths):
            wd = int(wd)
            if wd > T:
                continue
            B = P[wd:] - P[:-wd] if wd > 0 else None
            j = int(np.argmax(B))
            best[d, i] = B[j]
            arg[d, i] = j
            peak[d, i] = (float(B[j]) - mu_dw[d, i]) / sigma_dw[d, i]
    return peak, arg, best


def boxcar_series(x_row, width):
    """All B_w[t] of one row (float64 or int64)."""
    row = np.asarray(x_row)
    integer = np.issubdtype(row.dtype, np.integer)
    P = np.concatenate([[0], np.cumsum(row.astype(np.int64 if integer else np.float64))])
    return P[width:] - P[:-width]


def adjoint(I, g, delays, taps, w, t_offset=0, nsamp=None):
    """Transpose of the weighted eq. p_dedisp map (no counterpart in the paper).

    gw[d][c][k] = Σ_t g[d][t] · I[c][t_offset + t + δ_dc + k]
    gI[c][τ]    = Σ_d Σ_k w_dck · g[d][τ − t_offset − δ_dc − k]   (0 ≤ τ − … < T_out)
    Both in float64; gI has the shape of I.
    """
    I = np.asarray(I)
    g = np.asarray(g, np.float64)
    delays = np.asarray(delays, np.int64)
    taps = np.asarray(taps, np.int64)
    D, C = delays.shape
    K = w.shape[2]
    t_out = g.shape[1]
    X = I.astype(np.float64)
    gw = np.zeros((D, C, K))
    gI = np.zeros(X.shape)
    for d in range(D):
        for c in range(C):
            for k in range(int(taps[d, c])):
                s = t_offset + int(delays[d, c]) + k
                gw[d, c, k] = np.dot(g[d], X[c, s:s + t_out])
                gI[c, s:s + t_out] += np.float64(np.float32(w[d, c, k])) * g[d]
    return gw, gI


def dedisperse_points(I, delays, taps, points, w=None, t_offset=0):
    """eq. p_dedisp at chosen outputs only: out[d][t] for each (d, t) in `points`, summed
    over channels and taps as in `dedisperse` (int64 for uint8 input without weights,
    float64 otherwise).  For full-size checks where whole rows are too costly."""
    I = np.asarray(I)
    delays = np.asarray(delays, np.int64)
    taps = np.asarray(taps, np.int64)
    D, C = delays.shape
    integer = w is None and np.issubdtype(I.dtype, np.integer)
    res = []
    for d, t in points:
        acc = 0 if integer else 0.0
        for c in range(C):
            s = t_offset + int(t) + int(delays[d, c])
            n = int(taps[d, c])
            seg = I[c, s:s + n]
            if w is None:
                acc += int(seg.astype(np.int64).sum()) if integer else float(seg.astype(np.float64).sum())
            else:
                acc += float(np.dot(np.asarray(w[d, c, :n], np.float32).astype(np.float64),
                                    seg.astype(np.float64)))
        res.append(acc)
    return np.array(res, dtype=np.int64 if integer else np.float64)


def adjoint_points(I, g, delays, taps, w, gw_points=(), gi_points=(), t_offset=0):
    """The adjoint of `adjoint` at chosen entries: gw[d][c][k] for (d, c, k) in gw_points
    and gI[c][τ] for (c, τ) in gi_points, each summed directly from its definition."""
    I = np.asarray(I)
    g = np.asarray(g, np.float64)
    delays = np.asarray(delays, np.int64)
    taps = np.asarray(taps, np.int64)
    D, C = delays.shape
    t_out = g.shape[1]
    gw = []
    for d, c, k in gw_points:
        if k >= taps[d, c]:
            gw.append(0.0)
            continue
        s = t_offset + int(delays[d, c]) + int(k)
        gw.append(float(np.dot(g[d], I[c, s:s + t_out].astype(np.float64))))
    gi = []
    for c, tau in gi_points:
        acc = 0.0
        for d in range(D):
            for k in range(int(taps[d, c])):
                t = int(tau) - t_offset - int(delays[d, c]) - k
                if 0 <= t < t_out:
                    acc += float(np.float32(w[d, c, k])) * g[d, t]
        gi.append(acc)
    return np.array(gw), np.array(gi)


def select_samples(pbar):
    """Sample selection for maximum S/N (Sec. 2.2): starting from the empty set, take the
    sample of highest predicted power, then the next highest, while eq. sel_criterion
    P_next > (sqrt((N+1)/N) - 1) * (sum of the N taken) holds.  Equal powers are taken
    in row-major (channel, sample) order.  Returns a boolean mask of pbar's shape."""
    p = np.asarray(pbar, np.float64)
    flat = p.ravel()
    order = sorted((i for i in range(flat.size) if flat[i] > 0), key=lambda i: (-flat[i], i))
    mask = np.zeros(flat.size, bool)
    total, n = 0.0, 0
    for i in order:
        if n > 0 and not flat[i] > (math.sqrt((n + 1) / n) - 1.0) * total:
            break
        mask[i] = True
        total += flat[i]
        n += 1
    return mask.reshape(p.shape)


def set_snr(pbar, mask):
    """S/N of a sample set with equal noise per sample (eq. snr): sum P / sqrt(N)."""
    p = np.asarray(pbar, np.float64)[mask]
    return float(p.sum() / math.sqrt(p.size)) if p.size else 0.0


def detector_snrs(pbar, align, sigma=1.0):
    """S/N of the Sec. 5 detectors on one trial's predicted cell powers with noise sigma
    per cell: the dynamic-spectrum matched filter sqrt(sum P^2)/sigma; the time-series
    matched filter sqrt(sum_m T_m^2 / C)/sigma and boxcar sum_m T_m / sqrt(C N_t)/sigma on the
    series T_m = sum_c P[c][align_c + m] over the window holding power; the sample-selection
    detector (Sec. 2.2) and the every-sample-with-power detector sum P / sqrt(N)/sigma."""
    p = np.asarray(pbar, np.float64)
    C, nt = p.shape
    rows, cols = np.nonzero(p > 0)
    m = cols - np.asarray(align)[rows]
    lo, hi = int(m.min()), int(m.max())
    T = np.zeros(hi - lo + 1)
    for c in range(C):
        for k in range(hi - lo + 1):
            j = int(align[c]) + lo + k
            if 0 <= j < nt:
                T[k] += p[c, j]
    return {
        "dsmf": math.sqrt(float((p ** 2).sum())) / sigma,
        "ts_mf": math.sqrt(float((T ** 2).sum()) / C) / sigma,
        "ts_boxcar": float(T.sum()) / math.sqrt(C * T.size) / sigma,
        "selection": set_snr(p, select_samples(p)) / sigma,
        "all_samples": set_snr(p, p > 0) / sigma,
    }


def dsmf_snr(pbar, sigma):
    """Dynamic-spectrum matched filter S/N √(Σ P̄²)/σ (Sec. 5) for cell noise σ."""
    return math.sqrt(float((np.asarray(pbar, np.float64) ** 2).sum())) / sigma
