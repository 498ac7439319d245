"""Pins for the CPU oracle: it is checked against hand sums, textbook special cases,
closed forms and invariants fixed by the paper and by the mathematics, never against
itself.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import ref
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ----------------------------------------------------------------------------- hand sums


def test_hand_sums_unit_and_weighted():
    g = _gold("hand_sums.json")
    I = np.array(g["I"], dtype=np.uint8)
    dl = np.array(g["delays"], np.int32)
    tp = np.array(g["taps"], np.int32)
    out = ref.dedisperse(I, dl, tp)
    assert out.shape == (2, g["t_out"])
    assert out.tolist() == g["unit_out"]
    w = np.array(g["weights"], np.float32)
    outw = ref.dedisperse(I.astype(np.float32), dl, tp, w=w)
    np.testing.assert_array_equal(outw, np.array(g["weighted_out"]))
    # the C brute force gives the same numbers
    assert oracle.c_dedisperse(I, dl, tp).tolist() == g["unit_out"]
    np.testing.assert_array_equal(oracle.c_dedisperse(I.astype(np.float32), dl, tp, w=w),
                                  np.array(g["weighted_out"]))


def test_hand_boxcar():
    g = _gold("hand_sums.json")
    x = np.array(g["unit_out"], np.int64)
    bc = g["boxcar_width2_trial0"]
    assert ref.boxcar_series(x[0], 2).tolist() == bc["B"]
    mu = np.zeros((2, 1))
    sd = np.ones((2, 1))
    peak, arg, best = ref.boxcar_snr(x, [2], mu, sd)
    assert arg[0, 0] == bc["peak_t"] and best[0, 0] == bc["peak_B"]


def test_abs_scale_hand_values():
    """The fp32 tolerance scale Σ_c Σ_k |w_dck|·|I[c][t+δ+k]| on a hand-worked case with
    inputs and weights of both signs (tests/golden/abs_scale.json): the signed sums
    differ from it, so dropping either absolute value fails."""
    g = _gold("abs_scale.json")
    I = np.array(g["I"], np.float32)
    dl = np.array(g["delays"], np.int32)
    tp = np.array(g["taps"], np.int32)
    w = np.array(g["weights"], np.float32)
    scale = oracle.c_abs_scale(I, dl, tp, w=w)
    np.testing.assert_array_equal(scale, np.array(g["abs_scale"]))
    signed = oracle.c_dedisperse(I, dl, tp, w=w)
    assert signed[0, 0] == g["signed_trial0_t0"] and signed[1, 0] == g["signed_trial1_t0"]
    # planted mistakes: absolute value of I only, of w only
    assert not np.array_equal(oracle.c_dedisperse(np.abs(I), dl, tp, w=w), scale)
    assert not np.array_equal(oracle.c_dedisperse(I, dl, tp, w=np.abs(w)), scale)


def test_abs_scale_brute_force_and_rows():
    """The scale against a pure-Python loop over every (c, k) term on a small random case
    of mixed signs, for all rows, a row subset and an offset window."""
    rng = np.random.default_rng(31)
    C, T, D, K = 5, 40, 4, 4
    I = rng.standard_normal((C, T)).astype(np.float32)
    dl = rng.integers(0, 6, size=(D, C)).astype(np.int32)
    tp = rng.integers(1, K + 1, size=(D, C)).astype(np.int32)
    w = rng.uniform(-1.5, 1.5, size=(D, C, K)).astype(np.float32)
    t_off, nsamp = 3, 30
    t_out = nsamp - int((dl.astype(np.int64) + tp - 1).max())
    brute = np.zeros((D, t_out))
    for d in range(D):
        for t in range(t_out):
            s = 0.0
            for c in range(C):
                for k in range(int(tp[d, c])):
                    s += abs(float(w[d, c, k])) * abs(float(I[c, t_off + t + dl[d, c] + k]))
            brute[d, t] = s
    got = oracle.c_abs_scale(I, dl, tp, w=w, t_offset=t_off, nsamp=nsamp)
    np.testing.assert_allclose(got, brute, rtol=1e-13, atol=0)
    rows = np.array([1, 3], np.int32)
    np.testing.assert_allclose(oracle.c_abs_scale(I, dl, tp, w=w, t_offset=t_off, nsamp=nsamp, rows=rows),
                               brute[rows], rtol=1e-13, atol=0)
    # unit weights: Σ |I| over the sample set
    unit = oracle.c_abs_scale(I, dl, tp, t_offset=t_off, nsamp=nsamp)
    np.testing.assert_allclose(unit, ref.dedisperse(np.abs(I).astype(np.float64), dl, tp,
                                                    w=np.ones((D, C, K)), t_offset=t_off, nsamp=nsamp),
                               rtol=1e-13, atol=0)


def test_hand_adjoint():
    g = _gold("hand_sums.json")
    I = np.array(g["I"], np.float32)
    dl = np.array(g["delays"], np.int32)
    tp = np.array(g["taps"], np.int32)
    w = np.array(g["weights"], np.float32)
    a = g["adjoint_impulse_trial0"]
    gw, gI = ref.adjoint(I, np.array(a["g"], np.float64), dl, tp, w)
    np.testing.assert_array_equal(gI, np.array(a["gI"]))
    np.testing.assert_array_equal(gw[0], np.array(a["gw_trial0"]))


# ----------------------------------------------------------------------------- brute force


def test_boxcar_matches_explicit_loops():
    rng = np.random.default_rng(5)
    x = rng.integers(-50, 50, size=(3, 40)).astype(np.int64)
    widths = [1, 3, 7]
    mu = rng.normal(size=(3, 3))
    sd = rng.uniform(1, 2, size=(3, 3))
    peak, arg, best = ref.boxcar_snr(x, widths, mu, sd)
    for d in range(3):
        for i, w in enumerate(widths):
            sums = [sum(int(x[d, t + j]) for j in range(w)) for t in range(40 - w + 1)]
            m = max(sums)
            assert best[d, i] == m and arg[d, i] == sums.index(m)
            assert peak[d, i] == pytest.approx((m - mu[d, i]) / sd[d, i], rel=1e-12)


def test_dedisperse_matches_explicit_loops():
    rng = np.random.default_rng(6)
    C, T, D = 3, 30, 4
    I = rng.integers(0, 256, size=(C, T)).astype(np.uint8)
    dl = rng.integers(0, 6, size=(D, C)).astype(np.int32)
    tp = rng.integers(1, 5, size=(D, C)).astype(np.int32)
    out = ref.dedisperse(I, dl, tp)
    dmax = max(int(dl[d, c]) + int(tp[d, c]) - 1 for d in range(D) for c in range(C))
    for d in range(D):
        for t in range(T - dmax):
            s = 0
            for c in range(C):
                for k in range(int(tp[d, c])):
                    s += int(I[c, t + int(dl[d, c]) + k])
            assert out[d, t] == s


# ----------------------------------------------------------------------------- special cases


def test_dm_zero_is_channel_sum():
    rng = np.random.default_rng(7)
    band = synth.Band(16, 1200.0, 10.0, 1.0)
    I = rng.integers(0, 256, size=(16, 200)).astype(np.uint8)
    dl, _ = ref.delay_table([0.0], band.nchan, band.f_lo_mhz, band.df_mhz, band.dt_ms)
    tp, _ = ref.taps_table([0.0], band.nchan, band.f_lo_mhz, band.df_mhz, band.dt_ms)
    assert (dl == 0).all() and (tp == 1).all()
    out = ref.dedisperse(I, dl, tp)
    np.testing.assert_array_equal(out[0], I.astype(np.int64).sum(axis=0))


def test_single_channel_is_moving_sum():
    rng = np.random.default_rng(8)
    I = rng.integers(0, 256, size=(1, 300)).astype(np.uint8)
    for delta, n in [(0, 1), (3, 5), (10, 17)]:
        out = ref.dedisperse(I, np.array([[delta]]), np.array([[n]]))
        mv = np.convolve(I[0].astype(np.int64), np.ones(n, np.int64), "valid")
        np.testing.assert_array_equal(out[0], mv[delta:delta + out.shape[1]])


def test_one_tap_is_shift_and_add():
    """taps ≡ 1 reduces to one sample per channel (DART-style shift and add)."""
    rng = np.random.default_rng(9)
    C, T, D = 12, 500, 6
    I = rng.integers(0, 256, size=(C, T)).astype(np.uint8)
    dl = rng.integers(0, 40, size=(D, C)).astype(np.int32)
    tp = np.ones((D, C), np.int32)
    out = ref.dedisperse(I, dl, tp)
    t_out = T - int(dl.max())
    idx = np.arange(t_out)[None, None, :] + dl[:, :, None]                     # [D,C,T]
    gathered = np.take_along_axis(np.broadcast_to(I.astype(np.int64), (D, C, T)), idx, axis=2)
    np.testing.assert_array_equal(out, gathered.sum(axis=1))


def test_linearity_and_shift_equivariance():
    rng = np.random.default_rng(10)
    C, T, D = 8, 400, 5
    A = rng.integers(0, 100, size=(C, T)).astype(np.uint8)
    B = rng.integers(0, 100, size=(C, T)).astype(np.uint8)
    dl = rng.integers(0, 30, size=(D, C)).astype(np.int32)
    tp = rng.integers(1, 8, size=(D, C)).astype(np.int32)
    np.testing.assert_array_equal(ref.dedisperse(A + B, dl, tp),
                                  ref.dedisperse(A, dl, tp) + ref.dedisperse(B, dl, tp))
    s = 17
    full = ref.dedisperse(A, dl, tp)
    shifted = ref.dedisperse(A, dl, tp, t_offset=s, nsamp=T - s)
    np.testing.assert_array_equal(shifted, full[:, s:])


def test_numpy_and_c_oracles_agree():
    rng = np.random.default_rng(11)
    C, T, D, K = 10, 700, 7, 6
    dl = rng.integers(0, 50, size=(D, C)).astype(np.int32)
    tp = rng.integers(1, K + 1, size=(D, C)).astype(np.int32)
    I8 = rng.integers(0, 256, size=(C, T)).astype(np.uint8)
    np.testing.assert_array_equal(ref.dedisperse(I8, dl, tp, t_offset=3, nsamp=650),
                                  oracle.c_dedisperse(I8, dl, tp, t_offset=3, nsamp=650))
    If = rng.standard_normal((C, T)).astype(np.float32)
    w = rng.standard_normal((D, C, K)).astype(np.float32)
    np.testing.assert_allclose(ref.dedisperse(If, dl, tp, w=w),
                               oracle.c_dedisperse(If, dl, tp, w=w), rtol=0, atol=1e-11)
    rows = [4, 0, 6]
    np.testing.assert_allclose(oracle.c_dedisperse(If, dl, tp, w=w, rows=rows),
                               ref.dedisperse(If, dl, tp, w=w)[rows], rtol=0, atol=1e-11)


# ----------------------------------------------------------------------------- delay law


def test_delay_formula_plain_config():
    b = synth.PLAIN_BAND
    dms = np.linspace(0.0, 500.0, 128)
    dl, raw = ref.delay_table(dms, b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms)
    tp, _ = ref.taps_table(dms, b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms)
    # DM 500: lowest channel's top edge 1204.6875 MHz, top of band 1500 MHz
    expect = math.floor(4.15 * 500 * (1 / 1.2046875 ** 2 - 1 / 1.5 ** 2))
    assert dl[-1, 0] == expect == 507
    assert tp[-1, 0] == math.ceil(4.15 * 500 * (1 / 1.2 ** 2 - 1 / 1.2046875 ** 2)) == 12
    assert ref.d_max(dl, tp) == 518
    assert (dl[:, -1] == 0).all()                       # top channel starts at sample 0
    assert (np.diff(dl, axis=0) >= 0).all()             # monotone in DM
    assert (np.diff(dl, axis=1) <= 0).all()             # lower frequency, later arrival
    assert (np.diff(tp, axis=1) <= 0).all()
    # descending channel order mirrors the table
    dld, _ = ref.delay_table(dms, b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, descending=True)
    np.testing.assert_array_equal(dld, dl[:, ::-1])


def test_taps_cover_smear_and_exceed_taylor():
    """Δτ_c from the edge difference is ≥ the first-order 2·DM·Δν/(κ ν_c³) (ν⁻² is convex)."""
    b = synth.CRAFT_BAND
    dms = [100.0, 1000.0, 4000.0]
    _, raw = ref.taps_table(dms, b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms)
    nu = ref.channel_top_ghz(b.nchan, b.f_lo_mhz, b.df_mhz)
    taylor = np.array([[2 * dm * (b.df_mhz / 1000) * 4.15 / nu[c] ** 3 for c in range(b.nchan)] for dm in dms])
    assert (raw >= taylor).all() and (raw <= taylor * 1.01).all()


# ----------------------------------------------------------------------------- trial DMs


@pytest.mark.parametrize("eps,n,dm0,C,flo,df,dt,target", [
    (1.492, 442, 10.0, 304, 700.0, 1.0, 1.0, 3000.0),      # CRAFT, Sec. 6.3 / Fig. 7
    (0.580, 128, 50.0, 256, 21000.0, 7.8125, 0.1, 10000.0),  # Galactic Centre, 256 ch
    (0.287, 128, 50.0, 32, 21000.0, 62.5, 0.1, 10000.0),     # Galactic Centre, 32 ch
])
def test_trial_rule_printed_examples(eps, n, dm0, C, flo, df, dt, target):
    """With a single smear term (DM_diag = DM_τ here, since the pulse width equals Δt)
    the paper's ε values reproduce its printed DM ranges within 0.5 %."""
    dms = ref.trial_dms_for_eps(eps, n, dm0, C, flo, df, dt, dt, smear_terms=1)
    assert abs(dms[-1] - target) / target < 0.005
    assert (np.diff(dms) > 0).all()


def test_trial_rule_dropouts_and_limits():
    assert ref.dropout(1.492) == pytest.approx(0.75, abs=0.005)
    assert ref.dropout(0.580) == pytest.approx(0.93, abs=0.005)
    assert ref.dropout(0.287) == pytest.approx(0.98, abs=0.005)
    # exponential alternative of Fig. 7(b): 10·1.013^441 ≈ 3000
    assert 10 * 1.013 ** 441 == pytest.approx(3000, rel=0.01)
    b = synth.CRAFT_BAND
    dms, eps = ref.trial_dms(0.0, 4000.0, 4096, b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, 1.0)
    assert dms[-1] == pytest.approx(4000.0, rel=1e-9)
    dd = _smear_root_dm(b, b.dt_ms)
    dt_ = _smear_root_dm(b, 1.0)
    # low-DM step: (2ε/C)·√(DM_diag² + DM_τ²) from DM_0 = 0
    assert dms[1] - dms[0] == pytest.approx(2 * eps / b.nchan * math.sqrt(dd ** 2 + dt_ ** 2), rel=1e-12)
    # high-DM ratio tends to 1 + 2ε/C
    r = dms[-1] / dms[-2]
    lim = 1 + 2 * eps / b.nchan
    assert abs(r - lim) < 0.05 * (lim - 1)
    # DM_diag is where the mean first-order channel smear equals Δt
    nu = ref.channel_top_ghz(b.nchan, b.f_lo_mhz, b.df_mhz)
    mean_smear = np.mean(2 * ref.dm_diag(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms)
                         * (b.df_mhz / 1000) * 4.15 / nu ** 3)
    assert mean_smear == pytest.approx(b.dt_ms, rel=1e-12)


def _smear_root_dm(band, target_ms, k_dm=4.15):
    """The DM at which the mean first-order smear across a channel, 2·DM·Δν·k_dm/ν_c³
    (Sec. 3, averaged over the channels as in Sec. 6.2), equals target_ms: found by
    bisection on the smear itself, not from the closed form of eq. DM_tau."""
    nu = (band.f_lo_mhz + (np.arange(band.nchan) + 1) * band.df_mhz) / 1000.0
    dnu = band.df_mhz / 1000.0

    def mean_smear(dm):
        return float(np.mean([2.0 * dm * dnu * k_dm / v ** 3 for v in nu]))

    lo, hi = 0.0, 1.0
    while mean_smear(hi) < target_ms:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mean_smear(mid) < target_ms:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("band,tau_ms", [
    (synth.CRAFT_BAND, 3.0),                        # pulse three samples wide
    (synth.Band(304, 700.0, 1.0, 1.0), 0.25),       # narrower than a sample
    (synth.Band(256, 21000.0, 7.8125, 0.1), 2.0),   # Galactic-Centre band, 100 us sampling
])
def test_dm_tau_is_where_mean_smear_equals_pulse_width(band, tau_ms):
    """DM_τ (eq. DM_tau, Sec. 6.2) is the DM whose mean smear across a channel equals the
    scattered pulse width τ'_av; DM_diag the one whose smear equals Δt.  Checked at
    τ'_av ≠ Δt against a bisection on the smear, so that swapping τ' for Δt or dropping
    it fails; the ratio DM_τ/DM_diag is τ'_av/Δt."""
    dt_ = ref.dm_tau(band.nchan, band.f_lo_mhz, band.df_mhz, tau_ms)
    dd = ref.dm_diag(band.nchan, band.f_lo_mhz, band.df_mhz, band.dt_ms)
    assert dt_ == pytest.approx(_smear_root_dm(band, tau_ms), rel=1e-12)
    assert dd == pytest.approx(_smear_root_dm(band, band.dt_ms), rel=1e-12)
    assert dt_ / dd == pytest.approx(tau_ms / band.dt_ms, rel=1e-12)
    # the trial rule's low-DM step with both smear terms (eq. trial DMs at DM_0 = 0)
    dms, eps = ref.trial_dms(0.0, 2000.0, 512, band.nchan, band.f_lo_mhz, band.df_mhz,
                             band.dt_ms, tau_ms)
    step = 2 * eps / band.nchan * math.sqrt(_smear_root_dm(band, band.dt_ms) ** 2
                                            + _smear_root_dm(band, tau_ms) ** 2)
    assert dms[1] - dms[0] == pytest.approx(step, rel=1e-9)


def test_dm_error_attenuation_closed_form():
    """eq. snrb/snri_approx at the trial-spacing bound equals the drop-out (ε²+1)^(-1/4)."""
    C, dm, dd, dt_ = 336, 800.0, 255.0, 255.0
    for eps in (0.1, 0.5, 1.492):
        ddm = eps / C * math.sqrt(dm ** 2 + dd ** 2 + dt_ ** 2)
        assert ref.snr_b_over_snr_i(ddm, dm, C, dd, dt_) == pytest.approx(ref.dropout(eps), rel=1e-12)


# ----------------------------------------------------------------------------- noise model


def test_unit_weight_noise_is_sigma_sqrt_ns():
    """eq. P_N_dedisp: unit weights, width 1 → σ_dedisp = σ√N_S."""
    rng = np.random.default_rng(12)
    tp = rng.integers(1, 9, size=(5, 7))
    sig = 3.0
    mu, sd = ref.boxcar_norm(tp, [1], np.zeros(7), np.full(7, sig))
    np.testing.assert_allclose(sd[:, 0], sig * np.sqrt(tp.sum(axis=1)), rtol=1e-14)


def test_unit_weight_boxcar_norm_trapezoid():
    """Σ_m v_m² of 1_n ⊛ 1_w (a trapezoid) has the closed form (m−1)m(2m−1)/3 + m²(|n−w|+1)."""
    for n in (1, 2, 5, 13):
        for w in (1, 3, 8, 20):
            mu, sd = ref.boxcar_norm(np.array([[n]]), [w], np.array([2.0]), np.array([1.0]))
            m = min(n, w)
            closed = (m - 1) * m * (2 * m - 1) / 3 + m * m * (abs(n - w) + 1)
            assert sd[0, 0] ** 2 == pytest.approx(closed, rel=1e-13)
            assert mu[0, 0] == pytest.approx(2.0 * n * w, rel=1e-13)


def _noise_snr_moments(norm_fn):
    rng = np.random.default_rng(13)
    C, T, D, K = 24, 40000, 6, 6
    I = (rng.standard_normal((C, T)) * rng.uniform(0.5, 2.0, size=(C, 1)) + 3.0).astype(np.float32)
    dl = np.sort(rng.integers(0, 200, size=(D, C)), axis=1)[:, ::-1].astype(np.int32)
    tp = rng.integers(1, K + 1, size=(D, C)).astype(np.int32)
    w = rng.uniform(0.2, 1.5, size=(D, C, K)).astype(np.float32)
    widths = [1, 2, 5, 16]
    x = ref.dedisperse(I, dl, tp, w=w)
    mu_c, sd_c = ref.channel_stats(I)
    mu, sd = norm_fn(tp, widths, mu_c, sd_c, w)
    res = []
    for i, wd in enumerate(widths):
        s = np.concatenate([(ref.boxcar_series(x[d], wd) - mu[d, i]) / sd[d, i] for d in range(D)])
        res.append((s.mean(), s.std()))
    return res


def test_noise_boxcar_snr_is_unit_normal():
    """Pure noise through a weighted, tapped profile and every boxcar width gives S/N with
    mean 0 and standard deviation 1: the closed-form σ_dw accounts for the correlation
    that shared taps put between neighbouring outputs."""
    for m, s in _noise_snr_moments(ref.boxcar_norm):
        assert abs(m) < 0.05
        assert abs(s - 1.0) < 0.03


def test_noise_pin_catches_independent_sample_normaliser():
    """Planted mistake: treating the w boxcar outputs as independent (σ√w per output)
    must fail the unit-variance pin."""
    def naive(tp, widths, mu_c, sd_c, w):
        mu1, sd1 = ref.boxcar_norm(tp, [1], mu_c, sd_c, w)
        mu = np.concatenate([mu1 * wd for wd in widths], axis=1)
        sd = np.concatenate([sd1 * math.sqrt(wd) for wd in widths], axis=1)
        return mu, sd
    stds = [s for _, s in _noise_snr_moments(naive)]
    assert any(abs(s - 1.0) > 0.1 for s in stds)


# ----------------------------------------------------------------------------- injected pulse


def _plain_tables(b, dms):
    dl, _ = ref.delay_table(dms, b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms)
    tp, _ = ref.taps_table(dms, b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms)
    return dl, tp


def _best_trials(snr_total):
    out = []
    for s in range(20):
        p = synth.make_plain(seed=synth.sub_seed("tests", s), snr_total=snr_total)
        b = p["band"]
        dl, tp = _plain_tables(b, p["dms"])
        x = oracle.c_dedisperse(p["data"], dl, tp, nsamp=p["nsamp"])
        mu_c, sd_c = ref.channel_stats(p["data"], nsamp=p["nsamp"])
        widths = [1, 2, 3, 4, 6, 8]
        mu, sd = ref.boxcar_norm(tp, widths, mu_c, sd_c)
        peak, arg, _ = ref.boxcar_snr(x, widths, mu, sd)
        d_best = int(np.unravel_index(np.argmax(peak), peak.shape)[0])
        t76 = int(arg[76, int(np.argmax(peak[76]))])
        out.append((d_best, t76))
    return out


def test_injected_pulse_peaks_at_true_trial():
    """Plain config: the DM-300 pulse (top-of-band arrival sample 1000) is recovered at the
    nearest trial, index 76 (299.2 pc cm^-3).  At the config's 8σ amplitude the best
    trial is within one of 76 for ≥ 18 of 20 seeds and trial 76 always peaks within a
    sample of t = 1000; at 16σ every seed peaks exactly at trial 76."""
    res8 = _best_trials(8.0)
    assert sum(abs(d - 76) <= 1 for d, _ in res8) >= 18
    assert all(abs(t - 1000) <= 1 for _, t in res8)
    res16 = _best_trials(16.0)
    assert all(d == 76 and abs(t - 1000) <= 1 for d, t in res16)


# ----------------------------------------------------------------------------- paper closed forms


def _rect_snr(band, dm, tau, frac=0.37):
    """SNR[n0] of eq. snr for the noise-free rectangular pulse with S = every sample
    holding pulse power (Sec. 3), through the oracle's dedispersion and normaliser."""
    T = int(math.ceil((4.15 * dm * (1 / (band.f_lo_mhz / 1000) ** 2 - 1 / band.f_top_ghz ** 2)
                       + 3 * tau + 20 * band.dt_ms) / band.dt_ms)) + 4
    t0 = (2 + frac) * band.dt_ms
    P = synth.rect_pulse_cells(band, T, dm, t0, tau, tau)
    first = np.array([np.flatnonzero(P[c] > 0)[0] for c in range(band.nchan)])
    last = np.array([np.flatnonzero(P[c] > 0)[-1] for c in range(band.nchan)])
    n0 = int(first.min())
    dl = (first - n0)[None, :].astype(np.int32)
    tp = (last - first + 1)[None, :].astype(np.int32)
    x = ref.dedisperse(P, dl, tp, w=np.ones((1, band.nchan, int(tp.max())), np.float32))
    sigma_n = math.sqrt(band.df_mhz / 1000.0 / band.dt_ms)     # kT √(Δν/Δt), kT = 1
    _, sd = ref.boxcar_norm(tp, [1], np.zeros(band.nchan), np.full(band.nchan, sigma_n))
    return x[0, n0] / sd[0, 0]


def test_snr_decays_as_dt_to_minus_half():
    """Table tbl:snr_vs_dt_dv, coarse Δt (fine Δν): SNR[n0] ∝ Δt^(-1/2)."""
    snrs = [_rect_snr(synth.Band(3000, 700.0, 0.1, dt), 30.0, 1.0) for dt in (16.0, 64.0)]
    slope = math.log(snrs[1] / snrs[0]) / math.log(4.0)
    assert slope == pytest.approx(-0.5, abs=0.05)


def test_snr_decays_as_dnu_to_minus_half():
    """Table tbl:snr_vs_dt_dv, coarse Δν (fine Δt): SNR[n0] ∝ Δν^(-1/2)."""
    snrs = [_rect_snr(synth.Band(C, 700.0, 300.0 / C, 0.05), 300.0, 1.0) for C in (4, 32)]
    slope = math.log(snrs[1] / snrs[0]) / math.log(1 / 8)
    assert slope == pytest.approx(-0.5, abs=0.05)


@pytest.mark.parametrize("m", [0.05, 0.25, 1.0])
def test_snr_m_rule(m):
    """Δt = Av[Δτ_c] = m·τ'_av gives SNR[n0] ≈ SNR'_0/√(1+2m); > 0.80 SNR'_0 at m = 0.25 (Sec. 3)."""
    dm = 30.0
    nu = ref.channel_top_ghz(3000, 700.0, 0.1)
    dnu0 = 1.0 / (2 * 4.15 * dm) / np.mean(1 / nu ** 3)       # eq. delta_nu_0 in GHz, τ' = 1 ms
    C = int(round(0.3 / (m * dnu0)))
    snr = _rect_snr(synth.Band(C, 700.0, 300.0 / C, m * 1.0), dm, 1.0)
    snr0 = math.sqrt(0.3 * 1.0)                                # SNR'_0 = P0√(βτ)/kT, α = 0
    assert snr / snr0 == pytest.approx(1 / math.sqrt(1 + 2 * m), abs=0.02)
    if m <= 0.25:
        assert snr / snr0 > 0.80


# ----------------------------------------------------------------------------- adjoint


def test_adjoint_identities():
    """⟨A(w) I, g⟩ = ⟨I, Aᵀ g⟩ and, the map being linear in w too, = ⟨w, ∂_w⟩."""
    rng = np.random.default_rng(14)
    C, T, D, K = 9, 300, 5, 7
    I = rng.standard_normal((C, T)).astype(np.float32)
    dl = rng.integers(0, 40, size=(D, C)).astype(np.int32)
    tp = rng.integers(1, K + 1, size=(D, C)).astype(np.int32)
    w = rng.standard_normal((D, C, K)).astype(np.float32)
    for k in range(K):
        w[:, :, k] *= (k < tp)
    x = ref.dedisperse(I, dl, tp, w=w)
    g = rng.standard_normal(x.shape).astype(np.float32).astype(np.float64)
    gw, gI = ref.adjoint(I, g, dl, tp, w)
    lhs = float((x * g).sum())
    assert float((I.astype(np.float64) * gI).sum()) == pytest.approx(lhs, rel=1e-12)
    assert float((w.astype(np.float64) * gw).sum()) == pytest.approx(lhs, rel=1e-12)
    gw_c, gI_c = oracle.c_adjoint(I, g.astype(np.float32), dl, tp, w)
    np.testing.assert_allclose(gw_c, gw, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(gI_c, gI, rtol=1e-12, atol=1e-10)


def test_point_evaluations_match_full_oracle():
    """The point-wise forms used for full-size checks agree with the full sums: uint8
    exactly, float to rounding, and the adjoint points with `adjoint`."""
    rng = np.random.default_rng(77)
    C, T, D, K = 9, 400, 5, 7
    I8 = rng.integers(0, 256, size=(C, T)).astype(np.uint8)
    If = rng.standard_normal((C, T)).astype(np.float32)
    delay = rng.integers(0, 60, size=(D, C))
    taps = rng.integers(1, K + 1, size=(D, C))
    w = rng.standard_normal((D, C, K)).astype(np.float32)
    full8 = ref.dedisperse(I8, delay, taps, t_offset=3)
    fullf = ref.dedisperse(If, delay, taps, w=w, t_offset=3)
    pts = [(int(rng.integers(D)), int(rng.integers(full8.shape[1]))) for _ in range(25)]
    np.testing.assert_array_equal(ref.dedisperse_points(I8, delay, taps, pts, t_offset=3),
                                  [full8[d, t] for d, t in pts])
    np.testing.assert_allclose(ref.dedisperse_points(If, delay, taps, pts, w=w, t_offset=3),
                               [fullf[d, t] for d, t in pts], rtol=1e-12, atol=1e-12)
    g = rng.standard_normal((D, fullf.shape[1]))
    gw, gI = ref.adjoint(If, g, delay, taps, w, t_offset=3)
    gwp = [(int(rng.integers(D)), int(rng.integers(C)), int(rng.integers(K))) for _ in range(20)]
    gip = [(int(rng.integers(C)), int(rng.integers(T))) for _ in range(20)]
    a, b = ref.adjoint_points(If, g, delay, taps, w, gwp, gip, t_offset=3)
    np.testing.assert_allclose(a, [gw[d, c, k] for d, c, k in gwp], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(b, [gI[c, t] for c, t in gip], rtol=1e-12, atol=1e-12)


# ----------------------------------------------------------------------------- sample selection


def test_selection_is_the_first_peak_of_the_prefix_snr():
    """Sec. 2.2: the best set of each size is the top-N by power (brute force over every
    subset), and the greedy selection is the top-N at the first N where taking the next
    sample would lower S/N = sum/sqrt(N) (the criterion's algebra, checked by explicit
    S/N comparisons rather than the criterion itself)."""
    import itertools
    rng = np.random.default_rng(61)
    for trial in range(40):
        p = np.zeros((3, 4))
        k = int(rng.integers(3, 11))
        cells = rng.choice(12, size=k, replace=False)
        vals = rng.exponential(1.0, size=k) if trial % 3 else rng.integers(1, 4, size=k).astype(float)
        p.ravel()[cells] = vals
        top = sorted(cells, key=lambda c: (-p.ravel()[c], c))
        for r in range(1, k + 1):
            best_r = max(p.ravel()[list(sub)].sum() for sub in itertools.combinations(cells, r))
            assert p.ravel()[top[:r]].sum() == pytest.approx(best_r, rel=1e-12)
        f = [p.ravel()[top[:r]].sum() / math.sqrt(r) for r in range(1, k + 1)]
        n = next((r for r in range(1, k) if not f[r] > f[r - 1]), k)
        mask = ref.select_samples(p)
        assert sorted(np.flatnonzero(mask.ravel())) == sorted(top[:n])


def test_selection_is_optimal_on_pulse_maps():
    """On predicted pulse maps the first S/N peak is the global one: the greedy set
    matches the best prefix (hence the best subset) of the sorted powers."""
    for C, dt, dm, ph in ((60, 1.0, 30.0, 0.0), (122, 1.0, 30.0, 0.3), (244, 2.0, 100.0, 0.7)):
        b = synth.Band(C, 700.0, 300.0 / C, dt)
        P = synth.rect_pulse_cells(b, int(400 / dt), dm, 10.0 + ph * dt, 1.0, 1.0)
        v = np.sort(P[P > 0])[::-1]
        best = max(np.cumsum(v) / np.sqrt(np.arange(1, v.size + 1)))
        assert ref.set_snr(P, ref.select_samples(P)) == pytest.approx(best, rel=1e-12)


def test_selection_takes_every_sample_of_a_flat_map():
    p = np.full((5, 7), 2.5)
    assert ref.select_samples(p).all()
    p[2, 3] = 0.0
    m = ref.select_samples(p)
    assert m.sum() == 34 and not m[2, 3]


def test_selection_gain_peaks_near_twenty_percent_at_nominal_resolution():
    """Sec. 3 (Fig. snr_vs_dt_dv): 700-1000 MHz, 1 ms rectangular pulse, alpha = 0, DM 30,
    no scattering; the selection improves the all-samples S/N by at most ~20 %, at the
    nominal resolution (dnu ~ dnu_0 = 2.46 MHz, dt = tau' = 1 ms)."""
    gains = {}
    for C in (60, 122, 244):
        for dt in (0.5, 1.0, 2.0):
            b = synth.Band(C, 700.0, 300.0 / C, dt)
            P = synth.rect_pulse_cells(b, int(200 / dt), 30.0, 10.0, 1.0, 1.0)
            gains[(C, dt)] = ref.set_snr(P, ref.select_samples(P)) / ref.set_snr(P, P > 0)
    assert max(gains, key=gains.get) == (122, 1.0)
    assert gains[(122, 1.0)] == pytest.approx(1.20, abs=0.02)
    assert all(1.0 <= g <= 1.21 for g in gains.values())


def test_rect_pulse_cells_conserve_fluence():
    """eq. Pavg integrates eq. profile_sb exactly in time: each channel's cells sum to
    p0 tau x (channel width in GHz) / dt for alpha = 0 (the midpoint rule in frequency is
    exact for a constant spectrum), whatever the DM and arrival phase."""
    b = synth.Band(16, 700.0, 18.75, 1.0)
    for dm, t0 in ((0.0, 3.3), (300.0, 5.0), (1500.0, 0.7)):
        P = synth.rect_pulse_cells(b, 20000, dm, t0, 1.0, 2.5, p0=3.0)
        np.testing.assert_allclose(P.sum(axis=1) * b.dt_ms, 3.0 * 1.0 * b.df_mhz / 1000.0, rtol=1e-12)
    # DM 0: the pulse fills [t0, t0 + tau') exactly in every channel
    P = synth.rect_pulse_cells(b, 20, 0.0, 3.25, 1.0, 2.5)
    want = np.array([0, 0, 0, 0.75, 1.0, 0.75] + [0] * 14) * (b.df_mhz / 1000.0) / 2.5
    np.testing.assert_allclose(P, np.tile(want, (16, 1)), atol=1e-15)


# ----------------------------------------------------------------------------- Sec. 5 detectors


def test_detectors_agree_on_a_perfectly_dedispersed_pulse():
    """Sec. 5: with N_S = C N_t and a constant P over the block, every detector gives the
    same S/N (here P = 2 over 6 channels x 4 samples: 2 sqrt(24))."""
    p = np.zeros((6, 10))
    p[:, 3:7] = 2.0
    s = ref.detector_snrs(p, align=np.zeros(6, int))
    for v in s.values():
        assert v == pytest.approx(2.0 * math.sqrt(24.0), rel=1e-12)


def test_detector_ordering_on_pulse_maps():
    """Sec. 5: the dynamic-spectrum matched filter bounds every detector (Cauchy-Schwarz);
    the time-series matched filter beats the time-series boxcar; the sample-selection
    detector beats taking every sample with power, which beats the boxcar (N_S <= C N_t)."""
    for C, dt, dm in ((40, 1.0, 30.0), (122, 1.0, 30.0), (300, 0.5, 100.0), (12, 2.0, 300.0)):
        b = synth.Band(C, 700.0, 300.0 / C, dt)
        P = synth.rect_pulse_cells(b, int(3000 / dt), dm, 20.0, 1.0, 1.0)
        dl, _ = ref.delay_table([dm], C, 700.0, 300.0 / C, dt)
        s = ref.detector_snrs(P, align=dl[0] + 20)
        assert all(s["dsmf"] >= v * (1 - 1e-12) for v in s.values())
        assert s["ts_mf"] >= s["ts_boxcar"]
        assert s["selection"] >= s["all_samples"] >= s["ts_boxcar"]
