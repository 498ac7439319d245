"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

uint8 unit-weight sums must be bit-exact; fp32 sums must satisfy the scale-aware bound
|gpu - oracle| <= 1e-5 * sum_{c,k} |w_dck| |I[c][t+delta+k]| per output (the float64
oracle is exact to far better than that); S/N peaks agree to 1e-5 relative.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import ref
import synth

pytestmark = pytest.mark.gpu

RTOL = 1e-5


@pytest.fixture(scope="module")
def dd():
    import torch
    from paper_1301_3968_gb300 import build
    build.build()
    import paper_1301_3968_gb300 as m
    torch.cuda.set_device(0)
    return m


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _band(dd, b, nsamp, in_type):
    return dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, nsamp, in_type, b.descending)


def _assert_f32_close(got, I, delay, taps, w, t_offset=0, nsamp=None, rows=None):
    want = oracle.c_dedisperse(I, delay, taps, w=w, t_offset=t_offset, nsamp=nsamp, rows=rows)
    scale = oracle.c_abs_scale(I, delay, taps, w=w, t_offset=t_offset, nsamp=nsamp, rows=rows)
    err = np.abs(got.astype(np.float64) - want)
    bad = err > RTOL * scale + 1e-30
    assert not bad.any(), f"{bad.sum()} outputs outside 1e-5 scale; max ratio {(err / np.maximum(scale, 1e-30)).max():.3g}"


# ----------------------------------------------------------------------------- dedispersion


def test_plain_config_bit_exact(dd):
    cfg = synth.make_plain()
    plan = dd.Plan(_band(dd, cfg["band"], cfg["nsamp"], "u8"), cfg["dms"])
    x = _dev(cfg["data"])
    out = plan.dedisperse(x, nsamp=cfg["nsamp"]).cpu().numpy()
    delay, taps = plan.tables()
    assert plan.d_max == 518 and out.shape == (128, 3578)
    want = oracle.c_dedisperse(cfg["data"], delay, taps, nsamp=cfg["nsamp"])
    np.testing.assert_array_equal(out.astype(np.int64), want)


@pytest.mark.parametrize("seed,C,T,D,maxdel,maxtap,t_off", [
    (1, 37, 3001, 21, 300, 9, 0),        # ragged channels, trials and time
    (2, 5, 2500, 9, 40, 45, 13),         # taps above the register window (31)
    (3, 1, 1200, 3, 10, 4, 0),           # one channel
    (4, 64, 1100, 1, 60, 3, 16),         # one trial
    (5, 16, 5000, 17, 4000, 2, 0),       # delays spread far apart (small CTA blocks)
])
def test_u8_random_profiles_bit_exact(dd, seed, C, T, D, maxdel, maxtap, t_off):
    rng = np.random.default_rng(seed)
    ld = (T + t_off + 15) // 16 * 16
    I = np.zeros((C, ld), np.uint8)
    I[:, :T + t_off] = rng.integers(0, 256, size=(C, T + t_off))
    band = dd.Band(C, 1200.0, 1.0, 1.0, T, "u8")
    plan = dd.Plan(band, np.zeros(D))
    delay = rng.integers(0, maxdel + 1, size=(D, C)).astype(np.int32)
    taps = rng.integers(1, maxtap + 1, size=(D, C)).astype(np.int32)
    plan.set_profiles(delay=delay, taps=taps)
    out = plan.dedisperse(_dev(I), t_offset=t_off, nsamp=T).cpu().numpy()
    want = oracle.c_dedisperse(I, delay, taps, t_offset=t_off, nsamp=T)
    np.testing.assert_array_equal(out.astype(np.int64), want)


def test_minimal_output_length(dd):
    """nsamp = d_max + 1 leaves exactly one output per trial."""
    rng = np.random.default_rng(9)
    C, D = 8, 5
    delay = rng.integers(0, 50, size=(D, C)).astype(np.int32)
    taps = rng.integers(1, 6, size=(D, C)).astype(np.int32)
    dmax = int((delay + taps - 1).max())
    T = dmax + 1
    ld = (T + 15) // 16 * 16
    I = np.zeros((C, ld), np.uint8)
    I[:, :T] = rng.integers(0, 256, size=(C, T))
    plan = dd.Plan(dd.Band(C, 1200.0, 1.0, 1.0, T, "u8"), np.zeros(D))
    plan.set_profiles(delay=delay, taps=taps)
    out = plan.dedisperse(_dev(I), nsamp=T).cpu().numpy()
    assert out.shape == (D, 1)
    np.testing.assert_array_equal(out.astype(np.int64), oracle.c_dedisperse(I, delay, taps, nsamp=T))


def test_descending_band_matches_oracle(dd):
    b = synth.Band(48, 700.0, 6.25, 0.5, descending=True)
    rng = np.random.default_rng(10)
    T = 6000
    I = rng.integers(0, 256, size=(48, T)).astype(np.uint8)
    dms = np.linspace(0, 300, 40)
    plan = dd.Plan(_band(dd, b, T, "u8"), dms)
    delay, taps = plan.tables()
    od, _ = ref.delay_table(dms, b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, True)
    np.testing.assert_array_equal(delay, od)
    out = plan.dedisperse(_dev(I), nsamp=T).cpu().numpy()
    np.testing.assert_array_equal(out.astype(np.int64), oracle.c_dedisperse(I, delay, taps, nsamp=T))


def _craft_plan(dd, ndm, nsamp, dm_max=4000.0):
    b = synth.CRAFT_BAND
    band = _band(dd, b, nsamp, "f32")
    dms, eps = dd.trial_dms(band, 0.0, dm_max, ndm, tau_av_ms=1.0)
    plan = dd.Plan(band, dms)
    delay, taps = plan.tables()
    K = int(taps.max())
    wc = synth.spectral_weights(b)
    w = np.zeros((ndm, b.nchan, K), np.float32)
    for k in range(K):
        w[:, :, k] = np.where(k < taps, wc[None, :], 0.0)
    plan.set_profiles(weights=w)
    return plan, delay, taps, w


def test_f32_weighted_reduced_craft(dd):
    """CRAFT band and weights, 512 trials of eq. trial DMs to DM 4000, 8192 samples."""
    cfg = synth.make_craft(nsamp=8192, npulse=4)
    plan, delay, taps, w = _craft_plan(dd, 512, 8192)
    out = plan.dedisperse(_dev(cfg["data"]), nsamp=8192).cpu().numpy()
    assert out.shape[1] == 8192 - plan.d_max
    _assert_f32_close(out, cfg["data"], delay, taps, w, nsamp=8192)


def test_f32_full_craft_sampled_rows(dd):
    """Full CRAFT-like size (336 x 65536, 4096 trials) in the benchmark's launch shape;
    32 sampled trial rows, including the first and the last, against the oracle."""
    cfg = synth.make_craft()
    plan, delay, taps, w = _craft_plan(dd, 4096, 65536)
    out = plan.dedisperse(_dev(cfg["data"]), nsamp=65536).cpu().numpy()
    rows = sorted(set([0, 1, 4095, 4094] + list(np.random.default_rng(3).integers(0, 4096, 28))))
    _assert_f32_close(out[rows], cfg["data"], delay, taps, w, nsamp=65536, rows=rows)


def test_f32_unit_and_random_weights(dd):
    rng = np.random.default_rng(12)
    C, T, D, K = 29, 4100, 19, 37
    I = rng.standard_normal((C, 4112)).astype(np.float32) * 3 + 1
    delay = rng.integers(0, 200, size=(D, C)).astype(np.int32)
    taps = rng.integers(1, K + 1, size=(D, C)).astype(np.int32)
    plan = dd.Plan(dd.Band(C, 1200.0, 1.0, 1.0, T, "f32"), np.zeros(D))
    plan.set_profiles(delay=delay, taps=taps)
    out = plan.dedisperse(_dev(I), nsamp=T).cpu().numpy()
    _assert_f32_close(out, I, delay, taps, None, nsamp=T)
    w = rng.standard_normal((D, C, K)).astype(np.float32)
    plan.set_profiles(delay=delay, taps=taps, weights=w)
    out = plan.dedisperse(_dev(I), t_offset=3, nsamp=T).cpu().numpy()
    _assert_f32_close(out, I, delay, taps, w, t_offset=3, nsamp=T)


@pytest.mark.parametrize("kmax,maxdel", [(23, 3), (23, 300), (70, 5), (70, 400)])
def test_f32_pair_windows_all_tap_passes(dd, kmax, maxdel):
    """Pair units whose two trials start apart (both signs) and have different tap counts,
    on every tap-pass form: one unrolled pass (<= 27 taps), two (<= 54) and the loop (more).
    Small delay spreads give the common shifts of 0-3 samples, large ones long shifts and
    runs that read far past the shorter trial's own taps (with zero weight)."""
    rng = np.random.default_rng(kmax * 1000 + maxdel)
    C, T, D = 23, 3100, 21
    I = (rng.standard_normal((C, 3104)) * 2 - 0.5).astype(np.float32)
    delay = rng.integers(0, maxdel + 1, size=(D, C)).astype(np.int32)
    taps = rng.integers(1, kmax + 1, size=(D, C)).astype(np.int32)
    w = rng.uniform(-1.0, 1.5, size=(D, C, kmax)).astype(np.float32)
    plan = dd.Plan(dd.Band(C, 1200.0, 1.0, 1.0, T, "f32"), np.zeros(D))
    plan.set_profiles(delay=delay, taps=taps, weights=w)
    out = plan.dedisperse(_dev(I), t_offset=2, nsamp=T).cpu().numpy()
    _assert_f32_close(out, I, delay, taps, w, t_offset=2, nsamp=T)
    assert plan.device_status() == 0


def test_u8_input_with_weights(dd):
    rng = np.random.default_rng(13)
    C, T, D, K = 20, 3000, 12, 7
    I = np.zeros((C, 3008), np.uint8)
    I[:, :T] = rng.integers(0, 256, size=(C, T))
    delay = rng.integers(0, 100, size=(D, C)).astype(np.int32)
    taps = rng.integers(1, K + 1, size=(D, C)).astype(np.int32)
    w = rng.uniform(0, 2, size=(D, C, K)).astype(np.float32)
    plan = dd.Plan(dd.Band(C, 1200.0, 1.0, 1.0, T, "u8"), np.zeros(D))
    plan.set_profiles(delay=delay, taps=taps, weights=w)
    out = plan.dedisperse(_dev(I), nsamp=T)
    assert out.dtype.is_floating_point
    _assert_f32_close(out.cpu().numpy(), I.astype(np.float32), delay, taps, w, nsamp=T)


def test_streaming_chunks_equal_one_shot(dd):
    """Chunks of L outputs (input windows [t0, t0 + L + d_max)) concatenate exactly."""
    cfg = synth.make_plain(nsamp=8192)
    plan = dd.Plan(_band(dd, cfg["band"], 8192, "u8"), cfg["dms"])
    x = _dev(cfg["data"])
    full = plan.dedisperse(x, nsamp=8192).cpu().numpy()
    L = 1000
    parts = []
    t0 = 0
    while t0 < full.shape[1]:
        n = min(L, full.shape[1] - t0)
        parts.append(plan.dedisperse(x, t_offset=t0, nsamp=n + plan.d_max).cpu().numpy())
        t0 += n
    np.testing.assert_array_equal(np.concatenate(parts, axis=1), full)


# ----------------------------------------------------------------------------- statistics


def test_channel_stats(dd):
    cfg = synth.make_plain()
    plan = dd.Plan(_band(dd, cfg["band"], cfg["nsamp"], "u8"), cfg["dms"])
    m, s = plan.channel_stats(_dev(cfg["data"]), t_offset=5, nsamp=4000)
    om, osd = ref.channel_stats(cfg["data"], t_offset=5, nsamp=4000)
    np.testing.assert_allclose(m.cpu().numpy(), om, rtol=1e-12)
    np.testing.assert_allclose(s.cpu().numpy(), osd, rtol=1e-9)
    rng = np.random.default_rng(14)
    If = (rng.standard_normal((7, 10000)) * 2 + 1000).astype(np.float32)
    plan2 = dd.Plan(dd.Band(7, 1200.0, 1.0, 1.0, 10000, "f32"), [0.0])
    m, s = plan2.channel_stats(_dev(If))
    om, osd = ref.channel_stats(If)
    np.testing.assert_allclose(m.cpu().numpy(), om, rtol=1e-12)
    np.testing.assert_allclose(s.cpu().numpy(), osd, rtol=1e-9)


def _boxcar_compare(peak, arg, x, widths, mu, sd, snr_rtol=RTOL):
    opeak, oarg, obest = ref.boxcar_snr(x, widths, mu, sd)
    np.testing.assert_allclose(peak, opeak, rtol=snr_rtol, atol=snr_rtol)
    # the earliest maximum; near-ties (S/N within 1e-5) may pick either time
    mism = arg != oarg
    for d, j in zip(*np.nonzero(mism)):
        B = ref.boxcar_series(x[d], int(widths[j]))
        assert abs(B[arg[d, j]] - B[oarg[d, j]]) <= 1e-5 * max(abs(B[oarg[d, j]]), sd[d, j])


def test_boxcar_plain_integer(dd):
    cfg = synth.make_plain()
    plan = dd.Plan(_band(dd, cfg["band"], cfg["nsamp"], "u8"), cfg["dms"])
    x = _dev(cfg["data"])
    out = plan.dedisperse(x, nsamp=cfg["nsamp"])
    mean, sd = plan.channel_stats(x, nsamp=cfg["nsamp"])
    widths = np.array([1, 2, 3, 5, 8, 13, 21, 34, 55, 89, 144, 233, 377], np.int32)
    peak, arg, _ = plan.boxcar_snr(out, widths, mean, sd)
    delay, taps = plan.tables()
    xo = out.cpu().numpy().astype(np.int64)
    mu_c, sd_c = ref.channel_stats(cfg["data"], nsamp=cfg["nsamp"])
    mu, sdw = ref.boxcar_norm(taps, widths, mu_c, sd_c)
    _, oarg, _ = ref.boxcar_snr(xo, widths, mu, sdw)
    np.testing.assert_array_equal(arg.cpu().numpy(), oarg)        # integer sums: exact
    _boxcar_compare(peak.cpu().numpy(), arg.cpu().numpy(), xo, widths, mu, sdw)


def test_boxcar_all_widths_int64_path(dd):
    """256 widths on long rows of large values select the int64 boxcar sums."""
    rng = np.random.default_rng(15)
    C, T, D = 64, 20000, 6
    I = rng.integers(100, 256, size=(C, T)).astype(np.uint8)
    delay = rng.integers(0, 500, size=(D, C)).astype(np.int32)
    taps = np.full((D, C), 600, np.int32)                 # 256 * 255 * 38400 > 2^31
    plan = dd.Plan(dd.Band(C, 1200.0, 1.0, 1.0, T, "u8"), np.zeros(D))
    plan.set_profiles(delay=delay, taps=taps)
    x = _dev(I)
    out = plan.dedisperse(x, nsamp=T)
    mean, sd = plan.channel_stats(x, nsamp=T)
    widths = np.arange(1, 257, dtype=np.int32)
    peak, arg, _ = plan.boxcar_snr(out, widths, mean, sd)
    xo = out.cpu().numpy().astype(np.int64)
    np.testing.assert_array_equal(xo, oracle.c_dedisperse(I, delay, taps, nsamp=T))
    mu_c, sd_c = ref.channel_stats(I, nsamp=T)
    mu, sdw = ref.boxcar_norm(taps, widths, mu_c, sd_c)
    _, oarg, _ = ref.boxcar_snr(xo, widths, mu, sdw)
    np.testing.assert_array_equal(arg.cpu().numpy(), oarg)
    _boxcar_compare(peak.cpu().numpy(), arg.cpu().numpy(), xo, widths, mu, sdw)


def test_boxcar_int64_rows_split(dd):
    """Rows whose boxcar sums exceed int32 (a bright half, long tap runs) take the int64
    scan, the others the int32 scan, in one call; both exact against the oracle."""
    C, T, D = 64, 20000, 6
    I = np.zeros((C, T), np.uint8)
    I[:, : T // 2] = 255
    rng = np.random.default_rng(16)
    I[:, T // 2:] = rng.integers(0, 3, size=(C, T - T // 2))
    delay = rng.integers(0, 300, size=(D, C)).astype(np.int32)
    taps = np.full((D, C), 1200, np.int32)
    taps[3:] = 10                                   # these rows stay within int32
    plan = dd.Plan(dd.Band(C, 1200.0, 1.0, 1.0, T, "u8"), np.zeros(D))
    plan.set_profiles(delay=delay, taps=taps)
    plan.set_method("direct")
    x = _dev(I)
    out = plan.dedisperse(x, nsamp=T)
    mean, sd = plan.channel_stats(x, nsamp=T)
    widths = np.arange(1, 257, dtype=np.int32)
    peak, arg, _ = plan.boxcar_snr(out, widths, mean, sd)
    xo = out.cpu().numpy().astype(np.int64)
    np.testing.assert_array_equal(xo, oracle.c_dedisperse(I, delay, taps, nsamp=T))
    mu_c, sd_c = ref.channel_stats(I, nsamp=T)
    mu, sdw = ref.boxcar_norm(taps, widths, mu_c, sd_c)
    _, oarg, _ = ref.boxcar_snr(xo, widths, mu, sdw)
    np.testing.assert_array_equal(arg.cpu().numpy(), oarg)
    _boxcar_compare(peak.cpu().numpy(), arg.cpu().numpy(), xo, widths, mu, sdw)
    # the wide rows really exceed int32 and the narrow ones do not
    o = np.rint((mu[:, 0]))
    assert (np.abs(xo[:3] - o[:3, None]).max(axis=1) * 256 > 2**31).all()
    assert (np.abs(xo[3:] - o[3:, None]).max(axis=1) * 256 < 2**31).all()


def test_boxcar_weighted_float(dd):
    cfg = synth.make_craft(nsamp=8192, npulse=6, amp=3.0)
    plan, delay, taps, w = _craft_plan(dd, 256, 8192)
    x = _dev(cfg["data"])
    out = plan.dedisperse(x, nsamp=8192)
    mean, sd = plan.channel_stats(x, nsamp=8192)
    widths = np.arange(1, 33, dtype=np.int32)
    peak, arg, _ = plan.boxcar_snr(out, widths, mean, sd)
    xo = out.cpu().numpy().astype(np.float64)              # same series on both sides
    mu_c, sd_c = ref.channel_stats(cfg["data"], nsamp=8192)
    mu, sdw = ref.boxcar_norm(taps, widths, mu_c, sd_c, w=w)
    _boxcar_compare(peak.cpu().numpy(), arg.cpu().numpy(), xo, widths, mu, sdw)


@pytest.mark.parametrize("seed,T,w0,nw,trim", [
    (21, 30000, 5, 20, 7),       # several chunks, a ragged second width group
    (22, 17008, 1, 16, 0),       # one full group, chunk boundary tails
    (23, 3008, 30, 3, 2000),     # shorter than one chunk, series cut short
])
def test_boxcar_contiguous_widths_int(dd, seed, T, w0, nw, trim):
    """Contiguous width lists (the prefix-window kernel) on integer series: arg exact,
    including widths not starting at 1, a ragged last group and a cut-short series."""
    rng = np.random.default_rng(seed)
    C, D = 32, 8
    I = rng.integers(0, 256, size=(C, T)).astype(np.uint8)
    I[:, T // 3:T // 3 + 40] = 255                       # a broad dispersion-free pulse
    delay = rng.integers(0, 200, size=(D, C)).astype(np.int32)
    delay[0] = 0
    taps = rng.integers(1, 5, size=(D, C)).astype(np.int32)
    plan = dd.Plan(dd.Band(C, 1200.0, 1.0, 1.0, T, "u8"), np.zeros(D))
    plan.set_profiles(delay=delay, taps=taps)
    x = _dev(I)
    out = plan.dedisperse(x, nsamp=T)
    t_len = out.shape[1] - trim
    mean, sd = plan.channel_stats(x, nsamp=T)
    widths = np.arange(w0, w0 + nw, dtype=np.int32)
    peak, arg, _ = plan.boxcar_snr(out, widths, mean, sd, t_len=t_len)
    xo = out.cpu().numpy().astype(np.int64)[:, :t_len]
    mu_c, sd_c = ref.channel_stats(I, nsamp=T)
    mu, sdw = ref.boxcar_norm(taps, widths, mu_c, sd_c)
    _, oarg, _ = ref.boxcar_snr(xo, widths, mu, sdw)
    np.testing.assert_array_equal(arg.cpu().numpy(), oarg)
    _boxcar_compare(peak.cpu().numpy(), arg.cpu().numpy(), xo, widths, mu, sdw)


def test_boxcar_contiguous_widths_float(dd):
    cfg = synth.make_craft(nsamp=8192, npulse=6, amp=3.0)
    plan, delay, taps, w = _craft_plan(dd, 128, 8192)
    x = _dev(cfg["data"])
    out = plan.dedisperse(x, nsamp=8192)
    t_len = out.shape[1] - 333
    mean, sd = plan.channel_stats(x, nsamp=8192)
    widths = np.arange(3, 43, dtype=np.int32)
    peak, arg, _ = plan.boxcar_snr(out, widths, mean, sd, t_len=t_len)
    xo = out.cpu().numpy().astype(np.float64)[:, :t_len]
    mu_c, sd_c = ref.channel_stats(cfg["data"], nsamp=8192)
    mu, sdw = ref.boxcar_norm(taps, widths, mu_c, sd_c, w=w)
    _boxcar_compare(peak.cpu().numpy(), arg.cpu().numpy(), xo, widths, mu, sdw)
    # the contiguous and the general kernel agree: drop one width to force the latter
    gen = np.concatenate([widths[:5], widths[6:]])
    p2, a2, _ = plan.boxcar_snr(out, gen, mean, sd, t_len=t_len)
    keep = np.r_[0:5, 6:len(widths)]
    np.testing.assert_allclose(p2.cpu().numpy(), peak.cpu().numpy()[:, keep], rtol=RTOL, atol=RTOL)


def test_candidates_above_threshold(dd):
    cfg = synth.make_plain(snr_total=16.0)
    plan = dd.Plan(_band(dd, cfg["band"], cfg["nsamp"], "u8"), cfg["dms"])
    x = _dev(cfg["data"])
    out = plan.dedisperse(x, nsamp=cfg["nsamp"])
    mean, sd = plan.channel_stats(x, nsamp=cfg["nsamp"])
    widths = np.arange(1, 9, dtype=np.int32)
    peak, arg, cands = plan.boxcar_snr(out, widths, mean, sd, thresh=7.0, cap=4096)
    got = sorted((d, j, t) for d, j, t, _ in dd.candidates_to_list(cands))
    p = peak.cpu().numpy()
    a = arg.cpu().numpy()
    want = sorted((int(d), int(j), int(a[d, j])) for d, j in zip(*np.nonzero(p > 7.0)))
    assert got == want and len(want) > 0
    # capacity overflow: the count keeps going, the buffer keeps the first `cap`
    _, _, small = plan.boxcar_snr(out, widths, mean, sd, thresh=7.0, cap=2)
    assert int(small[1].item()) == len(want)
    assert len(dd.candidates_to_list(small)) == min(2, len(want))
    # the 16σ pulse peaks at trial 76 (DM 299.2) near sample 1000
    d_best, j_best = np.unravel_index(np.argmax(p), p.shape)
    assert d_best == 76 and abs(a[d_best, j_best] - 1000) <= 2


# ----------------------------------------------------------------------------- adjoint


def _diff_problem(dd, seed=16, C=24, T=3000, D=10, K=12):
    rng = np.random.default_rng(seed)
    I = rng.standard_normal((C, T)).astype(np.float32)
    delay = rng.integers(0, 300, size=(D, C)).astype(np.int32)
    taps = rng.integers(1, K + 1, size=(D, C)).astype(np.int32)
    w = rng.standard_normal((D, C, K)).astype(np.float32)
    plan = dd.Plan(dd.Band(C, 1200.0, 1.0, 1.0, T, "f32"), np.zeros(D))
    plan.set_profiles(delay=delay, taps=taps, weights=w)
    return rng, I, delay, taps, w, plan


def test_backward_matches_oracle(dd):
    rng, I, delay, taps, w, plan = _diff_problem(dd)
    t_out = I.shape[1] - plan.d_max
    g = rng.standard_normal((w.shape[0], t_out)).astype(np.float32)
    gw, gI = plan.backward(_dev(I), _dev(g))
    ogw, ogI = oracle.c_adjoint(I, g, delay, taps, w)
    # scale-aware: each entry is a sum of products; bound by the sum of |products|
    sgw, sgI = oracle.c_adjoint(np.abs(I), np.abs(g), delay, taps, np.abs(w))
    assert (np.abs(gw.cpu().numpy() - ogw) <= RTOL * sgw + 1e-30).all()
    assert (np.abs(gI.cpu().numpy() - ogI) <= RTOL * sgI + 1e-30).all()


def test_adjoint_dot_product(dd):
    rng, I, delay, taps, w, plan = _diff_problem(dd, seed=17)
    x = _dev(I)
    out = plan.dedisperse(x).cpu().numpy().astype(np.float64)
    g = rng.standard_normal(out.shape).astype(np.float32)
    gw, gI = plan.backward(x, _dev(g))
    lhs = float((out * g).sum())
    r1 = float((I.astype(np.float64) * gI.cpu().numpy()).sum())
    wm = w.copy()
    for k in range(w.shape[2]):
        wm[:, :, k] *= k < taps
    r2 = float((wm.astype(np.float64) * gw.cpu().numpy()).sum())
    scale = float((np.abs(out) * np.abs(g)).sum())
    assert abs(lhs - r1) <= 1e-5 * scale
    assert abs(lhs - r2) <= 1e-5 * scale


def test_autograd_matches_finite_differences(dd):
    """J = mean_p (x_{d_p}[t_p] − μ_p)/σ_p through DDFunction; ∂J/∂w and ∂J/∂I against
    central differences of the float64 oracle at 64 random weights and 64 inputs."""
    import torch
    rng, I, delay, taps, w, plan = _diff_problem(dd, seed=18, C=12, T=900, D=6, K=8)
    D, C, K = w.shape
    t_out = I.shape[1] - plan.d_max
    pts = [(int(rng.integers(D)), int(rng.integers(t_out))) for _ in range(8)]
    sig_c = np.ones(C)

    def J_oracle(Iv, wv):
        x = ref.dedisperse(Iv, delay, taps, w=wv)
        vals = []
        for d, t in pts:
            wm = np.array([[wv[d, c, k] if k < taps[d, c] else 0.0 for k in range(K)] for c in range(C)],
                          np.float64)
            s = math.sqrt(float((sig_c[:, None] ** 2 * wm ** 2).sum()))
            vals.append(x[d, t] / s)
        return float(np.mean(vals))

    xt = _dev(I).requires_grad_(True)
    wt = _dev(w).requires_grad_(True)
    mask = torch.from_numpy((np.arange(K)[None, None, :] < taps[:, :, None]).astype(np.float32)).cuda()
    out = dd.DDFunction.apply(xt, wt, plan)
    dsel = torch.tensor([p[0] for p in pts], device="cuda")
    tsel = torch.tensor([p[1] for p in pts], device="cuda")
    sig = torch.sqrt(((wt * mask) ** 2).sum(dim=(1, 2)))[dsel]
    J = (out[dsel, tsel] / sig).mean()
    J.backward()
    gw = wt.grad.cpu().numpy()
    gI = xt.grad.cpu().numpy()
    Iw = I.astype(np.float64)
    w64 = w.astype(np.float64)
    for _ in range(64):
        d, c = int(rng.integers(D)), int(rng.integers(C))
        k = int(rng.integers(taps[d, c]))
        h = 1e-3 * max(abs(w64[d, c, k]), 1.0)
        wp, wm_ = w64.copy(), w64.copy()
        wp[d, c, k] += h
        wm_[d, c, k] -= h
        fd = (J_oracle(Iw, wp) - J_oracle(Iw, wm_)) / (2 * h)
        assert gw[d, c, k] == pytest.approx(fd, rel=1e-3, abs=1e-5)
    for _ in range(64):
        c, t = int(rng.integers(C)), int(rng.integers(I.shape[1]))
        h = 1e-3 * max(abs(Iw[c, t]), 1.0)
        Ip, Im = Iw.copy(), Iw.copy()
        Ip[c, t] += h
        Im[c, t] -= h
        fd = (J_oracle(Ip, w64) - J_oracle(Im, w64)) / (2 * h)
        assert gI[c, t] == pytest.approx(fd, rel=1e-3, abs=1e-5)


def test_backward_differentiable_band_sampled(dd):
    """Differentiable-config shape at reduced size: CRAFT band, 32 learnable taps per
    channel on every trial, eq. trial DMs to 2000, against the float64 oracle."""
    rng = np.random.default_rng(19)
    b = synth.CRAFT_BAND
    T, D, K = 6144, 64, 32
    band = dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, T, "f32")
    dms, _ = dd.trial_dms(band, 0.0, 2000.0, D, tau_av_ms=1.0)
    plan = dd.Plan(band, dms)
    delay, taps0 = plan.tables()
    taps = np.full_like(taps0, K)
    w = (rng.uniform(0.5, 1.5, size=(D, b.nchan, K)) * (np.arange(K)[None, None, :] < taps0[:, :, None])).astype(np.float32)
    plan.set_profiles(delay=delay, taps=taps, weights=w)
    I = rng.standard_normal((b.nchan, T)).astype(np.float32)
    t_out = T - plan.d_max
    g = rng.standard_normal((D, t_out)).astype(np.float32)
    gw, gI = plan.backward(_dev(I), _dev(g))
    ogw, ogI = oracle.c_adjoint(I, g, delay, taps, w)
    sgw, sgI = oracle.c_adjoint(np.abs(I), np.abs(g), delay, taps, np.abs(w))
    assert (np.abs(gw.cpu().numpy() - ogw) <= RTOL * sgw + 1e-30).all()
    assert (np.abs(gI.cpu().numpy() - ogI) <= RTOL * sgI + 1e-30).all()
    # device weights (the training path) give the same gradients
    plan2 = dd.Plan(band, dms)
    plan2.set_profiles(delay=delay, taps=taps, weights=np.ones_like(w))
    plan2.set_weights(_dev(w))
    gw2, gI2 = plan2.backward(_dev(I), _dev(g))
    np.testing.assert_array_equal(gw2.cpu().numpy(), gw.cpu().numpy())
    np.testing.assert_array_equal(gI2.cpu().numpy(), gI.cpu().numpy())
