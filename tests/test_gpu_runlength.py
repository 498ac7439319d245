"""Run-length tap sums (prefix-sum differences, uint8 unit weights) through the C ABI:
bit-exact against the oracle's brute-force sums and against the direct path, in
streamed chunks, and on the large low-band configuration at reduced length."""
import numpy as np
import pytest

import oracle
from oracle import ref
import synth

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("seed,C,T,D,maxdel,maxtap,t_off", [
    (41, 37, 5008, 29, 900, 300, 0),     # ragged channels, trials (24 per CTA) and time
    (42, 5, 3000, 50, 40, 1, 16),        # single taps
    (43, 64, 2400, 24, 10, 1500, 13),    # runs longer than the staged tile
    (44, 1, 1500, 3, 0, 700, 0),         # one channel, zero delays
])
def test_runlength_bit_exact(dd, seed, C, T, D, maxdel, maxtap, t_off):
    rng = np.random.default_rng(seed)
    ld = (T + t_off + 15) // 16 * 16
    I = np.zeros((C, ld), np.uint8)
    I[:, :T + t_off] = rng.integers(0, 256, size=(C, T + t_off))
    plan = dd.Plan(dd.Band(C, 1200.0, 1.0, 1.0, T, "u8"), np.zeros(D))
    delay = rng.integers(0, maxdel + 1, size=(D, C)).astype(np.int32)
    taps = rng.integers(1, maxtap + 1, size=(D, C)).astype(np.int32)
    plan.set_profiles(delay=delay, taps=taps)
    plan.set_method("runlength")
    assert plan.method == "runlength"
    out = plan.dedisperse(_dev(I), t_offset=t_off, nsamp=T).cpu().numpy()
    want = oracle.c_dedisperse(I, delay, taps, t_offset=t_off, nsamp=T)
    np.testing.assert_array_equal(out.astype(np.int64), want)


def test_runlength_equals_direct_plain(dd):
    cfg = synth.make_plain()
    b = cfg["band"]
    plan = dd.Plan(dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, cfg["nsamp"], "u8"), cfg["dms"])
    x = _dev(cfg["data"])
    assert plan.method == "direct"
    direct = plan.dedisperse(x, nsamp=cfg["nsamp"]).cpu().numpy()
    plan.set_method("runlength")
    rl = plan.dedisperse(x, nsamp=cfg["nsamp"]).cpu().numpy()
    np.testing.assert_array_equal(rl, direct)


def test_runlength_streamed_chunks(dd):
    """Overlapping chunks (t_offset advancing by the chunk's output length) reproduce the
    one-shot sums; the prefix scratch is rebuilt for every chunk."""
    import torch
    rng = np.random.default_rng(45)
    C, T, D = 48, 12000, 30
    I = rng.integers(0, 256, size=(C, T)).astype(np.uint8)
    plan = dd.Plan(dd.Band(C, 1200.0, 1.0, 1.0, T, "u8"), np.zeros(D))
    delay = rng.integers(0, 1500, size=(D, C)).astype(np.int32)
    taps = rng.integers(20, 120, size=(D, C)).astype(np.int32)
    plan.set_profiles(delay=delay, taps=taps)
    assert plan.method == "runlength"                    # automatic: mean taps >= 12
    x = _dev(I)
    full = plan.dedisperse(x, nsamp=T).cpu().numpy()
    dmax = plan.d_max
    L = 2500
    parts = []
    for t0 in range(0, T - dmax, L):
        n = min(L, T - dmax - t0) + dmax
        parts.append(plan.dedisperse(x, t_offset=t0, nsamp=n).cpu().numpy())
    np.testing.assert_array_equal(np.concatenate(parts, axis=1), full)
    rows = [0, D // 2, D - 1]
    want = oracle.c_dedisperse(I, delay, taps, nsamp=T, rows=rows)
    np.testing.assert_array_equal(full[rows].astype(np.int64), want)


def test_large_lowband_reduced_sampled(dd):
    """Large low-band band and trial list (1024 ch over 700-1000 MHz, dt 64 us, 8192 DMs
    to 2000) on 2^18 samples: sampled trials against the oracle, bit-exact; boxcar S/N over
    widths 1-256 on those trials against the oracle's; the strongest pulse is found near
    its DM."""
    import torch
    cfg = synth.make_large(nsamp=1 << 18)
    b = cfg["band"]
    T = cfg["nsamp"]
    plan = dd.Plan(dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, T, "u8"), cfg["dms"])
    assert plan.method == "runlength"
    x = _dev(cfg["data"])
    out = plan.dedisperse(x, nsamp=T)
    delay, taps = plan.tables()
    rng = np.random.default_rng(46)
    rows = sorted(set([0, 8191] + rng.integers(0, 8192, size=10).tolist()))
    got = out[rows].cpu().numpy().astype(np.int64)
    want = oracle.c_dedisperse(cfg["data"], delay, taps, nsamp=T, rows=rows)
    np.testing.assert_array_equal(got, want)
    mean, sd = plan.channel_stats(x, nsamp=T)
    widths = np.arange(1, 257, dtype=np.int32)
    peak, arg, _ = plan.boxcar_snr(out, widths, mean, sd)
    mu_c, sd_c = ref.channel_stats(cfg["data"], nsamp=T)
    mu, sdw = ref.boxcar_norm(taps[rows], widths, mu_c, sd_c)
    opeak, oarg, _ = ref.boxcar_snr(want, widths, mu, sdw)
    np.testing.assert_array_equal(arg.cpu().numpy()[rows], oarg)
    np.testing.assert_allclose(peak.cpu().numpy()[rows], opeak, rtol=1e-5, atol=1e-5)
    # the best detection lies on a pulse that arrives inside the output span
    t_out = T - plan.d_max
    p = peak.cpu().numpy()
    d_best = int(np.unravel_index(np.argmax(p), p.shape)[0])
    inside = [q for q in cfg["pulses"] if q["t0_ms"] / b.dt_ms < t_out]
    assert min(abs(cfg["dms"][d_best] - q["dm"]) for q in inside) < 5.0


def test_runlength_shared_difference_rows_bit_exact(dd):
    """Tap counts with at most two values per block of 24 trials and channel let the CTA
    share difference rows; ragged trial blocks, random delays, streamed offsets."""
    rng = np.random.default_rng(47)
    C, T, D = 33, 6000, 50
    I = rng.integers(0, 256, size=(C, T + 16)).astype(np.uint8)
    delay = rng.integers(0, 700, size=(D, C)).astype(np.int32)
    taps = np.zeros((D, C), np.int32)
    for b0 in range(0, D, 24):
        for c in range(C):
            pair = rng.integers(1, 400, size=2)
            taps[b0:b0 + 24, c] = rng.choice(pair, size=min(24, D - b0))
    plan = dd.Plan(dd.Band(C, 1200.0, 1.0, 1.0, T, "u8"), np.zeros(D))
    plan.set_profiles(delay=delay, taps=taps)
    plan.set_method("runlength")
    assert plan.schedule()["trials_per_cta"] == 24
    x = _dev(I)
    out = plan.dedisperse(x, t_offset=16, nsamp=T).cpu().numpy()
    want = oracle.c_dedisperse(I, delay, taps, t_offset=16, nsamp=T)
    np.testing.assert_array_equal(out.astype(np.int64), want)
    plan.set_method("direct")
    np.testing.assert_array_equal(plan.dedisperse(x, t_offset=16, nsamp=T).cpu().numpy(), out)
