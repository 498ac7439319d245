"""Dedispersion fused with the boxcar S/N (dd_dedisperse_boxcar) through the C ABI: the
same peak S/N (bit for bit) and earliest start as dd_dedisperse followed by dd_boxcar_snr,
on both integer tap-sum methods and on fp32 plans (fp32 and weighted uint8 input), across
part counts (part boundaries inside and between trial blocks, seams), ragged tiles,
offsets, CTA shapes and width ranges (with and without the pruned wide groups, up to the
largest carry a tile holds); against the oracle's dedispersion and boxcar scan; the large
low-band configuration at reduced length, the CRAFT-like band at reduced size; and the
overflow status."""
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


def _plan(dd, rng, C, T, D, maxdel, maxtap, method):
    plan = dd.Plan(dd.Band(C, 1200.0, 1.0, 1.0, T, "u8"), np.zeros(D))
    delay = rng.integers(0, maxdel + 1, size=(D, C)).astype(np.int32)
    taps = rng.integers(1, maxtap + 1, size=(D, C)).astype(np.int32)
    plan.set_profiles(delay=delay, taps=taps)
    plan.set_method(method)
    return plan, delay, taps


def _unfused(plan, x, widths, mean, sd, t_offset, nsamp, thresh=None, cap=0):
    out = plan.dedisperse(x, t_offset=t_offset, nsamp=nsamp)
    return plan.boxcar_snr(out, widths, mean, sd, thresh=thresh, cap=cap)


@pytest.mark.parametrize("method", ["direct", "runlength"])
@pytest.mark.parametrize("seed,C,T,D,maxdel,maxtap,t_off,w0,w1,parts", [
    (61, 24, 5000, 30, 300, 20, 0, 1, 32, 0),       # automatic parts
    (62, 37, 7100, 27, 900, 60, 16, 1, 256, 3),     # parts end inside blocks, ragged last tile
    (63, 16, 4200, 9, 100, 5, 0, 5, 40, 1000),      # one tile per part: a seam at every tile
    (64, 12, 3300, 25, 50, 3, 32, 1, 1, 2),         # width 1 only: no carry
    (65, 40, 9000, 50, 2000, 200, 0, 100, 160, 7),  # long runs, widths 100-160 (pruned groups)
    (69, 30, 12000, 60, 500, 40, 0, 1, 300, 11),    # widths 1-300: a partial last group
])
def test_fused_equals_unfused(dd, method, seed, C, T, D, maxdel, maxtap, t_off, w0, w1, parts):
    rng = np.random.default_rng(seed)
    ld = (T + t_off + 15) // 16 * 16
    I = np.zeros((C, ld), np.uint8)
    I[:, :T + t_off] = np.clip(rng.normal(128, 20, size=(C, T + t_off)), 0, 255).astype(np.uint8)
    plan, delay, taps = _plan(dd, rng, C, T, D, maxdel, maxtap, method)
    x = _dev(I)
    mean, sd = plan.channel_stats(x, t_offset=t_off, nsamp=T)
    widths = np.arange(w0, w1 + 1, dtype=np.int32)
    plan.test_set_fused_parts(parts)
    p0, a0, _ = _unfused(plan, x, widths, mean, sd, t_off, T)
    p1, a1, _ = plan.dedisperse_boxcar(x, widths, mean, sd, t_offset=t_off, nsamp=T)
    assert plan.device_status() == 0
    np.testing.assert_array_equal(a1.cpu().numpy(), a0.cpu().numpy())
    np.testing.assert_array_equal(p1.cpu().numpy(), p0.cpu().numpy())


@pytest.mark.parametrize("method,nch", [("direct", 2), ("runlength", 2), ("direct", 4)])
def test_fused_multi_chunk_ctas(dd, method, nch):
    """CTA shapes with several time chunks (a trial's row is written by nch warps and
    scanned by all of them): fused = unfused."""
    rng = np.random.default_rng(70 + nch)
    C, T, D = 20, 9008, 40
    I = np.clip(rng.normal(128, 20, size=(C, T)), 0, 255).astype(np.uint8)
    plan, _, _ = _plan(dd, rng, C, T, D, 600, 50, method)
    plan.set_schedule(nch, 2)
    assert plan.schedule()["nch"] == nch
    x = _dev(I)
    mean, sd = plan.channel_stats(x, nsamp=T)
    widths = np.arange(1, 200, dtype=np.int32)
    for parts in (0, 5):
        plan.test_set_fused_parts(parts)
        p0, a0, _ = _unfused(plan, x, widths, mean, sd, 0, T)
        p1, a1, _ = plan.dedisperse_boxcar(x, widths, mean, sd, nsamp=T)
        assert plan.device_status() == 0
        np.testing.assert_array_equal(a1.cpu().numpy(), a0.cpu().numpy())
        np.testing.assert_array_equal(p1.cpu().numpy(), p0.cpu().numpy())


@pytest.mark.parametrize("method", ["direct", "runlength"])
def test_fused_against_oracle(dd, method):
    """A pulse on noise: the oracle's dedispersion and boxcar scan (int64 sums, float64
    S/N) give the same earliest starts and S/N within 1e-5."""
    rng = np.random.default_rng(66)
    C, T, D = 32, 6000, 20
    I = np.clip(rng.normal(100, 15, size=(C, T)), 0, 255).astype(np.uint8)
    plan, delay, taps = _plan(dd, rng, C, T, D, 400, 40, method)
    for c in range(C):  # a bright run along trial 7's profile
        s = 2500 + delay[7, c]
        I[c, s:s + taps[7, c]] = np.minimum(255, I[c, s:s + taps[7, c]].astype(int) + 60)
    x = _dev(I)
    mean, sd = plan.channel_stats(x, nsamp=T)
    widths = np.arange(1, 65, dtype=np.int32)
    plan.test_set_fused_parts(3)
    peak, arg, _ = plan.dedisperse_boxcar(x, widths, mean, sd, nsamp=T)
    xo = oracle.c_dedisperse(I, delay, taps, nsamp=T)
    mu, sdw = ref.boxcar_norm(taps, widths, *ref.channel_stats(I, nsamp=T))
    opeak, oarg, _ = ref.boxcar_snr(xo, widths, mu, sdw)
    np.testing.assert_array_equal(arg.cpu().numpy(), oarg)
    np.testing.assert_allclose(peak.cpu().numpy(), opeak, rtol=1e-5, atol=1e-5)
    assert int(np.argmax(peak.cpu().numpy().max(axis=1))) == 7


def test_fused_candidates_match(dd):
    import torch
    rng = np.random.default_rng(67)
    C, T, D = 20, 4000, 33
    I = np.clip(rng.normal(128, 20, size=(C, T)), 0, 255).astype(np.uint8)
    plan, _, _ = _plan(dd, rng, C, T, D, 200, 30, "runlength")
    x = _dev(I)
    mean, sd = plan.channel_stats(x, nsamp=T)
    widths = np.arange(1, 17, dtype=np.int32)
    _, _, (c0, n0) = _unfused(plan, x, widths, mean, sd, 0, T, thresh=3.0, cap=4096)
    _, _, (c1, n1) = plan.dedisperse_boxcar(x, widths, mean, sd, nsamp=T, thresh=3.0, cap=4096)
    n = int(n0.item())
    assert 0 < n <= 4096 and int(n1.item()) == n
    key = lambda c: sorted(map(tuple, c[:n].cpu().numpy().tolist()))
    assert key(c1) == key(c0)


def test_fused_large_lowband_reduced(dd):
    """Large low-band band and trial list (1024 ch over 700-1000 MHz, dt 64 us, 8192 DMs
    to 2000, widths 1-256) on 2^18 samples: fused = unfused for every trial and width,
    and sampled trials against the oracle."""
    cfg = synth.make_large(nsamp=1 << 18)
    b = cfg["band"]
    T = cfg["nsamp"]
    plan = dd.Plan(dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, T, "u8"), cfg["dms"])
    assert plan.method == "runlength"
    x = _dev(cfg["data"])
    mean, sd = plan.channel_stats(x, nsamp=T)
    widths = np.arange(1, 257, dtype=np.int32)
    p1, a1, _ = plan.dedisperse_boxcar(x, widths, mean, sd, nsamp=T)
    assert plan.device_status() == 0
    out = plan.dedisperse(x, nsamp=T)
    p0, a0, _ = plan.boxcar_snr(out, widths, mean, sd)
    np.testing.assert_array_equal(a1.cpu().numpy(), a0.cpu().numpy())
    np.testing.assert_array_equal(p1.cpu().numpy(), p0.cpu().numpy())
    delay, taps = plan.tables()
    rows = [0, 1234, 5000, 8191]
    want = oracle.c_dedisperse(cfg["data"], delay, taps, nsamp=T, rows=rows)
    mu, sdw = ref.boxcar_norm(taps[rows], widths, *ref.channel_stats(cfg["data"], nsamp=T))
    opeak, oarg, _ = ref.boxcar_snr(want, widths, mu, sdw)
    np.testing.assert_array_equal(a1.cpu().numpy()[rows], oarg)
    np.testing.assert_allclose(p1.cpu().numpy()[rows], opeak, rtol=1e-5, atol=1e-5)


def test_fused_overflow_is_reported(dd):
    """Sums that cannot fit int32 around the offset (all samples 255, zero channel means
    passed in) are reported through the device status, not returned silently."""
    import torch
    C, T, D = 128, 3008, 8
    I = np.full((C, T), 255, np.uint8)
    plan = dd.Plan(dd.Band(C, 1200.0, 1.0, 1.0, T, "u8"), np.zeros(D))
    plan.set_profiles(delay=np.zeros((D, C), np.int32), taps=np.full((D, C), 70, np.int32))
    x = _dev(I)
    zero = torch.zeros(C, dtype=torch.float64, device="cuda")
    widths = np.arange(1, 994, dtype=np.int32)
    plan.device_status()
    plan.dedisperse_boxcar(x, widths, zero, zero + 1.0, nsamp=T)
    assert plan.device_status() == 2  # DD_ERR_OVERFLOW
    mean, sd = plan.channel_stats(x, nsamp=T)
    plan.dedisperse_boxcar(x, widths, mean, sd + 1.0, nsamp=T)
    assert plan.device_status() == 0


def test_fused_refuses_what_it_does_not_cover(dd):
    import torch
    C, T, D = 8, 2048, 4
    m = torch.zeros(C, dtype=torch.float64, device="cuda")
    f32 = dd.Plan(dd.Band(C, 1200.0, 1.0, 1.0, T, "f32"), np.zeros(D))
    xf = torch.zeros((C, T), dtype=torch.float32, device="cuda")
    with pytest.raises(dd.DDError):
        f32.dedisperse_boxcar(xf, np.array([1, 2, 4], np.int32), m, m + 1)   # not contiguous
    with pytest.raises(dd.DDError):
        f32.dedisperse_boxcar(xf, np.arange(1, 837, dtype=np.int32), m, m + 1)  # wmax + 29 > 864
    u8 = dd.Plan(dd.Band(C, 1200.0, 1.0, 1.0, T, "u8"), np.zeros(D))
    xu = torch.zeros((C, T), dtype=torch.uint8, device="cuda")
    with pytest.raises(dd.DDError):
        u8.dedisperse_boxcar(xu, np.array([1, 2, 4], np.int32), m, m + 1)   # not contiguous
    with pytest.raises(dd.DDError):
        u8.dedisperse_boxcar(xu, np.arange(1, 1000, dtype=np.int32), m, m + 1)  # wmax - 1 > tile


# ----------------------------------------------------------------------------- fp32 plans

def _bits(t):
    return t.cpu().numpy().view(np.int32)


def _f32_case(dd, rng, C, T, D, maxdel, maxtap, in_type, t_off):
    """Random delays, taps and mixed-sign weights; noise input with ld padded so that
    every row starts on 16 bytes."""
    plan = dd.Plan(dd.Band(C, 1200.0, 1.0, 1.0, T, in_type), np.zeros(D))
    delay = rng.integers(0, maxdel + 1, size=(D, C)).astype(np.int32)
    taps = rng.integers(1, maxtap + 1, size=(D, C)).astype(np.int32)
    w = (rng.standard_normal((D, C, maxtap)) * 0.5 + 1.0).astype(np.float32)
    plan.set_profiles(delay=delay, taps=taps, weights=w)
    ld = (T + t_off + 15) // 16 * 16
    if in_type == "f32":
        I = np.zeros((C, ld), np.float32)
        I[:, :T + t_off] = rng.standard_normal((C, T + t_off)).astype(np.float32) * 3 + 1
    else:
        I = np.zeros((C, ld), np.uint8)
        I[:, :T + t_off] = np.clip(rng.normal(128, 20, size=(C, T + t_off)), 0, 255).astype(np.uint8)
    return plan, delay, taps, w, I


@pytest.mark.parametrize("in_type", ["f32", "u8"])
@pytest.mark.parametrize("seed,C,T,D,maxdel,maxtap,t_off,w0,w1,parts", [
    (81, 24, 5000, 30, 300, 20, 0, 1, 32, 0),        # automatic parts
    (82, 37, 7100, 27, 900, 40, 16, 1, 256, 3),      # parts end inside blocks, two-pass windows
    (83, 16, 4200, 9, 100, 5, 0, 5, 40, 1000),       # one tile per part: a seam at every tile
    (84, 12, 3300, 25, 50, 3, 32, 1, 1, 2),          # width 1 only: the shortest carry
    (85, 30, 12000, 40, 500, 60, 0, 1, 300, 11),     # long windows (looped pair sums), widths 1-300
    (86, 20, 9000, 17, 200, 10, 0, 800, 835, 4),     # carry = tile: wmax + 29 = 864
])
def test_fused_f32_equals_unfused(dd, in_type, seed, C, T, D, maxdel, maxtap, t_off, w0, w1, parts):
    """fp32 sums: bit-identical S/N and identical earliest starts to dd_dedisperse
    followed by dd_boxcar_snr (the unfused fp32 scan's prefix chains)."""
    rng = np.random.default_rng(seed)
    plan, delay, taps, w, I = _f32_case(dd, rng, C, T, D, maxdel, maxtap, in_type, t_off)
    x = _dev(I)
    mean, sd = plan.channel_stats(x, t_offset=t_off, nsamp=T)
    widths = np.arange(w0, w1 + 1, dtype=np.int32)
    plan.test_set_fused_parts(parts)
    p0, a0, _ = _unfused(plan, x, widths, mean, sd, t_off, T)
    p1, a1, _ = plan.dedisperse_boxcar(x, widths, mean, sd, t_offset=t_off, nsamp=T)
    assert plan.device_status() == 0
    np.testing.assert_array_equal(a1.cpu().numpy(), a0.cpu().numpy())
    np.testing.assert_array_equal(_bits(p1), _bits(p0))


@pytest.mark.parametrize("nch", [2, 4])
def test_fused_f32_multi_chunk_ctas(dd, nch):
    """fp32 CTA shapes with several time chunks (a trial's row written and scanned by nch
    warps; segments cross the warps' chunks): fused = unfused."""
    rng = np.random.default_rng(90 + nch)
    plan, _, _, _, I = _f32_case(dd, rng, 20, 9008, 24, 600, 12, "f32", 0)
    plan.set_schedule(nch, 2)
    assert plan.schedule()["nch"] == nch
    x = _dev(I)
    mean, sd = plan.channel_stats(x, nsamp=9008)
    widths = np.arange(1, 200, dtype=np.int32)
    for parts in (0, 5):
        plan.test_set_fused_parts(parts)
        p0, a0, _ = _unfused(plan, x, widths, mean, sd, 0, 9008)
        p1, a1, _ = plan.dedisperse_boxcar(x, widths, mean, sd, nsamp=9008)
        assert plan.device_status() == 0
        np.testing.assert_array_equal(a1.cpu().numpy(), a0.cpu().numpy())
        np.testing.assert_array_equal(_bits(p1), _bits(p0))


def test_fused_f32_ties_take_the_earliest_start(dd):
    """A constant series (every window of a width has the same sum, zeros included): the
    earliest start wins in both scans, across seams."""
    import torch
    C, T, D = 8, 6000, 6
    plan = dd.Plan(dd.Band(C, 1200.0, 1.0, 1.0, T, "f32"), np.zeros(D))
    plan.set_profiles(delay=np.zeros((D, C), np.int32), taps=np.ones((D, C), np.int32))
    for val in (0.0, 1.0):
        x = torch.full((C, T), val, dtype=torch.float32, device="cuda")
        mean = torch.full((C,), val, dtype=torch.float64, device="cuda")
        sd = torch.ones(C, dtype=torch.float64, device="cuda")
        widths = np.arange(1, 41, dtype=np.int32)
        for parts in (0, 7):
            plan.test_set_fused_parts(parts)
            p0, a0, _ = _unfused(plan, x, widths, mean, sd, 0, T)
            p1, a1, _ = plan.dedisperse_boxcar(x, widths, mean, sd, nsamp=T)
            np.testing.assert_array_equal(a1.cpu().numpy(), a0.cpu().numpy())
            np.testing.assert_array_equal(_bits(p1), _bits(p0))
            assert (a1.cpu().numpy() == 0).all()


def test_fused_f32_against_oracle(dd):
    """A pulse on noise along trial 5's weighted profile: the oracle's fp64 dedispersion,
    normaliser and boxcar scan give S/N within 1e-5 and, where the maximum is clear, the
    same start."""
    rng = np.random.default_rng(87)
    C, T, D, K = 32, 6000, 12, 30
    plan, delay, taps, w, I = _f32_case(dd, rng, C, T, D, 400, K, "f32", 0)
    for c in range(C):
        s = 2500 + delay[5, c]
        I[c, s:s + taps[5, c]] += 4.0
    x = _dev(I)
    mean, sd = plan.channel_stats(x, nsamp=T)
    widths = np.arange(1, 65, dtype=np.int32)
    plan.test_set_fused_parts(3)
    peak, arg, _ = plan.dedisperse_boxcar(x, widths, mean, sd, nsamp=T)
    peak, arg = peak.cpu().numpy(), arg.cpu().numpy()
    xo = oracle.c_dedisperse(I, delay, taps, w=w, nsamp=T)
    mu_c, sd_c = ref.channel_stats(I, nsamp=T)
    mu, sdw = ref.boxcar_norm(taps, widths, mu_c, sd_c, w=w)
    opeak, oarg, _ = ref.boxcar_snr(xo, widths, mu, sdw)
    np.testing.assert_allclose(peak, opeak, rtol=1e-5, atol=1e-5)
    for d, j in zip(*np.nonzero(arg != oarg)):  # near-ties may pick either start
        B = ref.boxcar_series(xo[d], int(widths[j]))
        assert abs(B[arg[d, j]] - B[oarg[d, j]]) <= 1e-5 * max(abs(B[oarg[d, j]]), sdw[d, j])
    assert int(np.argmax(peak.max(axis=1))) == 5
    assert arg[5, 0] == oarg[5, 0]


def test_fused_f32_candidates_match(dd):
    rng = np.random.default_rng(88)
    plan, _, _, _, I = _f32_case(dd, rng, 20, 4000, 33, 200, 8, "f32", 0)
    x = _dev(I)
    mean, sd = plan.channel_stats(x, nsamp=4000)
    widths = np.arange(1, 17, dtype=np.int32)
    _, _, (c0, n0) = _unfused(plan, x, widths, mean, sd, 0, 4000, thresh=3.0, cap=4096)
    _, _, (c1, n1) = plan.dedisperse_boxcar(x, widths, mean, sd, nsamp=4000, thresh=3.0, cap=4096)
    n = int(n0.item())
    assert 0 < n <= 4096 and int(n1.item()) == n
    key = lambda c: sorted(map(tuple, c[:n].cpu().numpy().tolist()))
    assert key(c1) == key(c0)


def test_fused_f32_reduced_craft(dd):
    """CRAFT band, eq. trial DMs to 4000 with nu^-1.4 weights on every tap, 1024 trials
    on 16384 samples, widths 1-32: fused = unfused for every trial and width."""
    cfg = synth.make_craft(nsamp=16384, npulse=4)
    b = synth.CRAFT_BAND
    band = dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, 16384, "f32")
    dms, _ = dd.trial_dms(band, 0.0, 4000.0, 1024, tau_av_ms=1.0)
    plan = dd.Plan(band, dms)
    delay, taps = plan.tables()
    K = int(taps.max())
    wc = synth.spectral_weights(b)
    w = np.where(np.arange(K)[None, None, :] < taps[:, :, None], wc[None, :, None], 0.0).astype(np.float32)
    plan.set_profiles(weights=w)
    x = _dev(cfg["data"])
    mean, sd = plan.channel_stats(x, nsamp=16384)
    widths = np.arange(1, 33, dtype=np.int32)
    p0, a0, _ = _unfused(plan, x, widths, mean, sd, 0, 16384)
    p1, a1, _ = plan.dedisperse_boxcar(x, widths, mean, sd, nsamp=16384)
    assert plan.device_status() == 0
    np.testing.assert_array_equal(a1.cpu().numpy(), a0.cpu().numpy())
    np.testing.assert_array_equal(_bits(p1), _bits(p0))


@pytest.mark.parametrize("kind", ["u8", "f32"])
@pytest.mark.parametrize("t_out", [1, 30, 31, 40, 863, 864, 865, 992, 993])
def test_fused_short_series(dd, kind, t_out):
    """Series shorter than, equal to and one past a tile (864 fp32 / 992 integer outputs)
    and a boxcar segment (31): fused = unfused, widths up to the series length (or the
    longest one whose carry fits a tile)."""
    rng = np.random.default_rng(100 + t_out)
    C, D, K = 12, 20, 3
    delay = rng.integers(0, 4, size=(D, C)).astype(np.int32)
    taps = rng.integers(1, K + 1, size=(D, C)).astype(np.int32)
    T = t_out + int((delay + taps - 1).max())
    ld = (T + 15) // 16 * 16
    plan = dd.Plan(dd.Band(C, 1200.0, 1.0, 1.0, T, kind), np.zeros(D))
    w = None if kind == "u8" else (rng.standard_normal((D, C, K)) * 0.5 + 1.0).astype(np.float32)
    plan.set_profiles(delay=delay, taps=taps, weights=w)
    if kind == "u8":
        I = np.zeros((C, ld), np.uint8)
        I[:, :T] = rng.integers(0, 256, size=(C, T))
    else:
        I = np.zeros((C, ld), np.float32)
        I[:, :T] = rng.standard_normal((C, T))
    x = _dev(I)
    mean, sd = plan.channel_stats(x, nsamp=T)
    wcap = 835 if kind == "f32" else 993  # the longest width whose carry fits a tile
    for widths in (np.arange(1, min(32, t_out) + 1, dtype=np.int32), np.array([min(t_out, wcap)], np.int32)):
        p0, a0, _ = _unfused(plan, x, widths, mean, sd, 0, T)
        p1, a1, _ = plan.dedisperse_boxcar(x, widths, mean, sd, nsamp=T)
        assert plan.device_status() == 0
        np.testing.assert_array_equal(a1.cpu().numpy(), a0.cpu().numpy())
        np.testing.assert_array_equal(_bits(p1), _bits(p0))


@pytest.mark.parametrize("kind", ["u8", "f32"])
def test_fused_call_replays_in_a_cuda_graph(dd, kind):
    """After one eager call (which sends the part tables and widths), the fused call captures
    into a CUDA graph; replays on new input data give the eager call's results for that data."""
    import torch
    rng = np.random.default_rng(120)
    C, T, D = 16, 6000, 24
    plan = dd.Plan(dd.Band(C, 1200.0, 1.0, 1.0, T, kind), np.zeros(D))
    delay = rng.integers(0, 200, size=(D, C)).astype(np.int32)
    taps = rng.integers(1, 12, size=(D, C)).astype(np.int32)
    w = None if kind == "u8" else (rng.standard_normal((D, C, 11)) * 0.5 + 1.0).astype(np.float32)
    plan.set_profiles(delay=delay, taps=taps, weights=w)

    def data():
        if kind == "u8":
            return rng.integers(0, 256, size=(C, T)).astype(np.uint8)
        return rng.standard_normal((C, T)).astype(np.float32)

    x = _dev(data())
    mean, sd = plan.channel_stats(x, nsamp=T)
    widths = np.arange(1, 41, dtype=np.int32)
    plan.dedisperse_boxcar(x, widths, mean, sd, nsamp=T)       # eager: tables on the device
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        gp, ga, _ = plan.dedisperse_boxcar(x, widths, mean, sd, nsamp=T)
    for _ in range(2):
        x.copy_(_dev(data()))
        g.replay()
        torch.cuda.synchronize()
        p0, a0, _ = plan.dedisperse_boxcar(x, widths, mean, sd, nsamp=T)
        assert plan.device_status() == 0
        np.testing.assert_array_equal(ga.cpu().numpy(), a0.cpu().numpy())
        np.testing.assert_array_equal(_bits(gp), _bits(p0))
