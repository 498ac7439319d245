"""Parity at the full sizes of the measured configurations, in the launch configuration
bench.py times, on outputs the oracle computes one by one (sampled rows or points)."""
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


def test_batched_36_beams_full_size(dd):
    """36 beams of 2^14-2^17 samples and 512-8192 trials, uint8 -> int32, one batched
    launch: three rows of every beam bit-exact against the oracle."""
    import torch
    cfg = synth.make_batched_beams()
    b = cfg["band"]
    plans, xs, outs, datas = [], [], [], []
    for beam in cfg["beams"]:
        band = dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, beam["nsamp"], "u8")
        dms, _ = dd.trial_dms(band, 0.0, beam["dm_max"], beam["ndm"], tau_av_ms=1.0)
        plan = dd.Plan(band, dms)
        data = synth.make_beam_data(beam)
        plans.append(plan)
        datas.append(data)
        xs.append(_dev(data))
        outs.append(torch.empty((len(dms), beam["nsamp"] - plan.d_max), dtype=torch.int32, device="cuda"))
    batch = dd.Batch(plans)
    batch.bind(xs, outs)
    batch.dedisperse()
    torch.cuda.synchronize()
    rng = np.random.default_rng(81)
    for plan, data, o in zip(plans, datas, outs):
        rows = sorted(set([0, plan.ndm - 1, int(rng.integers(plan.ndm))]))
        delay, taps = plan.tables()
        want = oracle.c_dedisperse(data, delay, taps, nsamp=plan.band.nsamp, rows=rows)
        np.testing.assert_array_equal(o[rows].cpu().numpy().astype(np.int64), want)
    batch.close()


def test_large_lowband_full_size_streamed(dd):
    """2^20 uint8 samples, 8192 trials to DM 2000, run-length sums in 4 overlapping chunks
    of 2^18 outputs (as bench.py streams them): 96 sampled outputs bit-exact."""
    import torch
    cfg = synth.make_large()
    b, T = cfg["band"], cfg["nsamp"]
    plan = dd.Plan(dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, T, "u8"), cfg["dms"])
    assert plan.method == "runlength"
    x = _dev(cfg["data"])
    dmax = plan.d_max
    t_out = T - dmax
    chunk = 1 << 18
    out = torch.empty((plan.ndm, chunk), dtype=torch.int32, device="cuda")
    delay, taps = plan.tables()
    rng = np.random.default_rng(82)
    for t0 in range(0, t_out, chunk):
        n = min(chunk, t_out - t0)
        plan.dedisperse(x, t_offset=t0, nsamp=n + dmax, out=out)
        pts = [(int(rng.integers(plan.ndm)), int(rng.integers(n))) for _ in range(24)]
        pts[0] = (plan.ndm - 1, n - 1)                # the last output of the chunk
        got = out.cpu().numpy()[[p[0] for p in pts], [p[1] for p in pts]]
        want = ref.dedisperse_points(cfg["data"], delay, taps, pts, t_offset=t0)
        np.testing.assert_array_equal(got.astype(np.int64), want)


def test_large_lowband_full_size_fused(dd):
    """The bench's large low-band block through the fused call, chunk by chunk (2^20
    samples, 8192 trials, widths 1-256, 4 overlapping chunks of 2^18 outputs): every peak
    and start equal to dedispersion + boxcar on the stored chunk, and sampled trials of
    one chunk equal to the oracle's dedispersion and scan."""
    import torch
    cfg = synth.make_large()
    b, T = cfg["band"], cfg["nsamp"]
    plan = dd.Plan(dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, T, "u8"), cfg["dms"])
    x = _dev(cfg["data"])
    dmax = plan.d_max
    t_out = T - dmax
    chunk = 1 << 18
    widths = np.arange(1, 257, dtype=np.int32)
    mean, sd = plan.channel_stats(x, nsamp=T)
    out = torch.empty((plan.ndm, chunk), dtype=torch.int32, device="cuda")
    delay, taps = plan.tables()
    rows = [3, 4100, 8190]
    for t0 in range(0, t_out, chunk):
        n = min(chunk, t_out - t0)
        p1, a1, _ = plan.dedisperse_boxcar(x, widths, mean, sd, t_offset=t0, nsamp=n + dmax)
        assert plan.device_status() == 0
        plan.dedisperse(x, t_offset=t0, nsamp=n + dmax, out=out)
        p0, a0, _ = plan.boxcar_snr(out, widths, mean, sd, t_len=n)
        np.testing.assert_array_equal(a1.cpu().numpy(), a0.cpu().numpy())
        np.testing.assert_array_equal(p1.cpu().numpy(), p0.cpu().numpy())
        if t0 == chunk:
            want = oracle.c_dedisperse(cfg["data"], delay, taps, t_offset=t0, nsamp=n + dmax, rows=rows)
            mu, sdw = ref.boxcar_norm(taps[rows], widths, *ref.channel_stats(cfg["data"], nsamp=T))
            opeak, oarg, _ = ref.boxcar_snr(want, widths, mu, sdw)
            np.testing.assert_array_equal(a1.cpu().numpy()[rows], oarg)
            np.testing.assert_allclose(p1.cpu().numpy()[rows], opeak, rtol=1e-5, atol=1e-5)


def test_differentiable_full_size_gradients(dd):
    """336 channels, 16384 fp32 samples, 1024 trials, 32 learnable taps: forward rows and
    sampled weight and input gradients through the adjoint kernels against the oracle
    within the 1e-5 scale-aware bound."""
    import torch
    cfg = synth.make_diff(npulse=0)
    b, T, D, K = cfg["band"], cfg["nsamp"], 1024, 32
    band = dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, T, "f32")
    dms, _ = dd.trial_dms(band, 0.0, 2000.0, D, tau_av_ms=1.0)
    plan = dd.Plan(band, dms)
    delay, taps0 = plan.tables()
    rng = np.random.default_rng(83)
    taps = np.full_like(taps0, K)
    w = rng.uniform(0.5, 1.5, size=(D, b.nchan, K)).astype(np.float32)
    plan.set_profiles(delay=delay, taps=taps, weights=w)
    I = cfg["data"]
    x = _dev(I)
    out = plan.dedisperse(x, nsamp=T).cpu().numpy()
    rows = [0, 511, 1023]
    want = oracle.c_dedisperse(I, delay, taps, w=w, nsamp=T, rows=rows)
    scale = oracle.c_abs_scale(I, delay, taps, w=w, nsamp=T, rows=rows)
    assert (np.abs(out[rows] - want) <= 1e-5 * scale + 1e-30).all()
    t_out = out.shape[1]
    g = rng.standard_normal((D, t_out)).astype(np.float32)
    gw, gI = plan.backward(x, _dev(g), nsamp=T)
    gw, gI = gw.cpu().numpy(), gI.cpu().numpy()
    gwp = [(int(rng.integers(D)), int(rng.integers(b.nchan)), int(rng.integers(K))) for _ in range(48)]
    gip = [(int(rng.integers(b.nchan)), int(rng.integers(T))) for _ in range(24)]
    a, bI = ref.adjoint_points(I, g, delay, taps, w, gwp, gip)
    sa, sb = ref.adjoint_points(np.abs(I), np.abs(g), delay, taps, np.abs(w), gwp, gip)
    got_w = np.array([gw[d, c, k] for d, c, k in gwp])
    got_i = np.array([gI[c, t] for c, t in gip])
    assert (np.abs(got_w - a) <= 1e-5 * sa + 1e-30).all()
    assert (np.abs(got_i - bI) <= 1e-5 * sb + 1e-30).all()


def test_craft_full_size_fused(dd):
    """The full CRAFT-like block (336 x 65536 fp32, 4096 weighted trials, widths 1-32) through
    the fused call in the bench's configuration: every peak S/N (bit for bit) and start
    equal to dedispersion + boxcar, and 8 sampled trials against the oracle's fp64
    dedispersion, normaliser and scan (S/N within 1e-5; starts equal or tied to 1e-5)."""
    import torch
    cfg = synth.make_craft()
    b = synth.CRAFT_BAND
    T = cfg["nsamp"]
    band = dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, T, "f32")
    dms, _ = dd.trial_dms(band, 0.0, cfg["dm_max"], cfg["ndm"], tau_av_ms=1.0)
    plan = dd.Plan(band, dms)
    delay, taps = plan.tables()
    K = int(taps.max())
    w = np.where(np.arange(K)[None, None, :] < taps[:, :, None], cfg["wchan"][None, :, None], 0.0)
    w = np.ascontiguousarray(w, dtype=np.float32)
    plan.set_profiles(weights=w)
    x = _dev(cfg["data"])
    widths = np.asarray(cfg["widths"], dtype=np.int32)
    mean, sd = plan.channel_stats(x, nsamp=T)
    p1, a1, _ = plan.dedisperse_boxcar(x, widths, mean, sd, nsamp=T)
    assert plan.device_status() == 0
    out = plan.dedisperse(x, nsamp=T)
    p0, a0, _ = plan.boxcar_snr(out, widths, mean, sd)
    np.testing.assert_array_equal(a1.cpu().numpy(), a0.cpu().numpy())
    np.testing.assert_array_equal(p1.cpu().numpy().view(np.int32), p0.cpu().numpy().view(np.int32))
    del out
    torch.cuda.empty_cache()
    rows = [0, 1, 700, 1500, 2222, 3000, 4094, 4095]
    xo = oracle.c_dedisperse(cfg["data"], delay, taps, w=w, nsamp=T, rows=rows)
    mu_c, sd_c = ref.channel_stats(cfg["data"], nsamp=T)
    mu, sdw = ref.boxcar_norm(taps[rows], widths, mu_c, sd_c, w=w[rows])
    opeak, oarg, _ = ref.boxcar_snr(xo, widths, mu, sdw)
    peak, arg = p1.cpu().numpy()[rows], a1.cpu().numpy()[rows]
    np.testing.assert_allclose(peak, opeak, rtol=1e-5, atol=1e-5)
    for i, j in zip(*np.nonzero(arg != oarg)):  # near-ties may pick either start
        B = ref.boxcar_series(xo[i], int(widths[j]))
        assert abs(B[arg[i, j]] - B[oarg[i, j]]) <= 1e-5 * max(abs(B[oarg[i, j]]), sdw[i, j])
