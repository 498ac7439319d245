"""Batched beams, CUDA graph replay and the schedule autotuner against per-beam launches
and the oracle."""
import os
import tempfile

import numpy as np
import pytest

import oracle
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


def _beams(dd, n=6, seed=31):
    """Small uneven beams on the CRAFT band (the batched configuration at reduced size)."""
    import torch
    rng = np.random.default_rng(seed)
    b = synth.CRAFT_BAND
    out = []
    for i in range(n):
        T = int(round(2 ** rng.uniform(12, 13.5)))
        D = int(round(2 ** rng.uniform(5, 8)))
        dm_max = float(np.exp(rng.uniform(np.log(100.0), np.log(600.0))))
        band = dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, T, "u8")
        dms, _ = dd.trial_dms(band, 0.0, dm_max, D, tau_av_ms=1.0)
        plan = dd.Plan(band, dms)
        beam = dict(nsamp=T, ndm=D, dm_max=dm_max, seed=1000 + i)
        data = synth.make_beam_data(beam)
        x = torch.from_numpy(data).cuda()
        outb = torch.zeros((D, T - plan.d_max), dtype=torch.int32, device="cuda")
        out.append((plan, x, outb, data))
    return out


def test_batched_equals_per_beam_and_oracle(dd):
    import torch
    beams = _beams(dd)
    batch = dd.Batch([p for p, _, _, _ in beams])
    batch.bind([x for _, x, _, _ in beams], [o for _, _, o, _ in beams])
    batch.dedisperse()
    torch.cuda.synchronize()
    info = batch.info()
    assert info["items"] > 0 and info["grid"] > 0
    for plan, x, o, data in beams:
        ref = plan.dedisperse(x, nsamp=plan.band.nsamp)
        np.testing.assert_array_equal(o.cpu().numpy(), ref.cpu().numpy())
        delay, taps = plan.tables()
        rows = [0, plan.ndm // 2, plan.ndm - 1]
        want = oracle.c_dedisperse(data, delay, taps, nsamp=plan.band.nsamp, rows=rows)
        np.testing.assert_array_equal(o.cpu().numpy()[rows].astype(np.int64), want)
    # a second launch gives the same result
    before = [o.clone() for _, _, o, _ in beams]
    for _, _, o, _ in beams:
        o.zero_()
    batch.dedisperse()
    torch.cuda.synchronize()
    for b_, (_, _, o, _) in zip(before, beams):
        assert torch.equal(b_, o)


def test_graph_replay_equals_eager(dd):
    import torch
    beams = _beams(dd, n=4, seed=32)
    batch = dd.Batch([p for p, _, _, _ in beams])
    batch.bind([x for _, x, _, _ in beams], [o for _, _, o, _ in beams])
    widths = np.arange(1, 17, dtype=np.int32)
    means = [torch.empty(p.band.nchan, dtype=torch.float64, device="cuda") for p, _, _, _ in beams]
    sds = [torch.empty_like(m) for m in means]
    peaks = [torch.empty((p.ndm, 16), dtype=torch.float32, device="cuda") for p, _, _, _ in beams]
    args = [torch.empty((p.ndm, 16), dtype=torch.int32, device="cuda") for p, _, _, _ in beams]
    batch.bind_boxcar(widths, means, sds, peaks, args)
    batch.run()
    torch.cuda.synchronize()
    eager = [(o.clone(), pk.clone(), a.clone()) for (_, _, o, _), pk, a in zip(beams, peaks, args)]
    s = torch.cuda.Stream()
    batch.capture(s)
    for (_, _, o, _), pk, a in zip(beams, peaks, args):
        o.zero_()
        pk.zero_()
        a.zero_()
    torch.cuda.synchronize()
    batch.replay(s)
    s.synchronize()
    for (o0, p0, a0), (_, _, o, _), pk, a in zip(eager, beams, peaks, args):
        assert torch.equal(o0, o) and torch.equal(p0, pk) and torch.equal(a0, a)
    # each beam's boxcar matches its own single-plan call
    for (plan, x, o, _), pk, a in zip(beams, peaks, args):
        m, sd = plan.channel_stats(x, nsamp=plan.band.nsamp)
        p1, a1, _ = plan.boxcar_snr(o, widths, m, sd)
        assert torch.equal(p1, pk) and torch.equal(a1, a)


def test_autotune_keeps_results_and_uses_cache(dd):
    import torch
    cfg = synth.make_craft(nsamp=8192, npulse=2)
    b = cfg["band"]
    band = dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, 8192, "f32")
    dms, _ = dd.trial_dms(band, 0.0, 1000.0, 128, tau_av_ms=1.0)
    plan = dd.Plan(band, dms)
    x = torch.from_numpy(cfg["data"]).cuda()
    ref = plan.dedisperse(x, nsamp=8192).clone()
    out = torch.empty_like(ref)
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "tune.txt")
        ms = plan.autotune(x, out, cache_path=path)
        assert ms > 0 and os.path.exists(path)
        sched = plan.schedule()
        got = plan.dedisperse(x, nsamp=8192)
        # fp32 sums in another stage grouping may round differently only by reassociation
        # across stage boundaries -- none here: the channel order is fixed, so identical
        assert torch.equal(got, ref)
        plan2 = dd.Plan(band, dms)
        assert plan2.autotune(x, out, cache_path=path) == -1.0
        assert plan2.schedule() == sched


def test_batched_long_taps_equals_per_beam(dd):
    """A beam whose tap runs exceed one register window takes the general tap loop for
    the whole batch; results still equal the per-beam launches and the oracle."""
    import torch
    beams = _beams(dd, n=3, seed=33)
    plan, x, o, data = beams[1]
    rng = np.random.default_rng(34)
    D, C = plan.ndm, plan.band.nchan
    delay = rng.integers(0, 200, size=(D, C)).astype(np.int32)
    taps = rng.integers(1, 61, size=(D, C)).astype(np.int32)     # up to 60 > 31
    plan.set_profiles(delay=delay, taps=taps)
    plan.set_method("direct")
    o2 = torch.zeros((D, plan.band.nsamp - plan.d_max), dtype=torch.int32, device="cuda")
    beams[1] = (plan, x, o2, data)
    batch = dd.Batch([p for p, _, _, _ in beams])
    batch.bind([x for _, x, _, _ in beams], [o for _, _, o, _ in beams])
    batch.dedisperse()
    torch.cuda.synchronize()
    for p, xb, ob, db in beams:
        np.testing.assert_array_equal(ob.cpu().numpy(), p.dedisperse(xb, nsamp=p.band.nsamp).cpu().numpy())
    want = oracle.c_dedisperse(data, delay, taps, nsamp=plan.band.nsamp, rows=[0, D - 1])
    np.testing.assert_array_equal(o2.cpu().numpy()[[0, D - 1]].astype(np.int64), want)


def _rl_beams(dd, n=5, seed=47, share_rows=True):
    """Uneven run-length beams on 256 channels of the low band (700-775 MHz, 64 us
    sampling): long tap runs, prefix-sum differences; with share_rows the trial lists
    are dense enough that each block of trials has at most two tap counts per channel."""
    import torch
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        T = int(round(2 ** rng.uniform(14, 15.5)))
        dm_max = float(rng.uniform(60.0, 150.0))
        # dense lists: a 24-trial block spans < 7 pc cm^-3, so at most two tap counts
        D = int(3.5 * dm_max) + int(rng.integers(0, 30)) if share_rows else int(rng.integers(40, 60))
        dms = np.linspace(0.0, dm_max, D)
        band = dd.Band(256, 700.0, 300.0 / 1024, 0.064, T, "u8")
        plan = dd.Plan(band, dms)
        plan.set_method("runlength")
        ld = (T + 15) // 16 * 16                # rows staged in 16-byte chunks
        data = np.zeros((256, ld), np.uint8)
        data[:, :T] = rng.integers(0, 256, size=(256, T))
        x = torch.from_numpy(data).cuda()
        outb = torch.zeros((D, T - plan.d_max), dtype=torch.int32, device="cuda")
        out.append((plan, x, outb, data))
    return out


@pytest.mark.parametrize("share_rows", [True, False])
def test_batched_runlength_equals_per_beam_and_oracle(dd, share_rows):
    """Run-length beams in one batched launch (prefix passes first) give the per-beam
    run-length sums bit for bit, sampled rows equal the oracle, and the graph replay
    repeats them."""
    import torch
    beams = _rl_beams(dd, share_rows=share_rows)
    assert all(p.method == "runlength" for p, _, _, _ in beams)
    batch = dd.Batch([p for p, _, _, _ in beams])
    batch.bind([x for _, x, _, _ in beams], [o for _, _, o, _ in beams])
    batch.dedisperse()
    torch.cuda.synchronize()
    for plan, x, o, data in beams:
        ref = plan.dedisperse(x, nsamp=plan.band.nsamp)
        np.testing.assert_array_equal(o.cpu().numpy(), ref.cpu().numpy())
        delay, taps = plan.tables()
        rows = [0, plan.ndm // 3, plan.ndm - 1]
        want = oracle.c_dedisperse(data, delay, taps, nsamp=plan.band.nsamp, rows=rows)
        np.testing.assert_array_equal(o.cpu().numpy()[rows].astype(np.int64), want)
    before = [o.clone() for _, _, o, _ in beams]
    for _, _, o, _ in beams:
        o.zero_()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        batch.capture(s)
        for _, _, o, _ in beams:
            o.zero_()
        batch.replay(s)
    s.synchronize()
    for b_, (_, _, o, _) in zip(before, beams):
        assert torch.equal(b_, o)
    batch.close()


def test_batch_refuses_mixed_methods(dd):
    beams = _rl_beams(dd, n=2)
    beams[1][0].set_method("direct")
    with pytest.raises(dd.DDError):
        dd.Batch([p for p, _, _, _ in beams])


def test_batched_fp32_weighted_equals_per_beam_and_oracle(dd):
    """fp32 weighted beams (pair units with each trial's own run in the shared window) in
    one batched launch: bit for bit the per-beam launches, sampled rows within the fp32
    tolerance of the oracle, and the graph replay repeats them."""
    import torch
    rng = np.random.default_rng(71)
    b = synth.CRAFT_BAND
    beams = []
    for i in range(4):
        T = int(rng.integers(5000, 9000)) // 4 * 4
        D = int(rng.integers(20, 70))
        band = dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, T, "f32")
        dms, _ = dd.trial_dms(band, 0.0, float(rng.uniform(300.0, 1500.0)), D, tau_av_ms=1.0)
        plan = dd.Plan(band, dms)
        _, taps = plan.tables()
        K = int(taps.max())
        w = (rng.uniform(0.2, 1.5, size=(D, b.nchan, K))
             * (np.arange(K)[None, None, :] < taps[:, :, None])).astype(np.float32)
        plan.set_profiles(weights=w)
        data = rng.standard_normal((b.nchan, T)).astype(np.float32)
        x = torch.from_numpy(data).cuda()
        out = torch.zeros((D, T - plan.d_max), dtype=torch.float32, device="cuda")
        beams.append((plan, x, out, data, w))
    batch = dd.Batch([p for p, _, _, _, _ in beams])
    batch.bind([x for _, x, _, _, _ in beams], [o for _, _, o, _, _ in beams])
    batch.dedisperse()
    torch.cuda.synchronize()
    for plan, x, o, data, w in beams:
        ref_ = plan.dedisperse(x, nsamp=plan.band.nsamp)
        assert torch.equal(o, ref_)
        delay, taps = plan.tables()
        rows = [0, plan.ndm // 2, plan.ndm - 1]
        want = oracle.c_dedisperse(data, delay, taps, w=w, nsamp=plan.band.nsamp, rows=rows)
        scale = oracle.c_abs_scale(data, delay, taps, w=w, nsamp=plan.band.nsamp, rows=rows)
        assert (np.abs(o.cpu().numpy()[rows] - want) <= 1e-5 * scale + 1e-30).all()
    before = [o.clone() for _, _, o, _, _ in beams]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        batch.capture(s)
        for _, _, o, _, _ in beams:
            o.zero_()
        batch.replay(s)
    s.synchronize()
    for b_, (_, _, o, _, _) in zip(before, beams):
        assert torch.equal(b_, o)
    batch.close()
