"""C-ABI library on the CPU: it loads, exports every declared symbol, and its host
logic (profile tables, trial DMs, argument checking) matches the oracle.  No device
compute runs here."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle
from oracle import ref
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1301_3968_gb300 import build
    build.build()
    from paper_1301_3968_gb300 import _lib
    return _lib.load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(dd_\w+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(lib):
    from paper_1301_3968_gb300 import _lib
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert names == set(_lib.SIGNATURES), "binding and header disagree"


def test_status_strings(lib):
    from paper_1301_3968_gb300 import _lib
    for code in _lib.STATUS:
        assert lib.dd_status_str(code)
    assert lib.dd_version() >= 100


def _plan(band, dms):
    import paper_1301_3968_gb300 as dd
    return dd.Plan(band, dms)


@pytest.mark.parametrize("cfg", ["plain", "craft", "large", "desc"])
def test_plan_tables_match_oracle(lib, cfg):
    import paper_1301_3968_gb300 as dd
    if cfg == "plain":
        b, dms, k = synth.PLAIN_BAND, np.linspace(0, 500, 128), 4.15
    elif cfg == "craft":
        b, k = synth.CRAFT_BAND, 4.1494
        dms, _ = ref.trial_dms(0.0, 4000.0, 512, b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, 1.0)
    elif cfg == "large":
        b, dms, k = synth.LARGE_BAND, np.linspace(0, 2000, 96), 4.15
    else:
        b, dms, k = synth.Band(48, 700.0, 6.25, 0.5, descending=True), np.linspace(3, 900, 40), 4.15
    band = dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, 1 << 16, "u8", b.descending, k)
    plan = dd.Plan(band, dms)
    gd, gt = plan.tables()
    od, raw_d = ref.delay_table(dms, b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, b.descending, k)
    ot, raw_t = ref.taps_table(dms, b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, b.descending, k)
    # a mismatch is only allowed where the pre-floor value sits within 1e-9 of an integer
    bad_d = (gd != od) & (np.abs(raw_d - np.rint(raw_d)) > 1e-9)
    bad_t = (gt != ot) & (np.abs(raw_t - np.rint(raw_t)) > 1e-9)
    assert not bad_d.any() and not bad_t.any()
    info = plan.info()
    assert info["d_max"] == ref.d_max(gd, gt)
    assert info["ns_total"] == int(gt.sum())
    assert info["kmax"] == int(gt.max())
    assert info["out_is_int"]


def test_trial_dms_match_oracle(lib):
    import paper_1301_3968_gb300 as dd
    b = synth.CRAFT_BAND
    band = dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, 1024, "f32")
    for st in (1, 2):
        g, geps = dd.trial_dms(band, 0.0, 4000.0, 4096, tau_av_ms=1.0, smear_terms=st)
        o, oeps = ref.trial_dms(0.0, 4000.0, 4096, b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, 1.0,
                                smear_terms=st)
        np.testing.assert_allclose(g, o, rtol=1e-12, atol=1e-9)
        assert geps == pytest.approx(oeps, rel=1e-10)


def test_argument_errors(lib):
    import paper_1301_3968_gb300 as dd
    from paper_1301_3968_gb300 import _lib
    band = dd.Band(8, 1200.0, 10.0, 1.0, 256, "f32")
    b = band.c_struct()
    h = ctypes.c_void_p()
    dms = np.array([0.0, 10.0])
    # bad plans
    assert lib.dd_plan_create(None, ctypes.byref(b), dms.ctypes.data, 2) == 1
    assert lib.dd_plan_create(ctypes.byref(h), ctypes.byref(b), dms.ctypes.data, 0) == 1
    neg = np.array([-1.0])
    assert lib.dd_plan_create(ctypes.byref(h), ctypes.byref(b), neg.ctypes.data, 1) == 1
    bad = dd.Band(0, 1200.0, 10.0, 1.0, 256, "f32").c_struct()
    assert lib.dd_plan_create(ctypes.byref(h), ctypes.byref(bad), dms.ctypes.data, 2) == 1
    assert lib.dd_plan_create(ctypes.byref(h), ctypes.byref(b), dms.ctypes.data, 2) == 0
    # misaligned leading dimension and pointer, short input, null pointers
    fake = ctypes.c_void_p(1 << 20)
    assert lib.dd_dedisperse(h, fake, 255, 0, 200, fake, 256, None) == 1
    assert lib.dd_dedisperse(h, ctypes.c_void_p((1 << 20) + 4), 256, 0, 200, fake, 256, None) == 1
    assert lib.dd_dedisperse(h, fake, 256, 100, 200, fake, 256, None) == 1
    assert lib.dd_dedisperse(h, None, 256, 0, 200, fake, 256, None) == 1
    # profile validation leaves the plan usable
    dl = np.zeros((2, 8), np.int32)
    tp = np.zeros((2, 8), np.int32)
    assert lib.dd_set_profiles(h, dl.ctypes.data, tp.ctypes.data, None, 0) == 1
    tp[:] = 5
    w = np.ones((2, 8, 4), np.float32)
    assert lib.dd_set_profiles(h, dl.ctypes.data, tp.ctypes.data, w.ctypes.data, 4) == 1
    # boxcar widths must be increasing and fit the series
    wl = np.array([3, 2], np.int32)
    assert lib.dd_boxcar_snr(h, fake, 100, 100, wl.ctypes.data, 2, fake, fake, fake, fake,
                             ctypes.c_float(1.0), None, 0, None, None) == 1
    wl = np.array([1, 101], np.int32)
    assert lib.dd_boxcar_snr(h, fake, 100, 100, wl.ctypes.data, 2, fake, fake, fake, fake,
                             ctypes.c_float(1.0), None, 0, None, None) == 1
    assert lib.dd_plan_destroy(h) == 0


def test_fused_argument_checks(lib):
    """dd_dedisperse_boxcar refuses, before any device work, what its kernels do not cover:
    non-contiguous widths, carries longer than a tile (wmax - 1 on integer plans, wmax + 29
    on fp32 plans), and the usual argument errors."""
    import paper_1301_3968_gb300 as dd
    fake = ctypes.c_void_p(1 << 20)

    def call(plan, wl, ld=2048, nsamp=2048, t_offset=0, x=fake):
        wl = np.ascontiguousarray(wl, np.int32)
        return lib.dd_dedisperse_boxcar(plan._h, x, ld, t_offset, nsamp, wl.ctypes.data, len(wl), fake,
                                        fake, fake, fake, ctypes.c_float(1.0), None, 0, None, None)

    f32 = dd.Plan(dd.Band(8, 1200.0, 1.0, 1.0, 2048, "f32"), np.zeros(4))
    assert f32.schedule()["nch"] == 1
    assert call(f32, [1, 2, 4]) == 8                      # not contiguous
    assert call(f32, np.arange(1, 837)) == 8              # wmax + 29 > 864
    u8 = dd.Plan(dd.Band(8, 1200.0, 1.0, 1.0, 2048, "u8"), np.zeros(4))
    assert u8.schedule()["nch"] == 1
    assert call(u8, [1, 2, 4]) == 8                       # not contiguous
    assert call(u8, np.arange(1, 995)) == 8               # wmax - 1 > 992
    assert call(u8, [3, 2]) == 1                          # not increasing
    assert call(u8, [1, 2049]) == 1                       # longer than the series
    assert call(u8, [1, 2], x=None) == 1
    assert call(u8, [1, 2], ld=2047, nsamp=2047) == 1     # leading dimension not 16-byte aligned
    assert call(u8, [1, 2], t_offset=16) == 1             # runs past the row
    weighted = dd.Plan(dd.Band(8, 1200.0, 1.0, 1.0, 2048, "u8"), np.zeros(4))
    weighted.set_profiles(weights=np.full((4, 8, 1), 0.5, np.float32))
    assert call(weighted, np.arange(1, 837)) == 8         # fp32 sums: wmax + 29 > 864
    assert call(f32, [1, 2], ld=2047, nsamp=2047) == 1    # fp32 rows not 16-byte aligned


def test_int32_overflow_is_refused(lib):
    """A uint8 plan whose sums could exceed int32 is rejected (DD_ERR_OVERFLOW)."""
    import paper_1301_3968_gb300 as dd
    band = dd.Band(4, 1200.0, 10.0, 1.0, 1 << 24, "u8")
    plan = dd.Plan(band, [0.0])
    taps = np.full((1, 4), 3_000_000, np.int32)
    with pytest.raises(dd.DDError) as e:
        plan.set_profiles(taps=taps)
    assert e.value.code in (2, 8)
    # the plan keeps its previous profile
    assert plan.tables()[1].max() == 1


def test_method_selection_host_logic(lib):
    """Run-length sums are chosen for uint8 unit-weight plans with long tap runs, are
    refused for weighted and fp32 plans, and widen the CTA to 24 trials."""
    import paper_1301_3968_gb300 as dd
    b = synth.LARGE_BAND
    band = dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, 1 << 18, "u8")
    plan = dd.Plan(band, np.linspace(0.0, 2000.0, 64))
    assert plan.method == "runlength"                     # mean taps ~66 >= 12
    assert plan.schedule()["trials_per_cta"] == 24 // plan.schedule()["nch"]
    plan.set_method("direct")
    assert plan.method == "direct" and plan.schedule()["trials_per_cta"] == 8 // plan.schedule()["nch"]
    plan.set_method("auto")
    assert plan.method == "runlength"
    pb = synth.PLAIN_BAND
    small = dd.Plan(dd.Band(pb.nchan, pb.f_lo_mhz, pb.df_mhz, pb.dt_ms, 4096, "u8"), np.linspace(0, 500, 128))
    assert small.method == "direct"                       # taps <= 12, mean ~3
    small.set_method("runlength")
    assert small.method == "runlength"
    f32 = dd.Plan(dd.Band(pb.nchan, pb.f_lo_mhz, pb.df_mhz, pb.dt_ms, 4096, "f32"), np.linspace(0, 500, 16))
    with pytest.raises(dd.DDError):
        f32.set_method("runlength")
    assert f32.method == "direct"
    # a run-length plan that gets weights sums directly
    small.set_profiles(weights=np.ones((128, pb.nchan, 16), np.float32))
    assert small.method == "direct"


# ----------------------------------------------------------------------------- profile construction


@pytest.mark.parametrize("dm,t0,alpha,desc", [(30.0, 10.0, 0.0, False), (300.0, 4.3, 2.0, False),
                                              (1200.0, 0.6, -1.5, True)])
def test_predict_rect_matches_pulse_model(lib, dm, t0, alpha, desc):
    import paper_1301_3968_gb300 as dd
    b = synth.Band(48, 700.0, 6.25, 1.0, descending=desc)
    T = 3000
    want = synth.rect_pulse_cells(b, T, dm, t0, 1.0, 2.0, alpha=alpha, nu0_ghz=1.1)
    band = dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, T, "f32", desc)
    got = dd.predict_rect(band, dm, T, t0_ms=t0, tau_ms=1.0, tau_prime_ms=2.0, alpha=alpha, nu0_ghz=1.1)
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-14)


def test_select_samples_matches_oracle(lib):
    import paper_1301_3968_gb300 as dd
    rng = np.random.default_rng(62)
    maps = [rng.exponential(1.0, size=(6, 9)) * (rng.random((6, 9)) < 0.6),
            rng.integers(0, 4, size=(5, 8)).astype(float)]
    for C, dt in ((60, 1.0), (122, 1.0), (244, 2.0)):
        b = synth.Band(C, 700.0, 300.0 / C, dt)
        maps.append(synth.rect_pulse_cells(b, int(200 / dt), 30.0, 10.0, 1.0, 1.0))
    for p in maps:
        C, nt = p.shape
        delay, taps, w, nsel, gain = dd.select_samples(p, nt)
        mask = np.zeros_like(p, dtype=bool)
        for c in range(C):
            for k in range(taps[c]):
                if w[c, k] == 1.0:
                    mask[c, delay[c] + k] = True
        want = ref.select_samples(p)
        np.testing.assert_array_equal(mask, want)
        assert nsel == want.sum()
        assert gain == pytest.approx(ref.set_snr(p, want) / ref.set_snr(p, p > 0), rel=1e-12)
        # every tap outside the selection has weight 0, and runs start and end on it
        for c in range(C):
            if mask[c].any():
                assert w[c, 0] == 1.0 and w[c, taps[c] - 1] == 1.0
    with pytest.raises(dd.DDError):
        dd.select_samples(np.ones((2, 10)), 4)          # a 10-sample run with kmax 4


def test_select_profiles_match_oracle_selection(lib):
    """dd_select_profiles (every trial of a plan) equals the oracle's Sec. 2.2 selection on
    the pulse model's cells of each trial, trial by trial, with the same gains."""
    import paper_1301_3968_gb300 as dd
    b = synth.Band(60, 700.0, 5.0, 1.0)
    dms = np.array([0.0, 12.5, 30.0, 55.0])
    band = dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, 4096, "f32")
    phase, tau, taup, alpha = 0.4, 1.0, 1.5, 1.0
    delay, taps, w, gains = dd.select_profiles(band, dms, tau_ms=tau, tau_prime_ms=taup, alpha=alpha,
                                               nu0_ghz=0.85, phase=phase)
    assert w.shape == (len(dms), b.nchan, int(taps.max()))
    for d, dm in enumerate(dms):
        # a map long enough for the whole sweep across the band
        nt = int(4.15 * dm * (1 / 0.7 ** 2 - 1 / 1.0 ** 2) / b.dt_ms) + 20
        P = synth.rect_pulse_cells(b, nt, dm, phase * b.dt_ms, tau, taup, alpha=alpha, nu0_ghz=0.85)
        want = ref.select_samples(P)
        mask = np.zeros_like(want)
        for c in range(b.nchan):
            for k in range(taps[d, c]):
                if w[d, c, k] == 1.0:
                    mask[c, delay[d, c] + k] = True
        np.testing.assert_array_equal(mask, want)
        assert gains[d] == pytest.approx(ref.set_snr(P, want) / ref.set_snr(P, P > 0), rel=1e-9)


def test_exact_profiles_cover_the_rect_pulse(lib):
    """eq. num_samples: delay = floor(t_A/dt), taps = ceil(t_B/dt) - floor(t_A/dt) is the
    extent of the cells holding power of a pulse arriving at t = 0 with width tau'.  The
    model's frequency quadrature samples sub-channel midpoints, so at either end of a run
    it may miss a cell that only the band-edge frequencies reach: exact there or one
    cell wider, never narrower."""
    import paper_1301_3968_gb300 as dd
    b = synth.Band(40, 700.0, 7.5, 1.0)
    dms = np.array([0.0, 17.3, 230.0, 911.0])
    plan = dd.Plan(dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, 8192, "f32"), dms)
    delay, taps = plan.exact_profiles(1.37)
    for d, dm in enumerate(dms):
        P = synth.rect_pulse_cells(b, 8192, dm, 0.0, 1.0, 1.37)
        first = np.array([np.flatnonzero(P[c] > 0)[0] for c in range(b.nchan)])
        last = np.array([np.flatnonzero(P[c] > 0)[-1] for c in range(b.nchan)])
        end = delay[d] + taps[d] - 1
        assert ((first - delay[d] >= 0) & (first - delay[d] <= 1)).all()
        assert ((end - last >= 0) & (end - last <= 1)).all()
        assert ((first - delay[d]) + (end - last) == 0).mean() > 0.8


@pytest.mark.parametrize("kind", ["dsmf", "ts_mf", "ts_boxcar"])
def test_detector_profiles_match_oracle(lib, kind):
    import paper_1301_3968_gb300 as dd
    for C, dt, dm in ((40, 1.0, 30.0), (122, 1.0, 30.0), (12, 2.0, 300.0)):
        b = synth.Band(C, 700.0, 300.0 / C, dt)
        P = synth.rect_pulse_cells(b, int(3000 / dt), dm, 20.0, 1.0, 1.0)
        dl, _ = ref.delay_table([dm], C, 700.0, 300.0 / C, dt)
        align = (dl[0] + 20).astype(np.int32)
        delay, taps, w, snr = dd.detector_profile(P, kind, 1024, align=align)
        assert snr == pytest.approx(ref.detector_snrs(P, align)[kind], rel=1e-12)
        # the profile's own S/N on the predicted cells is the closed form
        num = sum(float(np.dot(w[c, :taps[c]].astype(np.float64), P[c, delay[c]:delay[c] + taps[c]]))
                  for c in range(C))
        den = math.sqrt(float((w.astype(np.float64) ** 2).sum()))
        assert num / den == pytest.approx(snr, rel=1e-6)


def test_dd_log_reports_plan_decisions(lib):
    """DD_LOG=1 makes the library log its plan decisions to stderr; without it, nothing."""
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "import numpy as np, paper_1301_3968_gb300 as dd\n"
            "p = dd.Plan(dd.Band(64, 1200., 4.6875, 1.0, 4096, 'u8'), np.linspace(0, 500, 128))\n"
            "p.set_method('runlength')\n" % ROOT)
    env = dict(os.environ, DD_LOG="1")
    on = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    assert on.returncode == 0, on.stderr
    lines = [ln for ln in on.stderr.splitlines() if ln.startswith("[dd] ")]
    assert any("exact integer sums" in ln and "128 trials x 64 channels" in ln for ln in lines), lines
    assert any("run-length sums" in ln for ln in lines), lines
    env.pop("DD_LOG")
    off = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    assert off.returncode == 0 and "[dd]" not in off.stderr
