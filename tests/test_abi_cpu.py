"""C-ABI library on the CPU: it loads, exports every declared symbol, and its host
logic (profile tables, trial DMs, argument checking) matches the oracle.  No device
compute runs here."""
import ctypes
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
