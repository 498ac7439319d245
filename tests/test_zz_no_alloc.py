"""The allocation-free boxcar S/N entry point (dd_boxcar_snr_noalloc).

Some callers may not allocate device memory while running, e.g. a real-time pipeline
that fixes its device footprint at start-up.  This entry point keeps its scratch in a
fixed device array inside the library; here its results are checked against
dd_boxcar_snr on two calls in a row, through the C ABI, and the device's free memory
is checked to stay the same across calls (the first one included).  The file is named
so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_boxcar_matches_allocating_entry_point():
    import torch
    from paper_1301_3968_gb300 import build
    build.build()
    import paper_1301_3968_gb300 as dd
    torch.cuda.set_device(0)
    results = []
    for seed, weighted in ((1, False), (2, True)):
        cfg = synth.make_plain(seed=synth.sub_seed("tests", 40 + seed), snr_total=16.0)
        b = cfg["band"]
        in_type = "f32" if weighted else "u8"
        data = cfg["data"].astype(np.float32) if weighted else cfg["data"]
        plan = dd.Plan(dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, cfg["nsamp"], in_type), cfg["dms"])
        if weighted:
            d, t = plan.tables()
            K = int(t.max())
            w = np.random.default_rng(seed).uniform(0.5, 1.5, size=(len(cfg["dms"]), b.nchan, K))
            plan.set_profiles(weights=w.astype(np.float32))
        x = torch.from_numpy(data).cuda()
        out = plan.dedisperse(x, nsamp=cfg["nsamp"])
        mean, sd = plan.channel_stats(x, nsamp=cfg["nsamp"])
        widths = np.arange(1, 17, dtype=np.int32)
        want_p, want_a, want_c = plan.boxcar_snr(out, widths, mean, sd, thresh=6.0, cap=1024)
        want = sorted((dm, j, t) for dm, j, t, _ in dd.candidates_to_list(want_c))
        for call in range(2):
            peak = torch.full_like(want_p, -1.0)
            arg = torch.full_like(want_a, -1)
            cands = torch.zeros((1024, 4), dtype=torch.int32, device="cuda")
            ncand = torch.zeros(1, dtype=torch.int32, device="cuda")
            plan.boxcar_snr_noalloc(out, widths, mean, sd, peak, arg, thresh=6.0, cands=cands, ncand=ncand)
            torch.cuda.synchronize()
            np.testing.assert_allclose(peak.cpu().numpy(), want_p.cpu().numpy(), rtol=1e-5, atol=1e-5)
            np.testing.assert_array_equal(arg.cpu().numpy(), want_a.cpu().numpy())
            got = sorted((dm, j, t) for dm, j, t, _ in dd.candidates_to_list((cands, ncand)))
            assert got == want and len(want) > 0
            results.append(call)
        plan.close()
    assert len(results) == 4


def test_noalloc_rejects_oversize_and_missing_tables():
    import torch
    from paper_1301_3968_gb300 import build
    build.build()
    import paper_1301_3968_gb300 as dd
    from paper_1301_3968_gb300 import _lib
    lib = _lib.load()
    C, T, D = 4, 512, 4096
    plan = dd.Plan(dd.Band(C, 1200.0, 1.0, 1.0, T, "u8"), np.zeros(D))
    x = torch.zeros((C, T), dtype=torch.uint8, device="cuda")
    series = torch.zeros((D, T), dtype=torch.int32, device="cuda")
    mean = torch.zeros(C, dtype=torch.float64, device="cuda")
    peak = torch.zeros((D, 256), dtype=torch.float32, device="cuda")
    arg = torch.zeros((D, 256), dtype=torch.int32, device="cuda")
    wl = np.arange(1, 257, dtype=np.int32)

    def call(nw):
        return lib.dd_boxcar_snr_noalloc(plan._h, ctypes.c_void_p(series.data_ptr()), T, T,
                                         ctypes.c_void_p(wl.ctypes.data), nw,
                                         ctypes.c_void_p(mean.data_ptr()), ctypes.c_void_p(mean.data_ptr()),
                                         ctypes.c_void_p(peak.data_ptr()), ctypes.c_void_p(arg.data_ptr()),
                                         ctypes.c_float(1.0), None, 0, None,
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert call(8) == 5                      # DD_ERR_STATE: tables not on the device yet
    plan.dedisperse(x, nsamp=T)
    torch.cuda.synchronize()
    assert call(256) == 7                    # DD_ERR_CAPACITY: 4096 x 256 does not fit 8 MiB
    assert call(8) == 0
    torch.cuda.synchronize()


def test_noalloc_calls_leave_device_memory_unchanged():
    """Back-to-back calls on one stream, with different plans and width lists sharing the
    scratch array, change the device's free memory by nothing (the first call after the
    plans' tables went to the device included) and each matches dd_boxcar_snr."""
    import torch
    from paper_1301_3968_gb300 import build
    build.build()
    import paper_1301_3968_gb300 as dd
    torch.cuda.set_device(0)
    cases = []
    for seed, weighted, widths in ((5, False, np.arange(1, 17, dtype=np.int32)),
                                   (6, True, np.array([1, 2, 3, 5, 8, 13, 21], dtype=np.int32))):
        cfg = synth.make_plain(seed=synth.sub_seed("tests", 50 + seed), snr_total=16.0)
        b = cfg["band"]
        data = cfg["data"].astype(np.float32) if weighted else cfg["data"]
        plan = dd.Plan(dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, cfg["nsamp"],
                               "f32" if weighted else "u8"), cfg["dms"])
        if weighted:
            _, t = plan.tables()
            w = np.random.default_rng(seed).uniform(0.5, 1.5, size=(len(cfg["dms"]), b.nchan, int(t.max())))
            plan.set_profiles(weights=w.astype(np.float32))
        x = torch.from_numpy(data).cuda()
        out = plan.dedisperse(x, nsamp=cfg["nsamp"])           # puts the tables on the device
        mean, sd = plan.channel_stats(x, nsamp=cfg["nsamp"])
        peak = torch.full((plan.ndm, len(widths)), -1.0, dtype=torch.float32, device="cuda")
        arg = torch.full((plan.ndm, len(widths)), -1, dtype=torch.int32, device="cuda")
        cases.append((plan, out, mean, sd, widths, peak, arg))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for rep in range(2):
        for plan, out, mean, sd, widths, peak, arg in cases:   # no synchronisation between calls
            plan.boxcar_snr_noalloc(out, widths, mean, sd, peak, arg)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, f"free device memory changed (pass {rep})"
    for plan, out, mean, sd, widths, peak, arg in cases:
        want_p, want_a, _ = plan.boxcar_snr(out, widths, mean, sd)
        np.testing.assert_allclose(peak.cpu().numpy(), want_p.cpu().numpy(), rtol=1e-5, atol=1e-5)
        np.testing.assert_array_equal(arg.cpu().numpy(), want_a.cpu().numpy())
        plan.close()
