"""Small cases run against the debug build of the library (bounds checks in the kernels
that record DD_ERR_ARG in the plan's device status word).  Executed as a child process
by tests/test_gpu_debug.py with DD_DEBUG_LIB=1, so that the debug library is the one
loaded; prints one JSON line per case: its device status and its largest difference from
the oracle."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
from oracle import ref  # noqa: E402
import synth  # noqa: E402


def _emit(case, status, err, **kw):
    print(json.dumps({"case": case, "status": int(status), "err": float(err), **kw}), flush=True)


def main():
    from paper_1301_3968_gb300 import _lib
    assert _lib.load()._name.endswith("libdd_debug.so"), _lib.load()._name
    import paper_1301_3968_gb300 as dd
    torch.cuda.set_device(0)
    # 1. the plain configuration: exact integer path, dedispersion and boxcar
    cfg = synth.make_plain()
    b = cfg["band"]
    plan = dd.Plan(dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, cfg["nsamp"], "u8"), cfg["dms"])
    x = torch.from_numpy(cfg["data"]).cuda()
    out = plan.dedisperse(x, nsamp=cfg["nsamp"])
    mean, sd = plan.channel_stats(x, nsamp=cfg["nsamp"])
    for widths in (np.arange(1, 17, dtype=np.int32), np.array([1, 2, 3, 5, 8, 13], np.int32)):
        peak, arg, _ = plan.boxcar_snr(out, widths, mean, sd)
        delay, taps = plan.tables()
        want = oracle.c_dedisperse(cfg["data"], delay, taps, nsamp=cfg["nsamp"])
        mu_c, sd_c = ref.channel_stats(cfg["data"], nsamp=cfg["nsamp"])
        mu, sdw = ref.boxcar_norm(taps, widths, mu_c, sd_c)
        opeak, _, _ = ref.boxcar_snr(want, widths, mu, sdw)
        err = max(float(np.abs(out.cpu().numpy().astype(np.int64) - want).max()),
                  float(np.abs(peak.cpu().numpy() - opeak).max() / max(1.0, np.abs(opeak).max())))
        _emit(f"plain_int_w{len(widths)}", plan.device_status(), err)
    plan.close()
    # 2. fp32 weighted pair units on 64 trials of the CRAFT-like band (shifted windows)
    cb = synth.CRAFT_BAND
    T = 8192
    band = dd.Band(cb.nchan, cb.f_lo_mhz, cb.df_mhz, cb.dt_ms, T, "f32")
    dms, _ = dd.trial_dms(band, 0.0, 1500.0, 64, tau_av_ms=1.0)
    plan = dd.Plan(band, dms)
    delay, taps = plan.tables()
    K = int(taps.max())
    w = np.where(np.arange(K)[None, None, :] < taps[:, :, None],
                 synth.spectral_weights(cb)[None, :, None], 0.0).astype(np.float32)
    plan.set_profiles(weights=w)
    rng = np.random.default_rng(5)
    I = rng.standard_normal((cb.nchan, T)).astype(np.float32)
    xf = torch.from_numpy(I).cuda()
    out = plan.dedisperse(xf, nsamp=T).cpu().numpy()
    want = oracle.c_dedisperse(I, delay, taps, w=w, nsamp=T)
    scale = oracle.c_abs_scale(I, delay, taps, w=w, nsamp=T)
    _emit("craft_f32_pairs", plan.device_status(), float(np.max(np.abs(out - want) / scale)))
    # adjoint: weight gradient at sampled points against the oracle's
    g = torch.from_numpy(rng.standard_normal(out.shape).astype(np.float32)).cuda()
    gw, gi = plan.backward(xf, g, nsamp=T)
    ogw, _ = oracle.c_adjoint(I, g.cpu().numpy(), delay, taps, w)
    gwn = gw.cpu().numpy()[:, :, :ogw.shape[2]]
    _emit("craft_f32_adjoint", plan.device_status(),
          float(np.max(np.abs(gwn - ogw)) / max(1.0, float(np.max(np.abs(ogw))))))
    plan.close()
    # 3. run-length sums, with and without difference rows shared by the CTA
    for share in (True, False):
        Tl = 20000
        dms = np.linspace(0.0, 100.0, 380 if share else 48)
        plan = dd.Plan(dd.Band(256, 700.0, 300.0 / 1024, 0.064, Tl, "u8"), dms)
        plan.set_method("runlength")
        data = np.zeros((256, Tl), np.uint8)
        data[:] = rng.integers(0, 256, size=(256, Tl))
        out = plan.dedisperse(torch.from_numpy(data).cuda(), nsamp=Tl).cpu().numpy()
        delay, taps = plan.tables()
        rows = [0, len(dms) // 2, len(dms) - 1]
        want = oracle.c_dedisperse(data, delay, taps, nsamp=Tl, rows=rows)
        _emit(f"runlength_{'rows' if share else 'pairs'}", plan.device_status(),
              float(np.abs(out[rows].astype(np.int64) - want).max()))
        plan.close()
    # 4. the fused boxcar scan on an integer and an fp32 plan (five parts, so seams too):
    # err 0 when its peaks and starts equal the unfused path's bit for bit
    for kind in ("u8", "f32"):
        C, T, D = 24, 6000, 30
        plan = dd.Plan(dd.Band(C, 1200.0, 1.0, 1.0, T, kind), np.zeros(D))
        delay = rng.integers(0, 300, size=(D, C)).astype(np.int32)
        taps = rng.integers(1, 20, size=(D, C)).astype(np.int32)
        w = None if kind == "u8" else (rng.standard_normal((D, C, 19)) * 0.5 + 1.0).astype(np.float32)
        plan.set_profiles(delay=delay, taps=taps, weights=w)
        if kind == "u8":
            data = rng.integers(0, 256, size=(C, T)).astype(np.uint8)
        else:
            data = rng.standard_normal((C, T)).astype(np.float32)
        x = torch.from_numpy(data).cuda()
        mean, sd = plan.channel_stats(x, nsamp=T)
        widths = np.arange(1, 33, dtype=np.int32)
        plan.test_set_fused_parts(5)
        out = plan.dedisperse(x, nsamp=T)
        p0, a0, _ = plan.boxcar_snr(out, widths, mean, sd)
        p1, a1, _ = plan.dedisperse_boxcar(x, widths, mean, sd, nsamp=T)
        same = (np.array_equal(p0.cpu().numpy().view(np.int32), p1.cpu().numpy().view(np.int32))
                and np.array_equal(a0.cpu().numpy(), a1.cpu().numpy()))
        _emit(f"fused_{kind}", plan.device_status(), 0.0 if same else 1.0)
        plan.close()


if __name__ == "__main__":
    main()
