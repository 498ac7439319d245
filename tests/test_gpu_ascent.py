"""Profile weights learned by gradient ascent through DDFunction (forward kernel +
adjoint kernels) approach the dynamic-spectrum matched filter bound of Sec. 5,
S/N <= sqrt(sum P̄²)/σ (Cauchy-Schwarz: the optimum weights are w ∝ P̄), and never
exceed it."""
import math

import numpy as np
import pytest

import synth
from oracle import ref

pytestmark = pytest.mark.gpu


def test_ascent_approaches_dsmf_bound():
    import torch
    from paper_1301_3968_gb300 import build
    build.build()
    import paper_1301_3968_gb300 as dd
    torch.cuda.set_device(0)
    # one steep-spectrum, scatter-broadened pulse, noise-free cells (eq. Pavg), unit cell noise
    b = synth.Band(64, 1200.0, 4.6875, 1.0)
    T, dm, t0 = 1024, 150.0, 300.0
    cells = synth.cell_average_pulse(b, T, dm, t0, synth.scattered_boxcar_profile(2.0, 3.0),
                                     amp=1.0, alpha=2.5, nu0_ghz=1.3)
    P = np.zeros((b.nchan, T), np.float32)
    synth.add_cells(P, cells)
    band = dd.Band(b.nchan, b.f_lo_mhz, b.df_mhz, b.dt_ms, T, "f32")
    plan = dd.Plan(band, [dm])
    delay, taps = plan.tables()
    K = 32
    # the trial's window per channel starts a few samples before the sweep and has 32 taps
    start = np.maximum(delay - 2, 0).astype(np.int32)
    plan.set_profiles(delay=start, taps=np.full_like(taps, K), weights=np.ones((1, b.nchan, K), np.float32))
    # every sample holding pulse power must lie inside the profile for the bound to be reachable
    t_peak = int(round(t0 / b.dt_ms)) - 2
    covered = 0.0
    for c in range(b.nchan):
        seg = P[c, t_peak + start[0, c]:t_peak + start[0, c] + K]
        covered += float((seg.astype(np.float64) ** 2).sum())
    bound = ref.dsmf_snr(P, 1.0)                      # sqrt(sum P̄²)/σ with σ = 1
    assert covered == pytest.approx(bound ** 2, rel=1e-6)

    x = torch.from_numpy(P).cuda()
    w = torch.full((1, b.nchan, K), 0.1, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([w], lr=0.02)
    snr = None
    for step in range(200):
        out = dd.DDFunction.apply(x, w, plan)
        s = out[0, t_peak] / torch.sqrt((w * w).sum())
        (-s).backward()
        opt.step()
        opt.zero_grad()
        snr = float(s.item())
        assert snr <= bound * (1 + 1e-5)
    assert snr >= 0.99 * bound
    # the learned weights point along P̄ (cosine similarity)
    wv = w.detach().cpu().numpy()[0]
    pv = np.stack([P[c, t_peak + start[0, c]:t_peak + start[0, c] + K] for c in range(b.nchan)])
    cos = float((wv * pv).sum() / (np.linalg.norm(wv) * np.linalg.norm(pv)))
    assert cos > 0.99
