"""Failure detection without a GPU fault: a bulk-copy stage that is never issued makes
the dedispersion kernel's bounded barrier wait run out; the kernel records
DD_ERR_TIMEOUT, drains its own copies and returns, and the context stays usable."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_recovers():
    import torch
    from paper_1301_3968_gb300 import build
    build.build()
    import paper_1301_3968_gb300 as dd
    rng = np.random.default_rng(21)
    C, T, D = 40, 3008, 16
    I = rng.integers(0, 256, size=(C, T)).astype(np.uint8)
    delay = rng.integers(0, 100, size=(D, C)).astype(np.int32)
    taps = rng.integers(1, 6, size=(D, C)).astype(np.int32)
    plan = dd.Plan(dd.Band(C, 1200.0, 1.0, 1.0, T, "u8"), np.zeros(D))
    plan.set_profiles(delay=delay, taps=taps)
    x = torch.from_numpy(I).cuda()
    assert plan.device_status() == 0
    plan.test_set_wait(skip_stage=1, wait_ns=50_000_000)      # 50 ms
    plan.dedisperse(x, nsamp=T)
    assert plan.device_status() == 6                           # DD_ERR_TIMEOUT
    assert plan.device_status() == 0                           # cleared
    plan.test_set_wait(-1, 0)
    out = plan.dedisperse(x, nsamp=T).cpu().numpy()
    assert plan.device_status() == 0
    np.testing.assert_array_equal(out.astype(np.int64), oracle.c_dedisperse(I, delay, taps, nsamp=T))
