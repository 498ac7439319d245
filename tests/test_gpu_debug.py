"""The debug build (libdd_debug.so: bounds checks on every staged window and output store
of the dedispersion (plain, batched and fused) and boxcar kernels, recording DD_ERR_ARG in
the plan's device status word instead of faulting) on small cases of every path: status 0
and results equal to the oracle (the fused scan: equal to the unfused path).  Runs in a child process, since a process loads one of the two libraries."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_clean_on_every_path():
    from paper_1301_3968_gb300 import build
    build.build()
    env = dict(os.environ, DD_DEBUG_LIB="1")
    res = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_debug_build_cases.py")],
                         env=env, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-3000:]
    cases = {d["case"]: d for d in (json.loads(ln) for ln in res.stdout.splitlines() if ln.startswith("{"))}
    assert set(cases) == {"plain_int_w16", "plain_int_w6", "craft_f32_pairs", "craft_f32_adjoint",
                          "runlength_rows", "runlength_pairs", "fused_u8", "fused_f32"}
    for name, d in cases.items():
        assert d["status"] == 0, (name, d)
        if name.startswith("fused"):
            assert d["err"] == 0.0, (name, d)        # fused = unfused, bit for bit
        elif name.startswith("plain_int") or name.startswith("runlength"):
            assert d["err"] < 1e-5, (name, d)        # integer sums exact, S/N to 1e-5
        else:
            assert d["err"] < 1e-5, (name, d)        # fp32: scale-aware 1e-5
