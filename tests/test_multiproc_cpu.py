"""The N > 1 path of bench.py on CPU: two gloo ranks (each takes a contiguous range of
the trial list, so the only collectives are the barrier, the max of the step time over
ranks and the gather of the peak tables after the timed region), the DM split merged on
rank 0 equal to one rank's result (oracle rows), the launcher that starts the ranks, and
the reference arm printing on rank 0 only."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    r, ws = bench._dist()
    assert (r, ws) == (rank, world) and dist.get_backend() == "gloo"
    bench._barrier(ws)
    m = bench._max_over_ranks(10.0 + rank, ws)     # per-rank step times 10 and 11 ms
    q.put((rank, m))
    dist.destroy_process_group()


def _free_port():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_gloo_ranks_take_the_max_step_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 11.0), (1, 11.0)]


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], env=env, capture_output=True,
                         text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0 and out.stdout.strip() == ""


@pytest.mark.slow
def test_reference_arm_json_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], env=env, capture_output=True,
                         text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle"


def _split_rank_main(rank, world, port, q):
    """One rank of a DM split on CPU: its cost-balanced trial range of a small plan,
    dedispersed and boxcar-scanned by the oracle over the whole list's output span, its
    peak tables gathered on rank 0 the way bench.py gathers them."""
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch.distributed as dist
    import bench
    from oracle import ref
    r, ws = bench._dist()
    I, delay, taps, w, widths = _split_case()
    t_out = I.shape[1] - ref.d_max(delay, taps)
    lo, hi = bench.dm_shards(taps.sum(axis=1), ws, align=4)[r]
    x = ref.dedisperse(I, delay[lo:hi], taps[lo:hi], w=w[lo:hi], nsamp=I.shape[1])[:, :t_out]
    mu_c, sd_c = ref.channel_stats(I)
    mu, sd = ref.boxcar_norm(taps[lo:hi], widths, mu_c, sd_c, w=w[lo:hi])
    peak, arg, _ = ref.boxcar_snr(x, widths, mu, sd)
    got = [None] * ws if r == 0 else None
    dist.gather_object((peak, arg, (lo, hi)), got, dst=0)
    if r == 0:
        q.put(got)
    dist.destroy_process_group()


def _split_case():
    import numpy as np
    from oracle import ref
    rng = np.random.default_rng(77)
    C, T, D, K = 16, 900, 24, 8
    I = rng.standard_normal((C, T)).astype(np.float32)
    dms = np.linspace(0.0, 300.0, D)
    delay, _ = ref.delay_table(dms, C, 1200.0, 4.0, 1.0)
    taps, _ = ref.taps_table(dms, C, 1200.0, 4.0, 1.0)
    w = rng.uniform(0.5, 1.5, size=(D, C, int(taps.max()))).astype(np.float32)
    return I, delay, taps, w, [1, 2, 3, 4, 6, 8]


def test_dm_split_merged_on_rank_zero_equals_one_rank():
    import numpy as np
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import bench
    from oracle import ref
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    I, delay, taps, w, widths = _split_case()
    # ranges are contiguous, cover the list and are balanced by taps
    ranges = [g[2] for g in got]
    assert ranges[0][0] == 0 and ranges[0][1] == ranges[1][0] and ranges[1][1] == len(delay)
    cost = [int(taps[lo:hi].sum()) for lo, hi in ranges]
    assert abs(cost[0] - cost[1]) <= 0.25 * sum(cost)
    x = ref.dedisperse(I, delay, taps, w=w)
    mu_c, sd_c = ref.channel_stats(I)
    mu, sd = ref.boxcar_norm(taps, widths, mu_c, sd_c, w=w)
    peak, arg, _ = ref.boxcar_snr(x, widths, mu, sd)
    np.testing.assert_array_equal(np.concatenate([g[0] for g in got]), peak)
    np.testing.assert_array_equal(np.concatenate([g[1] for g in got]), arg)


def test_dm_shards_cover_and_align():
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    cost = np.linspace(1.0, 30.0, 4096)
    for ws in (1, 2, 3, 4, 8):
        sh = bench.dm_shards(cost, ws)
        assert sh[0][0] == 0 and sh[-1][1] == 4096
        assert all(a[1] == b[0] for a, b in zip(sh, sh[1:]))
        assert all(lo % 16 == 0 for lo, _ in sh)
        share = [cost[lo:hi].sum() / cost.sum() for lo, hi in sh]
        assert max(share) - min(share) < 0.02


def test_launcher_starts_ranks_and_rank_zero_prints_one_line():
    """`bench.py --gpus 2` with no launcher around it starts two ranks itself; on the
    reference arm rank 0 prints the one JSON line and the other rank exits 0."""
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2", "--impl",
                          "reference", "--steps", "1", "--warmup", "0"], env=env, capture_output=True,
                         text=True, timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0
