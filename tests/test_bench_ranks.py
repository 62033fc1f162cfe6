"""The benchmark's multi-rank logic on CPU: two gloo ranks (world size 2)
reduce their step times to the maximum, sum their domain counts, compute the
whole-job value, and only rank 0 of the reference arm prints."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = bench.rank_env()
    t = bench.max_over_ranks(1.5 + rank, w)
    out[rank] = (w, r, lr, t, bench.job_value(300, w, t), bench.sum_over_ranks(10 + rank, w))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        w, r, lr, t, v, n = out[rank]
        assert (w, r, lr) == (2, rank, rank)
        assert t == 2.5                      # max over ranks
        assert v == pytest.approx(2 * 300 / 2.5)
        assert n == 21                       # sum over ranks (slab domain counts)


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--gpus", "2"],
                       capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.job_value(300000, 1, 4.0) == 75000.0
    line = bench.workload_config(__import__("synth").configs.crs_line(0, n_cmp=3, ns=120, tau_max=0.4), 2)
    assert "replicas x2" in json.dumps(line)


def test_recovery_metric_counts_exact_truth():
    """bench.recovery: the exact recentred parameters at every domain count
    as recovered in A, B and C; a 2% error in C, or an error of 2% of B's
    bound range, does not (and only the parameter it was put in fails)."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    import synth
    from synth import configs
    wl = configs.crs_line(2, n_cmp=100, ns=400, n_events=10, tau_max=1.4)
    p = wl.problem
    th = np.zeros((p.n_dom, 3))
    for ev in wl.line.events:
        for c in range(wl.line.n_cmp):
            tr = synth.crs_recentre(ev, wl.line.cmp_x[c])
            if tr is None:
                continue
            it = int(round(tr[0] / wl.dt))
            if 0 <= it < p.n_t0:
                th[c * p.n_t0 + it] = (tr[1], tr[2], tr[3])
    r = bench.recovery(wl, th)
    n = r["of"]
    assert r is not None and n >= 1
    assert r["within_1pct"] == {"A": n, "B": n, "C": n, "all": n}
    assert r["B_edge_shift_samples"]["max"] < 1e-6
    tb = th.copy()
    tb[:, 1] += 0.02 * (configs.CRS_HI[1] - configs.CRS_LO[1])
    assert bench.recovery(wl, tb)["within_1pct"] == {"A": n, "B": 0, "C": n, "all": 0}
    th[:, 2] *= 1.02
    assert bench.recovery(wl, th)["within_1pct"] == {"A": n, "B": n, "C": 0, "all": 0}


def test_member_order_reading_for_the_traffic_figure():
    """bench.member_order_on reads the context's option and, for "auto",
    applies the library's rule (members in window order when the apertures
    hold at least 768 traces on average), so that `roofline.traffic` is
    reported only for the launch form its DRAM capture was taken in."""
    sys.path.insert(0, ROOT)
    import types

    import numpy as np

    import bench

    class FakeTT:
        def __init__(self, value):
            self.value = value

        def tt_ctx_get_option(self, ctx, option):
            assert option == "member_order"
            return self.value

    def problem(aps, per_group=3):
        ptr = np.concatenate([[0], np.cumsum(aps)]).astype(np.int32)
        return types.SimpleNamespace(ap_ptr=ptr,
                                     dom_group=np.repeat(np.arange(len(aps)), per_group))

    long_ap, short_ap = problem([800, 760, 780]), problem([700, 760, 790])
    assert bench.member_order_on(FakeTT("auto"), None, long_ap) is True    # mean 780
    assert bench.member_order_on(FakeTT("auto"), None, short_ap) is False  # mean 750
    assert bench.member_order_on(FakeTT(True), None, short_ap) is True
    assert bench.member_order_on(FakeTT(False), None, long_ap) is False
    assert bench.member_order_on(FakeTT("auto"), None, problem([], 0)) is False
    assert bench.K1_LINE_DRAM_MEMBER_ORDER is True  # the committed capture's form
