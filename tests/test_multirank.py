"""The multi-rank path of the benchmark on CPU ranks (gloo, world size 2):
every rank takes a distinct shot, the ranks exchange nothing but the step
time, and the reported time is the slowest rank's."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rk, ws, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rk), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rk))
    dist.init_process_group("gloo", rank=rk, world_size=ws)
    try:
        w_rk, r_rk, l_rk = bench.dist_env()
        src = bench.rank_source((30.0, 960.0, 960.0), r_rk, w_rk)
        ms = bench.max_over_ranks(10.0 + 5.0 * rk, "cpu")
        srcs = [None] * ws
        dist.all_gather_object(srcs, src)
        out.put((rk, w_rk, src, ms, srcs))
    finally:
        dist.destroy_process_group()


def test_two_cpu_ranks_take_distinct_shots_and_report_the_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res.sort()
    assert [r[1] for r in res] == [2, 2]
    srcs = res[0][4]
    assert srcs[0] != srcs[1]
    assert res[0][2] == srcs[0] and res[1][2] == srcs[1]
    assert res[0][3] == res[1][3] == 15.0


def test_single_rank_is_unchanged():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.max_over_ranks(12.5, "cpu") == 12.5
    assert bench.rank_source((1.0, 2.0, 4.0), 0, 1) == (1.0, 2.0, 4.0)
