"""Host logic of multi-GPU runs (independent replicas, one process per
GPU) with world size 2 on the CPU (gloo): the barrier, the maximum of the
per-rank times and the whole-job throughput; a rank that fails before the
timed region surfaces as an error in the other rank instead of a hang."""

import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q, fail_rank):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    try:
        import datetime
        import torch.distributed as dist
        from paper_1909_01149_gb300 import replicas
        if rank == fail_rank:
            raise RuntimeError("planted failure before the timed region")
        w, r, _ = replicas.world()
        dist.init_process_group("gloo", timeout=datetime.timedelta(seconds=20))
        replicas.barrier(w)
        elapsed = 10.0 + 5.0 * r          # this rank's "timed region" in ms
        mx = replicas.allreduce_max(elapsed, w, device="cpu")
        replicas.barrier(w)
        q.put((r, mx, replicas.job_throughput(100, w, mx)))
        replicas.teardown(w)
    except Exception as e:  # reported to the parent
        q.put((rank, "error", repr(e)[:200]))


def _run(ws, fail_rank=-1, timeout=120):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, ws, port, q, fail_rank)) for r in range(ws)]
    for p in ps:
        p.start()
    out = [q.get(timeout=timeout) for _ in range(ws)]
    for p in ps:
        p.join(timeout=timeout)
        if p.is_alive():
            p.kill()
    return sorted(out, key=lambda t: t[0])


def test_two_replicas_max_time_and_job_throughput():
    out = _run(2)
    assert [o[0] for o in out] == [0, 1]
    for r, mx, thr in out:
        assert mx == 15.0                       # max over ranks
        assert thr == pytest.approx(2 * 100 / 0.015)  # all ranks' units / slowest rank


def test_single_process_needs_no_group():
    from paper_1909_01149_gb300 import replicas
    assert replicas.allreduce_max(3.5, 1) == 3.5
    assert replicas.job_throughput(10, 1, 1000.0) == pytest.approx(10.0)


def test_failed_rank_surfaces_as_error_not_hang():
    out = _run(2, fail_rank=1, timeout=90)
    assert out[1][1] == "error" and "planted failure" in out[1][2]
    assert out[0][1] == "error"  # the survivor's rendezvous / collective times out
