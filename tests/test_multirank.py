"""Host logic of the multi-GPU benchmark (independent replicas, one process
per GPU), run as two gloo ranks on the CPU: the slowest rank's durations
bound the job and the throughput counts the units of every rank."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench as b

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = b._dist()
        # rank r took (r + 1) ms for the device loop and (5 - r) s end to end
        el_ms, e2e_s = b.aggregate_over_ranks([1.0 + r, 5.0 - r])
        rate = b.job_rate(4096 * 10, el_ms / 1e3, ws)
        with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
            json.dump({"ws": ws, "rank": r, "local": local, "el_ms": el_ms, "e2e_s": e2e_s, "rate": rate}, f)
    finally:
        dist.destroy_process_group()


def test_aggregate_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp

    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    for p in procs:
        if p.is_alive():
            p.kill()
            pytest.fail("gloo rank did not finish")
        assert p.exitcode == 0
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(world)]
    for r, x in enumerate(res):
        assert (x["ws"], x["rank"], x["local"]) == (world, r, r)
        # the maximum over ranks, the same on every rank
        assert x["el_ms"] == 2.0 and x["e2e_s"] == 5.0
        # both ranks' products over the slowest rank's time
        assert x["rate"] == pytest.approx(2 * 4096 * 10 / 2e-3)


def test_aggregate_single_process_is_identity():
    assert bench.aggregate_over_ranks([3.5, 7.25]) == [3.5, 7.25]


def test_job_rate():
    assert bench.job_rate(100, 2.0, 4) == 200.0
    with pytest.raises(ValueError):
        bench.job_rate(1, 0.0, 1)


def test_reference_arm_other_ranks_do_nothing(capsys):
    class A:
        steps, warmup, gpus = 1, 0, 2

    assert bench.run_reference(A(), 2, 1) is None
    assert capsys.readouterr().out == ""
