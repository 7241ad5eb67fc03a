"""The bench's multi-rank host logic on CPU: two gloo ranks, each with its
own measured time, agree on the slowest rank's time and report the job's
seconds per solve over all ranks' solves (replicas, weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_init() == (ws, rank, rank)
        local = [300.0, 450.0][rank]
        elapsed, value = bench.job_time(local, 3, ws, torch, device="cpu")
        out.put((rank, elapsed, value))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(out.get(timeout=10) for _ in range(2))
    for rank, elapsed, value in res:
        assert elapsed == 450.0
        assert value == pytest.approx(450.0 / 1e3 / (3 * 2))


def test_single_rank_job_time():
    import bench
    elapsed, value = bench.job_time(120.0, 4, 1, torch, device="cpu")
    assert elapsed == 120.0 and value == pytest.approx(0.03)


def test_traffic_records_name_existing_kernels():
    """Every DRAM-traffic record names source files and device functions that
    exist (each function found once), so its source hash can be checked; a
    record whose kernel changed is ignored by the bench (hash mismatch), not
    misattributed."""
    import json
    import os
    import re
    import bench
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "profiles", "traffic.json")) as fh:
        records = json.load(fh)
    csrc = os.path.join(root, "paper_2606_13429_gb300", "csrc")
    for cls, ent in records.items():
        assert ent["dram_bytes_per_launch"] > 0, cls
        for fn in ent.get("source_files", []):
            text = open(os.path.join(csrc, fn), encoding="utf-8").read()
            for name in ent.get("functions", []):
                found = re.findall(r"^(?:template <[^\n]*>\n)?(?:__global__|__device__)[^\n]*\b%s\(" % re.escape(name),
                                   text, re.M)
                assert len(found) == 1, (cls, name, len(found))
        h = bench.kernel_source_hash(ent.get("source_files"), ent.get("functions"))
        assert isinstance(h, str) and len(h) == 16
