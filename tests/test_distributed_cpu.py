"""The multi-rank plumbing of bench.py on CPU ranks (gloo, world size 2):
every rank advances its own replica, so the only reduction is the
max-over-ranks of the timed region; the reference arm runs on rank 0 only."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

import bench


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 7.5 * rank                  # the slower rank sets the job time
    m = bench.max_over_ranks(ms, world, "cpu")
    zones, steps = 1000, 4
    q.put((rank, m, world * zones * steps / (m * 1e-3)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=5) for _ in range(2))
    assert [o[1] for o in out] == [17.5, 17.5]
    assert all(abs(o[2] - 2 * 1000 * 4 / 17.5e-3) < 1e-6 for o in out)


def test_max_over_ranks_single_rank_is_identity():
    assert bench.max_over_ranks(3.25, 1, "cpu") == 3.25


def test_reference_arm_only_rank0_prints(monkeypatch):
    """Under torchrun the reference arm (the CPU oracle) runs on rank 0 alone;
    other ranks exit 0 without output."""
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.main() == 0
    assert buf.getvalue() == ""


@pytest.mark.slow
def test_reference_arm_rank0_json_line(monkeypatch):
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.main() == 0
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "zone-cycles/s" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
