"""The multi-rank path of bench.py on CPU: two gloo ranks (one process per
rank, rendezvous on 127.0.0.1) combine their local timings the way the GPU
ranks do under NCCL: the slowest rank's time and the sum of the units; the
reference arm runs on rank 0 only."""
import os
import socket
import sys
from pathlib import Path

import pytest

torch = pytest.importorskip("torch")
ROOT = Path(__file__).resolve().parents[1]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, str(ROOT))
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rmax, rsum = bench.reducers(dist, "cpu")
    # rank r took (r + 1) s for 100 (r + 1) lattice updates
    value, t, u = bench.aggregate(float(rank + 1), 100.0 * (rank + 1), world, rmax, rsum)
    out.put((rank, value, t, u, bench.dist_env()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t, u, env in res:
        assert t == 2.0 and u == 300.0 and value == 150.0   # slowest rank, summed units
        assert env == (rank, 2, rank)


def test_reference_arm_other_ranks_exit(monkeypatch):
    """Under torchrun only rank 0 times the oracle; the other ranks return 0
    at once without work."""
    sys.path.insert(0, str(ROOT))
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]) == 0


def test_single_process_reducers_are_identity():
    sys.path.insert(0, str(ROOT))
    import bench

    rmax, rsum = bench.reducers(None, "cpu")
    assert bench.aggregate(2.0, 10.0, 1, rmax, rsum) == (5.0, 2.0, 10.0)


def test_bench_calls_only_defined_functions():
    """Every module-level function bench.py calls by bare name is defined in it
    or imported (a static check: the GPU arms cannot run here)."""
    import ast
    import builtins

    src = (Path(__file__).resolve().parents[1] / "bench.py").read_text()
    tree = ast.parse(src)
    known = set(dir(builtins))
    for node in ast.walk(tree):
        if isinstance(node, (ast.FunctionDef, ast.ClassDef)):
            known.add(node.name)
        elif isinstance(node, (ast.Import, ast.ImportFrom)):
            known.update((a.asname or a.name).split(".")[0] for a in node.names)
        elif isinstance(node, ast.Name) and isinstance(node.ctx, ast.Store):
            known.add(node.id)
        elif isinstance(node, ast.arg):
            known.add(node.arg)
    called = {n.func.id for n in ast.walk(tree) if isinstance(n, ast.Call) and isinstance(n.func, ast.Name)}
    assert not called - known, sorted(called - known)


@pytest.mark.parametrize("workload", ["pulses", "hole"])
def test_reference_arm_line(workload, capsys, monkeypatch):
    """The reference arm (the FP64 oracle on the host cores) prints one JSON
    line with the base contract's keys, on a small lattice."""
    import json

    sys.path.insert(0, str(ROOT))
    import bench

    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    assert bench.main(["--impl", "reference", "--workload", workload, "--size", "96", "--steps", "2",
                       "--warmup", "1", "--ref-seconds", "0.2"]) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GLUPS" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == f"{workload}_96"
