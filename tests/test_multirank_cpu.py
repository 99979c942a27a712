"""The multi-GPU path shards independent queries across ranks (weak
scaling, no collective on the data path): with two gloo ranks on the CPU,
each rank gets its own query mix, the barrier works and the step time is the
max over ranks; the oracle reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    qs = bench.rank_queries(8, rank)
    sig = [(q.K, q.C, round(float(q.logits[0, 0]), 6)) for q in qs]
    bench.barrier(world)
    t = bench.max_over_ranks(world, 10.0 + rank, device="cpu")
    out[rank] = (sig, t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_queries_and_take_max_time():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        r0, r1 = out[0], out[1]
    assert r0[0] != r1[0], "ranks must get different query mixes"
    assert r0[1] == r1[1] == 11.0


def test_reference_arm_prints_on_rank0_only(monkeypatch, capsys):
    """Rank 0 alone runs the oracle reference arm (a fake pool stands in for
    the host-core workers); its line has real step times and the same
    cpu_baseline fields as the GPU arm's."""
    sys.path.insert(0, ROOT)
    import json
    import bench

    class A:
        queries, steps, warmup, gpus, params = 4, 2, 1, 2, "argmax8"
    called = []

    class FakePool:
        def map(self, fn, jobs, chunksize=1):
            called.append(len(jobs))
            return [0.5] * len(jobs)

        def close(self):
            pass

        def join(self):
            pass

    monkeypatch.setattr(bench, "oracle_pool", lambda cores: FakePool())
    monkeypatch.setattr(bench, "oracle_whole_queries",
                        lambda pool, cores, params: {"t_query": 40.0, "ks_query": 35, "refreshes": 1, "wall": 45.0})
    bench.run_reference(A, 2, 1)
    assert capsys.readouterr().out == "" and not called
    bench.run_reference(A, 2, 0)
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference" and len(called) == A.warmup + A.steps
    cores = line["cpu_baseline"]["cores"]
    relin, rot = bench.op_mix_per_query(bench.workloads_argmax_queries(A.queries))
    assert abs(line["value"] - cores * 35 / ((relin + rot) * 40.0)) < 1e-12
    assert line["cpu_baseline"]["value"] == line["value"] and line["e2e"]["value"] == line["value"]
