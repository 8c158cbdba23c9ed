"""The benchmark's multi-rank host logic with two gloo ranks on the CPU
(one process per rank, as under torchrun): per-rank inputs are distinct
draws of the same shape (weak scaling), the step time is the maximum over
ranks, and the whole-job rate counts every rank's units."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms = [5.0, 7.5][rank]
    m = bench.max_over_ranks(ms, ws, torch.device("cpu"))
    rate = bench.job_rate(ws, 100, m)
    bench.N_KERNELS, bench.N_QUERIES = 4, 1000
    inst, q, gd = bench.make_inputs(bench.rank_seed(rank))
    digest = torch.tensor([float(inst["y"].astype("float64").sum()) + float(q[:, 0].sum())],
                          dtype=torch.float64)
    every = [torch.zeros(1, dtype=torch.float64) for _ in range(ws)]
    dist.all_gather(every, digest)
    out.put((rank, m, rate, tuple(inst["x"].shape), tuple(q.shape), [float(v) for v in every]))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    for rank, m, rate, xs, qs, digests in res:
        assert m == 7.5                                   # the slowest rank's time
        assert abs(rate - 2 * 100 / 7.5e-3) < 1e-6         # units of both ranks
        assert digests[0] != digests[1]                    # distinct draws
    assert res[0][3] == res[1][3] and res[0][4] == res[1][4]   # same shapes
