"""The grouped search path (queries bucketed by kernel id on the device,
each kernel's table staged in shared memory) against the direct path
(every query gathers its table rows from global memory): identical outputs,
bit for bit, on the same program and queries -- both evaluate each
(query, configuration) with the same arithmetic, only the memory the
coefficients come from differs.  The direct path itself is checked against
the FP64 oracle in test_gpu_search.py (which runs grouped wherever the
sizes select it).

Cases: every degree; queries in kernel order and shuffled; out-of-range
kernel ids, non-finite and out-of-domain fields (bucket K, status BAD);
kernels without queries; tile tails (Q not a multiple of any launch
shape); more buckets than the shared-memory histogram holds (global
atomics).
"""
import numpy as np
import pytest
import torch

import paper_1906_00142_gb300 as rp
import workloads as W
from gpu_util import dev, host, need_gpu, program_to_device

pytestmark = pytest.mark.gpu


def both_paths(buf, K, d, q):
    assert rp.rp_search_workspace_size(K, q.shape[0]) > 0      # the grouped path is taken
    a = {k: host(v) for k, v in rp.rp_eval_search(buf, K, d, q, grouped=False).items()}
    b = {k: host(v) for k, v in rp.rp_eval_search(buf, K, d, q, grouped=True).items()}
    return a, b


def assert_same(a, b):
    assert np.array_equal(a["argmin"], b["argmin"])
    assert np.array_equal(a["status"], b["status"])
    assert np.array_equal(a["best"], b["best"], equal_nan=True)
    assert np.array_equal(a["second"], b["second"], equal_nan=True)


def edge_rows(q, K, rng):
    """Overwrite scattered rows with the query edge cases."""
    q = q.copy()
    n = len(q)
    rows = rng.choice(n, 64, replace=False)
    kid = W.query_kernel_ids(q).copy()
    kid[rows[:8]] = -1                         # kernel id out of range
    kid[rows[8:16]] = K
    kid[rows[16:20]] = 2 ** 30
    q[:, W.Q_KID] = kid.view(np.float32)
    q[rows[20:24], W.Q_N] = np.nan             # non-finite field
    q[rows[24:28], W.Q_BW] = np.inf
    q[rows[28:32], W.Q_N] = 0.5                # N < 1
    q[rows[32:36], W.Q_NSM] = 0.0              # no SMs
    q[rows[36:40], W.Q_FGHZ] = -1.0            # non-positive clock
    q[rows[40:44], W.Q_N] = 2.0 ** 32          # N beyond 2^32 - 256
    return q


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_grouped_equals_direct(d):
    need_gpu()
    K = 8
    prog = W.synthetic_program(K, d, seed=300 + d)
    buf = program_to_device(prog)
    rng = np.random.default_rng(d)
    q = edge_rows(W.queries(20000 + 37, K, seed=400 + d), K, rng)
    for order in ("sorted", "shuffled"):
        qq = q if order == "sorted" else q[rng.permutation(len(q))]
        a, b = both_paths(buf, K, d, dev(qq))
        assert_same(a, b)
        st = a["status"]
        assert (st & rp.RP_Q_BAD).sum() >= 44


def test_grouped_kernels_without_queries_and_one_dominant_kernel():
    """Buckets that are empty, and one kernel holding most queries (runs
    that span many tiles), with the others in short runs."""
    need_gpu()
    K, d = 64, 3
    prog = W.synthetic_program(K, d, seed=11)
    buf = program_to_device(prog)
    q = W.queries(4096, K, seed=12)
    kid = np.full(len(q), 17, np.int32)
    kid[::97] = 5
    kid[1::251] = 63
    kid[2::1009] = 0
    q[:, W.Q_KID] = kid.view(np.float32)
    qq = q[np.random.default_rng(3).permutation(len(q))]
    a, b = both_paths(buf, K, d, dev(qq))
    assert_same(a, b)
    assert (a["argmin"] >= 0).mean() > 0.9


def test_grouped_many_buckets_global_histogram():
    """K + 1 above the shared-memory histogram (8192 buckets): counts by
    global atomics."""
    need_gpu()
    K, d = 8200, 1
    prog = W.synthetic_program(K, d, seed=21)
    buf = program_to_device(prog)
    Q = 32 * K + 5
    q = W.queries(Q, K, seed=22)
    qq = q[np.random.default_rng(4).permutation(Q)]
    a, b = both_paths(buf, K, d, dev(qq))
    assert_same(a, b)


def test_grouped_workspace_reuse_and_graph():
    """A caller-provided workspace, reused across calls and inside a CUDA
    graph: replay equals the eager call."""
    need_gpu()
    K, d = 16, 2
    prog = W.synthetic_program(K, d, seed=31)
    buf = program_to_device(prog)
    q = dev(W.queries(5000, K, seed=32)[np.random.default_rng(5).permutation(5000)])
    Q = q.shape[0]
    out = dict(argmin=torch.empty(Q, dtype=torch.int32, device="cuda"),
               best=torch.empty(Q, dtype=torch.float32, device="cuda"),
               second=torch.empty(Q, dtype=torch.float32, device="cuda"),
               status=torch.empty(Q, dtype=torch.int32, device="cuda"),
               workspace=torch.empty(rp.rp_search_workspace_size(K, Q), dtype=torch.uint8,
                                     device="cuda"))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        rp.rp_eval_search(buf, K, d, q, out=out, stream=s)
    torch.cuda.synchronize()
    eager = {k: v.clone() for k, v in out.items() if k != "workspace"}
    for k in eager:
        out[k].zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rp.rp_eval_search(buf, K, d, q, out=out, stream=s)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    for k, v in eager.items():
        assert torch.equal(out[k], v), k
