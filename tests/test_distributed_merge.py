"""Multi-process pooling of the steerable covariance (images split over
ranks, Sec. IV), on CPU with the gloo backend and world size 2.

Each rank computes the FP64 oracle's statistics [n, mean0, C] of its own
shard; paper_1412_0781_gb300.distributed.pool_states all-gathers them and
pools them with the library's host-side ffb_cov_merge.  The pooled result
must equal the oracle's covariance of the union of the shards."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _data(L=16, n=37):
    from oracle import fb
    op = fb.make_plan(L, 0.5, L / 2)
    rng = np.random.default_rng(2024)
    a = rng.standard_normal((n, op.P)) + 1j * rng.standard_normal((n, op.P)) + 1.5
    a[:, :op.p[0]] = a[:, :op.p[0]].real
    a[:20] += 0.7          # shards with different means exercise the between-shard term
    return op, a


def _state(op, a):
    from oracle import fb
    mean0, blocks = fb.covariance(op, a)
    return np.concatenate([[a.shape[0]], mean0] + [b.ravel() for b in blocks])


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1412_0781_gb300 import distributed as fd
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    op, a = _data()
    cut = 20                               # uneven shards: 20 and 17 images
    shard = a[:cut] if rank == 0 else a[cut:]
    pooled = fd.pool_states(_state(op, shard), [int(v) for v in op.p])
    out.put((rank, pooled))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_pooling_matches_union():
    from paper_1412_0781_gb300 import build
    build.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = dict(q.get(timeout=240) for _ in range(2))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    op, a = _data()
    ref = _state(op, a)
    for r in (0, 1):
        assert res[r][0] == a.shape[0]
        assert np.max(np.abs(res[r] - ref)) < 1e-12 * np.max(np.abs(ref))


def test_merge_of_one_state_is_identity():
    from paper_1412_0781_gb300 import build
    from paper_1412_0781_gb300.ffb import cov_merge
    build.build()
    op, a = _data()
    st = _state(op, a)
    assert np.array_equal(cov_merge([int(v) for v in op.p], st[None]), st)


def test_merge_rejects_bad_counts():
    from paper_1412_0781_gb300 import build
    from paper_1412_0781_gb300.ffb import FFBError, cov_merge
    build.build()
    op, a = _data()
    st = _state(op, a)
    st[0] = 0.0
    with pytest.raises(FFBError):
        cov_merge([int(v) for v in op.p], st[None])
