"""Pair sharding (paper_1208_4271_gb300/shard.py) on CPU: the static blocks
cover the pair list exactly once in rank order, the cost-balanced split
balances, and with two gloo ranks the gathered scores equal a single-process
run.  The per-rank scoring is injected: here the oracle on tiny inputs (the
GPU call is the default on GPU ranks)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n_pairs,world", [(0, 1), (1, 2), (7, 3), (16, 2), (1999000, 8), (5, 8)])
def test_blocks_cover_pairs_once(n_pairs, world):
    from paper_1208_4271_gb300 import shard
    edges = [shard.block(n_pairs, world, r) for r in range(world)]
    assert edges[0][0] == 0 and edges[-1][1] == n_pairs
    for (a, b), (c, d) in zip(edges, edges[1:]):
        assert b == c and a <= b
    sizes = [b - a for a, b in edges]
    assert max(sizes) - min(sizes) <= 1


def test_cost_balanced_blocks():
    from paper_1208_4271_gb300 import shard
    rng = np.random.default_rng(3)
    cost = rng.pareto(1.5, 5000) + 0.01
    world = 4
    edges = [shard.block(5000, world, r, cost) for r in range(world)]
    assert edges[0][0] == 0 and edges[-1][1] == 5000
    loads = [cost[a:b].sum() for a, b in edges]
    # each block ends at the first pair that reaches its share: no block is
    # more than one pair's cost away from the ideal share
    assert max(loads) - cost.sum() / world <= cost.max() + 1e-9
    with pytest.raises(ValueError):
        shard.block(3, 2, 0, cost=[1.0, -1.0, 1.0])


def _oracle_compute(alpha, c):
    def compute(V, pl):
        import oracle
        from paper_1208_4271_gb300 import gmine
        out = np.zeros(pl.shape[0], dtype=gmine.SCORE_DTYPE)
        if pl.shape[0] == 0:
            return out, None
        r = oracle.score_batch(V, pl, alpha, c, nthreads=1, want_M=True)
        for j, name in enumerate(("mic", "mas", "mev", "mcn")):
            out[name] = r["stats"][:, j]
        out["n_used"], out["B"], out["mcn_xy"] = r["info"][:, 0], r["info"][:, 1], r["info"][:, 2]
        out["m_cells"], out["status"] = r["info"][:, 3], r["status"]
        B = oracle.B_of(V.shape[1], alpha)
        cells = max(oracle.m_cells(B), 1)
        M = np.zeros((pl.shape[0], cells))
        for j in range(pl.shape[0]):
            mc = int(r["info"][j, 3])
            M[j, :mc] = r["M"][r["M_offsets"][j]:r["M_offsets"][j] + mc]
        return out, M
    return compute


def _shard_worker(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1208_4271_gb300 import shard, workloads
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        V, P = workloads.config1()
        scores, M = shard.score_sharded(V, P, 0.6, 15.0, dist=dist, want_M=True,
                                        compute=_oracle_compute(0.6, 15.0))
        np.save(os.path.join(outdir, "s%d.npy" % rank), scores.view(np.uint8))
        np.save(os.path.join(outdir, "m%d.npy" % rank), M)
    finally:
        dist.destroy_process_group()


def test_score_sharded_gloo_world_size_2(tmp_path):
    import torch.multiprocessing as mp
    import oracle
    from paper_1208_4271_gb300 import gmine, workloads
    mp.spawn(_shard_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    V, P = workloads.config1()
    ref = oracle.score_batch(V, P, 0.6, 15.0, nthreads=2, want_M=True)
    cells = max(oracle.m_cells(oracle.B_of(V.shape[1], 0.6)), 1)
    for rank in range(2):
        s = np.load(tmp_path / ("s%d.npy" % rank)).view(gmine.SCORE_DTYPE)
        M = np.load(tmp_path / ("m%d.npy" % rank))
        assert s.shape[0] == P.shape[0] and M.shape == (P.shape[0], cells)
        got = np.stack([s["mic"], s["mas"], s["mev"], s["mcn"]], axis=1)
        assert np.array_equal(got, ref["stats"])          # every pair, in pair order
        assert np.array_equal(s["m_offset"], np.arange(P.shape[0]) * cells)
        for i in range(P.shape[0]):
            mc = int(ref["info"][i, 3])
            assert np.array_equal(M[i, :mc], ref["M"][ref["M_offsets"][i]:ref["M_offsets"][i] + mc])


@pytest.mark.gpu
def test_score_sharded_default_gpu_compute_world_size_1():
    """The default per-rank call (gmine_compute_batch on the rank's GPU)
    through the gather, with a one-rank gloo group: the same records as one
    direct batch call, m_offset in the gathered layout."""
    import torch
    import torch.distributed as dist
    from paper_1208_4271_gb300 import gmine, shard, workloads
    V, P = workloads.config1()
    Vd = torch.from_numpy(V).cuda()
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        s, M = shard.score_sharded(Vd, P, 0.6, 15.0, gmine.PLAIN_FP64, dist=dist, want_M=True)
    finally:
        dist.destroy_process_group()
    sc, Md = gmine.compute_batch(Vd, torch.from_numpy(P).cuda(), 0.6, 15.0, gmine.PLAIN_FP64)
    torch.cuda.synchronize()
    ref = gmine.scores_to_numpy(sc)
    for key in ("mic", "mas", "mev", "mcn", "status", "B", "m_offset"):
        assert np.array_equal(s[key], ref[key]), key
    assert np.array_equal(M.reshape(-1), Md.cpu().numpy())
