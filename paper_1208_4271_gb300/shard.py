"""Pair sharding across ranks: one pair list split into static blocks, each
rank scoring its block on its own GPU, the score records gathered afterwards.

The paper spreads the pairs of an analysis over worker processes (R
`parallel`, SI experiment 2A) and over MPI ranks (Rmpi, SI experiment 2B,
about 70x on 100 cores); pairs are independent, so the only exchange is the
gather of the results.  Here a rank is one process per GPU under
torch.distributed (NCCL on GPUs, gloo on CPUs): `block` gives each rank a
contiguous block of the pair list (optionally balanced by a per-pair cost),
`score_sharded` runs the batch on the local block and gathers the 72-byte
score records (and, if asked, M) to every rank in pair order.

There is no collective on the data path of the scoring itself; the gather
is the only communication, one all_gather of a padded byte buffer.
"""
import numpy as np

from . import gmine


def block(n_pairs, world, rank, cost=None):
    """[lo, hi) of this rank's contiguous block of pairs.  Without cost the
    blocks differ in size by at most one pair; with a non-negative cost per
    pair, the block ends are where the cumulative cost crosses k/world of the
    total (the same split on every rank, pairs in their given order)."""
    if world < 1 or not 0 <= rank < world or n_pairs < 0:
        raise ValueError("bad world/rank/n_pairs")
    if cost is None:
        base, extra = divmod(n_pairs, world)
        lo = rank * base + min(rank, extra)
        return lo, lo + base + (1 if rank < extra else 0)
    cost = np.asarray(cost, dtype=np.float64)
    if cost.shape != (n_pairs,) or np.any(cost < 0):
        raise ValueError("cost needs one non-negative value per pair")
    cum = np.concatenate([[0.0], np.cumsum(cost)])
    total = cum[-1]
    if total <= 0:
        return block(n_pairs, world, rank)
    edges = [0] + [int(np.searchsorted(cum, total * k / world, side="left")) for k in range(1, world)]
    edges.append(n_pairs)
    edges = np.maximum.accumulate(np.minimum(edges, n_pairs))
    return int(edges[rank]), int(edges[rank + 1])


def _gather_bytes(local, dist, device):
    """all_gather of a variable-length uint8 buffer; returns the per-rank
    buffers in rank order."""
    import torch
    world = dist.get_world_size()
    n = torch.tensor([local.size], dtype=torch.int64, device=device)
    sizes = [torch.zeros(1, dtype=torch.int64, device=device) for _ in range(world)]
    dist.all_gather(sizes, n)
    sizes = [int(x.item()) for x in sizes]
    m = max(max(sizes), 1)
    buf = torch.zeros(m, dtype=torch.uint8, device=device)
    if local.size:
        buf[:local.size] = torch.from_numpy(local).to(device)
    parts = [torch.zeros(m, dtype=torch.uint8, device=device) for _ in range(world)]
    dist.all_gather(parts, buf)
    return [p[:s].cpu().numpy() for p, s in zip(parts, sizes)]


def score_sharded(vars_, pairs, alpha=0.6, c=15.0, precision=gmine.PLAIN_FP64, dist=None,
                  cost=None, want_M=False, compute=None, device=None):
    """Score pairs[i] for all i, each rank its block, results on every rank.

    vars_: float64 [p, n] (a CUDA tensor on this rank's GPU, or host data that
    `compute` accepts); pairs: int32 [n_pairs, 2] host array.  compute(vars_,
    local_pairs) must return (scores as a structured array of
    gmine.SCORE_DTYPE, M as a float64 [n_local, cells] array or None); by
    default it is gmine.compute_batch on this rank's device.  Returns
    (scores [n_pairs] structured array, M [n_pairs, cells] or None), with
    m_offset rewritten to the gathered layout (cells of B = floor(n^alpha)
    per pair)."""
    import torch
    if dist is None:
        import torch.distributed as dist
    world, rank = dist.get_world_size(), dist.get_rank()
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    lo, hi = block(pairs.shape[0], world, rank, cost)
    if compute is None:
        def compute(v, pl):
            if pl.shape[0] == 0:
                return np.zeros(0, dtype=gmine.SCORE_DTYPE), None
            sc, M = gmine.compute_batch(v, torch.from_numpy(pl).to(v.device), alpha, c, precision,
                                        want_M=want_M)
            torch.cuda.synchronize(v.device)
            s = gmine.scores_to_numpy(sc)
            cells = M.numel() // max(pl.shape[0], 1) if M is not None else 0
            return s, (M.cpu().numpy().reshape(pl.shape[0], cells) if M is not None else None)
    scores, M = compute(vars_, pairs[lo:hi])
    scores = np.ascontiguousarray(scores, dtype=gmine.SCORE_DTYPE)
    if device is None:
        device = "cpu" if dist.get_backend() == "gloo" else torch.device("cuda", torch.cuda.current_device())
    parts = _gather_bytes(scores.view(np.uint8), dist, device)
    out = np.concatenate([p.view(gmine.SCORE_DTYPE) for p in parts]) if parts else scores
    # cells reserved per pair: those of B = floor(n^alpha) (gmine_plan's layout)
    cells = max(gmine.m_cells(gmine.B_of(max(int(vars_.shape[1]), 1), alpha)), 1)
    out["m_offset"] = np.arange(out.shape[0], dtype=np.int64) * cells
    Mall = None
    if want_M and M is not None:
        mparts = _gather_bytes(np.ascontiguousarray(M, dtype=np.float64).view(np.uint8).reshape(-1),
                               dist, device)
        Mall = np.concatenate([p.view(np.float64).reshape(-1, cells) for p in mparts])
    return out, Mall
