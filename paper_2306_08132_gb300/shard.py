"""Multi-GPU partition of one grasp-search workload, by object.

The paper's search runs many independent initialisations per object (Sec. III,
first paragraph): a candidate needs only its own object's SDF, the hand and its
own configuration.  So one workload splits across ranks by object: rank k holds
the grids of its objects only and optimises the candidates of those objects,
with no exchange between ranks in the step loop.  After the loop the ranks'
results (q, loss) are gathered on rank 0 in the workload's candidate order.

Host logic only (index bookkeeping and one gather at the end); the compute on
each rank is the library's own launch over its share.
"""

from __future__ import annotations

import numpy as np


def object_shard(n_obj: int, rank: int, world: int) -> np.ndarray:
    """The objects of rank `rank`: a contiguous block of the n_obj objects, blocks
    differing in size by at most one (the first n_obj % world ranks hold one more)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    return np.array_split(np.arange(n_obj), world)[rank]


def candidate_shard(obj_of_cand: np.ndarray, objects: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """The candidates whose object is in `objects`, in workload order, and their object
    indices renumbered into `objects` (0 .. len(objects) - 1)."""
    oc = np.asarray(obj_of_cand)
    objects = np.asarray(objects)
    cand = np.nonzero(np.isin(oc, objects))[0]
    local = np.searchsorted(objects, oc[cand]).astype(np.int32)
    return cand, local


def shard_workload(n_obj: int, obj_of_cand: np.ndarray, rank: int, world: int) -> dict:
    """Everything rank `rank` needs to build and run its share: its objects, its
    candidates (global indices) and their local object indices."""
    objs = object_shard(n_obj, rank, world)
    cand, local = candidate_shard(obj_of_cand, objs)
    return {"objects": objs, "candidates": cand, "obj_of_cand": local}


def gather_rows(rows: np.ndarray, candidates: np.ndarray, n_total: int, group=None):
    """Gather every rank's per-candidate rows (rows[i] belongs to global candidate
    candidates[i]) on rank 0 as one array in workload order; None on other ranks.
    Uses torch.distributed (any backend) when it is initialised, else returns the
    rows of this process placed at their candidates."""
    import torch.distributed as dist
    rows = np.ascontiguousarray(rows)
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        out = np.zeros((n_total,) + rows.shape[1:], dtype=rows.dtype)
        out[candidates] = rows
        return out
    rank = dist.get_rank(group)
    parts = [None] * dist.get_world_size(group) if rank == 0 else None
    dist.gather_object((np.asarray(candidates), rows), parts, dst=0, group=group)
    if rank != 0:
        return None
    out = np.zeros((n_total,) + rows.shape[1:], dtype=rows.dtype)
    seen = np.zeros(n_total, dtype=bool)
    for cand, r in parts:
        if seen[cand].any():
            raise RuntimeError("a candidate was computed by two ranks")
        seen[cand] = True
        out[cand] = r
    if not seen.all():
        raise RuntimeError("%d candidates were computed by no rank" % int((~seen).sum()))
    return out


class RequestRouter:
    """Routes serving requests to GPUs by HBM budget (one request queue per GPU).

    A request needs its optimiser state (q and loss: B (D + 1) floats) on the GPU
    that serves it, plus its object's grid unless that GPU already holds the object
    for another request.  Each request goes to the GPU where it adds the fewest
    bytes (its object already resident there first), ties broken by the most free
    budget, then the lowest index; a request that fits no GPU's remaining budget is
    refused (None) and can be submitted again after `release`.  Host bookkeeping
    only: the queues admit and run the requests."""

    def __init__(self, budgets):
        self.budget = [int(b) for b in budgets]
        self.used = [0] * len(self.budget)
        self.objects = [dict() for _ in self.budget]      # object key -> (bytes, requests using it)

    def need(self, gpu: int, state_bytes: int, obj_key, obj_bytes: int) -> int:
        return int(state_bytes) + (0 if obj_key in self.objects[gpu] else int(obj_bytes))

    def route(self, state_bytes: int, obj_key, obj_bytes: int):
        best = None
        for g in range(len(self.budget)):
            n = self.need(g, state_bytes, obj_key, obj_bytes)
            if self.used[g] + n > self.budget[g]:
                continue
            key = (n, -(self.budget[g] - self.used[g]), g)
            if best is None or key < best[0]:
                best = (key, g, n)
        if best is None:
            return None
        _, g, n = best
        self.used[g] += n
        b, refs = self.objects[g].get(obj_key, (int(obj_bytes), 0))
        self.objects[g][obj_key] = (b, refs + 1)
        return g

    def release(self, gpu: int, state_bytes: int, obj_key) -> None:
        """The request finished on `gpu`: its state, and its object once unused, free up."""
        self.used[gpu] -= int(state_bytes)
        b, refs = self.objects[gpu][obj_key]
        if refs == 1:
            del self.objects[gpu][obj_key]
            self.used[gpu] -= b
        else:
            self.objects[gpu][obj_key] = (b, refs - 1)
