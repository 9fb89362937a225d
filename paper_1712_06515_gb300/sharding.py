"""Template sharding across ranks and the host-side merge of per-rank top-k lists.

Templates are independent, so N ranks take disjoint contiguous template blocks and
run the search with no exchange on the data path.  The only collective is the
gather of each rank's top-k records, merged on the host with the same ordering the
device top-k uses (rho descending, ties by template then bin ascending).
"""
from __future__ import annotations

from typing import Optional, Tuple

import numpy as np

HIT_DTYPE = np.dtype([("tmpl", np.int64), ("bin", np.int32), ("freq", np.float64), ("rho", np.float32)])


def shard_range(n_templates: int, rank: int, world: int) -> Tuple[int, int]:
    """[start, stop) of rank's contiguous block; sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(n_templates, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def order_hits(hits: np.ndarray, k: int) -> np.ndarray:
    """The k best records: rho descending, then template, then bin ascending."""
    hits = np.asarray(hits, HIT_DTYPE)
    order = np.lexsort((hits["bin"], hits["tmpl"], -hits["rho"].astype(np.float64)))
    return hits[order[:k]]


def globalize(hits: np.ndarray, template_offset: int) -> np.ndarray:
    """Shift a rank's local template indices to global ones."""
    out = np.array(hits, HIT_DTYPE, copy=True)
    out["tmpl"] += template_offset
    return out


def merge_topk(local_hits: np.ndarray, k: int, group=None) -> Optional[np.ndarray]:
    """Gather every rank's (globally indexed) top-k records and merge them; every
    rank receives the merged list.  Works with any torch.distributed backend that
    supports object collectives (gloo on CPU, nccl on GPU)."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return order_hits(local_hits, k)
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, np.asarray(local_hits, HIT_DTYPE), group=group)
    return order_hits(np.concatenate(parts), k)
