"""One query split over several processes (one GPU each) by seed partition.

The library runs each part (``nuri_set_partition``): part ``index`` of ``count`` expands only
the seeds whose vertex ``nuri_seed_part`` puts in it, and calls back between rounds to share
the best threshold any part has reached.  This module supplies the host side of that:

* ``TauBoard``: the threshold exchange through a key-value store (the store of a
  ``torch.distributed`` process group, or any object with ``set``/``get``/``check``).  A part
  publishes its threshold under its own key and reads the others' keys that exist; it never
  waits for another part, because parts run different numbers of rounds.
* ``LocalBoard``: the same exchange between parts run one after another in one process.
* ``merge_rows`` / ``gather_merge``: the final step, the k best rows of all parts by the
  query's ranking (score descending, sorted vertex ids ascending, then sorted edges).

Every part's rows hold each row of the global top k whose seed lies in that part, so the
merge of the parts' top-k lists is the global top k.
"""
from __future__ import annotations

import ctypes

from . import NuriError, ERR_INVALID, lib, _check

INT64_MIN = -(1 << 63)

_EXCHANGE = ctypes.CFUNCTYPE(ctypes.c_int64, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64)


class _Partition(ctypes.Structure):
    _fields_ = [("index", ctypes.c_int32), ("count", ctypes.c_int32),
                ("exchange", _EXCHANGE), ("ctx", ctypes.c_void_p)]


def seed_part(v: int, count: int) -> int:
    """The part of seed vertex ``v`` among ``count`` parts (nuri_seed_part)."""
    return int(lib().nuri_seed_part(int(v), int(count)))


class LocalBoard:
    """Threshold exchange between parts that run in one process (one after another)."""

    def __init__(self):
        self.best = {}

    def __call__(self, query: int, local: int) -> int:
        b = max(self.best.get(query, INT64_MIN), int(local))
        self.best[query] = b
        return b


class TauBoard:
    """Threshold exchange through a key-value store: publish, then read what exists."""

    def __init__(self, store, rank: int, world: int, tag: str = "nuri-tau"):
        self.store, self.rank, self.world, self.tag = store, rank, world, tag
        self.mine = {}

    def _key(self, query, rank):
        return f"{self.tag}/{query}/{rank}"

    def __call__(self, query: int, local: int) -> int:
        local = int(local)
        if local > self.mine.get(query, INT64_MIN):
            self.mine[query] = local
            self.store.set(self._key(query, self.rank), str(local))
        best = self.mine.get(query, INT64_MIN)
        for r in range(self.world):
            if r == self.rank:
                continue
            k = self._key(query, r)
            if self.store.check([k]):
                best = max(best, int(self.store.get(k)))
        return best


def set_partition(G, index: int, count: int, board=None):
    """Restrict later clique and isomorphism queries on G to part ``index`` of ``count``,
    exchanging thresholds through ``board`` (a callable (query, local_tau) -> best)."""
    if count == 1:
        _check(lib().nuri_set_partition(G.handle, None))
        G._partition = None
        return
    if not (0 <= index < count):
        raise NuriError(ERR_INVALID, "need 0 <= index < count")
    cb = _EXCHANGE(lambda ctx, q, t: int(board(int(q), int(t)))) if board else _EXCHANGE()
    p = _Partition(int(index), int(count), cb, None)
    _check(lib().nuri_set_partition(G.handle, ctypes.byref(p)))
    G._partition = (p, cb, board)  # the callback must outlive the queries


def _rank_key(row):
    return (-row[0], tuple(row[1])) + ((tuple(row[2]),) if len(row) > 2 else ())


def merge_rows(parts, k: int):
    """The k best rows over the parts' rank-ordered row lists."""
    rows = [tuple(r) for part in parts for r in part]
    rows.sort(key=_rank_key)
    return rows[:k]


def gather_merge(rows, k: int, group=None):
    """All parts' rows gathered on every process (torch.distributed, any backend), merged."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    allp = [None] * world
    dist.all_gather_object(allp, [tuple(r) for r in rows], group=group)
    return merge_rows(allp, k)
