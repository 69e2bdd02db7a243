"""Serving loop: many independent Online TT-ALS streams, frames arriving over time.

A ``Server`` keeps every admitted stream's state resident on the device and steps streams
with continuous batching:

* **Pools.** Streams of one shape share a pool: a batch (``ttals_create_batch``) of
  ``slots`` streams with a double-buffered input block [2][slots][slice].  A stream takes
  a free slot of a pool of its shape; a new pool is created only if the HBM budget allows
  (``ttals_device_bytes`` of the batch plus its input blocks).  A stream that does not fit
  waits in the admission queue until a departing stream frees a slot or memory.
* **Shapes.** Requested ranks are rounded up to a multiple of ``rank_step`` (never down),
  so that streams with nearby ranks share pools; the stream then tracks with the rounded
  ranks (at least the accuracy it asked for).
* **Steps.** ``tick()`` takes, for every pool, the oldest pending frame of each of its
  streams and hands them to the library in one call (``ttals_batch_push_host``): it copies
  them host -> device into the pool's next input block on the pool's copy stream and
  enqueues one masked batch step (only the streams with a frame step) on its compute stream.  Pools have their own CUDA streams, so the
  work of different pools overlaps on the GPU; frames that arrive while a step is in
  flight wait for the pool's next tick.
* **Wire format.** With ``wire="u8"`` frames are 8-bit pixels (the paper's video data):
  bytes cross the host link and ``ttals_widen_u8`` widens them to the ingest type on the
  device (exact), half the host-link traffic of FP16 frames.
* **Latency.** Per frame: from its arrival time to the host's detection of the completion
  event of the step that consumed it (``poll()``), in seconds.

The admission and queueing logic is plain host code; ``pool_factory`` lets tests drive it
without a GPU.
"""
from __future__ import annotations

import collections
import time
from typing import Callable, Dict, List, Optional, Sequence, Tuple


def round_ranks(ranks: Sequence[int], step: int) -> Tuple[int, ...]:
    return tuple(((int(r) + step - 1) // step) * step for r in ranks)


def feasible_ranks(dims: Sequence[int], ranks: Sequence[int]) -> Tuple[int, ...]:
    """The ranks a stream is created with (the library's clamp, Sec. 3.4: r_k <= r_{k-1} I_k
    and r_k <= I_{k+1} r_{k+1}, r_0 = 1, iterated to a fixed point); pools are keyed on them."""
    d = [int(v) for v in dims]
    r = [int(v) for v in ranks]
    while True:
        old = list(r)
        prev = 1
        for k in range(len(d)):
            r[k] = min(r[k], prev * d[k])
            prev = r[k]
        for k in range(len(d) - 2, -1, -1):
            r[k] = min(r[k], d[k + 1] * r[k + 1])
        if r == old:
            return tuple(r)


class _Pool:
    """Device side of a pool: a batch with the library's host ingest (its own double-buffered
    input blocks, 8-bit staging, copy and compute streams, completion tickets)."""

    def __init__(self, dims, ranks, slots, ingest, wire="f16"):
        from .ttals import Stream
        self.dims, self.ranks, self.slots = tuple(dims), tuple(ranks), int(slots)
        self.batch = Stream(dims, ranks, ingest=ingest, n_streams=self.slots)
        self.wire = wire
        self.batch.ingest_init(u8=(wire == "u8"))
        self.bytes = self.batch.device_bytes

    def reset_slot(self, slot, sid, init_cores=None):
        """A new stream in this slot: its initial cores (the library's default random cores
        seeded by the stream id, unless `init_cores` gives them), step count and statistics
        zero."""
        self.batch.select(slot)
        if init_cores is not None:
            cores, g = init_cores(sid, self.dims, self.batch.ranks)
            self.batch.set_cores(cores, g, 0)
        else:
            # a stable seed (Python's hash of a string id changes from process to process)
            import zlib
            self.batch.seed_cores((zlib.crc32(repr(sid).encode()) & 0x7FFFFFFF) + 1)

    def step(self, frames: Dict[int, object]):
        """frames: slot -> pinned host tensor (the slice in the ingest type, or bytes with the
        8-bit wire).  One library call: copies, widening, masked step.  Returns the step's
        completion handle, which also keeps the frames alive until the step is done."""
        slots = list(frames)
        ticket = self.batch.push_host(slots, [frames[q].data_ptr() for q in slots])
        return _Done(self.batch, ticket, [frames[q] for q in slots])

    def close(self):
        self.batch.close()


class _Done:
    """Completion of one pool step (its ticket); holds the step's host frames until then."""

    def __init__(self, batch, ticket, keep):
        self.batch, self.ticket, self.keep = batch, ticket, keep

    def query(self) -> bool:
        if self.batch.ticket_done(self.ticket):
            self.keep = None
            return True
        return False


class Server:
    def __init__(self, budget_bytes: int, ingest: str = "f16", slots: int = 16, rank_step: int = 16,
                 pool_factory: Optional[Callable] = None, init_cores: Optional[Callable] = None,
                 wire: str = "f16"):
        self.budget = int(budget_bytes)
        self.used = 0
        self.ingest = ingest
        self.slots = int(slots)
        self.rank_step = int(rank_step)
        self.pool_factory = pool_factory or (lambda d, r, n: _Pool(d, r, n, ingest, wire))
        self.init_cores = init_cores           # (stream_id, dims, ranks) -> (cores, g), or seeded
        self.pools: Dict[tuple, List[object]] = collections.defaultdict(list)
        self.where: Dict[object, Tuple[object, int]] = {}     # stream id -> (pool, slot)
        self.owner: Dict[Tuple[int, int], object] = {}        # (id(pool), slot) -> stream id
        self.free: Dict[int, List[int]] = {}                  # id(pool) -> free slots
        self.waiting: collections.OrderedDict = collections.OrderedDict()  # id -> (dims, ranks)
        self.pending: Dict[object, collections.deque] = collections.defaultdict(collections.deque)
        self.inflight: List[Tuple[object, List[Tuple[object, float]]]] = []
        self.latencies: List[float] = []
        self.completed: Dict[object, int] = collections.defaultdict(int)
        self.steps = 0

    # -- admission
    def key(self, dims, ranks):
        d = tuple(int(v) for v in dims)
        return d, feasible_ranks(d, round_ranks(ranks, self.rank_step))

    def _try_place(self, sid, dims, ranks) -> bool:
        k = self.key(dims, ranks)
        for pool in self.pools[k]:
            if self.free[id(pool)]:
                return self._assign(sid, pool, k)
        # a new pool, if the budget allows
        pool = self.pool_factory(k[0], k[1], self.slots)
        if self.used + pool.bytes > self.budget:
            pool.close()
            return False
        self.used += pool.bytes
        self.pools[k].append(pool)
        self.free[id(pool)] = list(range(self.slots))
        return self._assign(sid, pool, k)

    def _assign(self, sid, pool, k) -> bool:
        slot = self.free[id(pool)].pop(0)
        self.where[sid] = (pool, slot)
        self.owner[(id(pool), slot)] = sid
        pool.reset_slot(slot, sid, self.init_cores)
        return True

    def connect(self, sid, dims, ranks) -> bool:
        """Admit stream `sid` now if a slot or the budget allows, else queue it.  True if admitted."""
        if not self.waiting and self._try_place(sid, dims, ranks):
            return True
        self.waiting[sid] = (dims, ranks)
        return False

    def disconnect(self, sid):
        """Free the stream's slot (after its pending frames are served) and admit waiters."""
        if sid in self.waiting:
            del self.waiting[sid]
            return
        pool, slot = self.where.pop(sid)
        del self.owner[(id(pool), slot)]
        self.free[id(pool)].append(slot)
        self.pending.pop(sid, None)
        self._admit_waiting()

    def _admit_waiting(self):
        for sid in list(self.waiting):
            dims, ranks = self.waiting[sid]
            if self._try_place(sid, dims, ranks):
                del self.waiting[sid]
            else:
                break            # first come, first served

    def admitted(self, sid) -> bool:
        return sid in self.where

    # -- frames
    def submit(self, sid, frame, t_arrival: float):
        """Queue a frame (a pinned host tensor of the stream's slice shape) of an admitted
        or waiting stream."""
        self.pending[sid].append((frame, t_arrival))

    def tick(self) -> int:
        """Enqueue one masked step per pool that has pending frames; returns frames enqueued."""
        n = 0
        for k, pools in self.pools.items():
            for pool in pools:
                frames, meta = {}, []
                for slot in range(self.slots):
                    sid = self.owner.get((id(pool), slot))
                    if sid is None or not self.pending.get(sid):
                        continue
                    f, ta = self.pending[sid].popleft()
                    frames[slot] = f
                    meta.append((sid, ta))
                if frames:
                    ev = pool.step(frames)
                    self.inflight.append((ev, meta))
                    self.steps += 1
                    n += len(frames)
        return n

    def poll(self, now: Optional[float] = None) -> int:
        """Record the latency of every frame whose step has completed; returns their number."""
        done, keep = 0, []
        for ev, meta in self.inflight:
            if ev.query():
                t = time.perf_counter() if now is None else now
                for sid, ta in meta:
                    self.latencies.append(t - ta)
                    self.completed[sid] += 1
                done += len(meta)
            else:
                keep.append((ev, meta))
        self.inflight = keep
        return done

    def restart_streams(self):
        """Every admitted stream back to its initial cores, step count and statistics zero, and
        the latency record cleared (frames still pending or in flight are dropped from it);
        admission, pools and their device resources stay.  For starting a measurement on a
        server whose pools have already run (first steps of a pool pay one-time costs)."""
        for sid, (pool, slot) in self.where.items():
            pool.reset_slot(slot, sid, self.init_cores)
        self.latencies = []
        self.completed = collections.defaultdict(int)
        self.steps = 0

    def backlog(self) -> int:
        return sum(len(q) for q in self.pending.values()) + sum(len(m) for _, m in self.inflight)

    def stream(self, sid):
        """(batch Stream selected on this stream's slot) for readout: cores, x^, statistics."""
        pool, slot = self.where[sid]
        pool.batch.select(slot)
        return pool.batch

    def close(self):
        for pools in self.pools.values():
            for p in pools:
                p.close()
        self.pools.clear()


def percentiles(lat: Sequence[float]) -> dict:
    if not lat:
        return {"p50": None, "p99": None, "n": 0}
    s = sorted(lat)
    return {"p50": s[len(s) // 2], "p99": s[min(len(s) - 1, int(0.99 * len(s)))], "n": len(s)}
