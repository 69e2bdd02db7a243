"""Many independent Online TT-ALS streams of uneven shapes stepped together.

Streams of one shape (slice dims, ranks, ingest) share a batch (``ttals_create_batch``): one
launch of each fused kernel per step serves all of them, whatever their number.  A group
therefore steps S streams of K distinct shapes with 3K launches.  The batches are
independent, so each runs on a CUDA stream of its own, forked from and joined back into the
caller's stream: their latency-bound kernel chains overlap on the GPU.  ``capture`` records
an even number of steps into one CUDA graph (K parallel branches per step), so that a
replay costs one graph launch.

Each batch's schedule (environment kernel and local-solve kernel with their tile shapes,
k-splits of the local solve, factor cluster size) comes from ``tune.best_schedule`` unless
``tune=False``.  The schedule changes only the order of FP32
sums, never what is computed.

Inputs live in device memory owned by the group: for every batch a ring of ``depth``
blocks, each [n_streams][slice], so that a caller (or a serving loop) writes stream i's
next slice into ``group.slot(i, p)`` and steps with ``group.step(p)``.
Argument marshalling and bookkeeping only: every step of the update runs in the library's
CUDA kernels.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import ttals
from .ttals import Stream

_TORCH_DT = {"f16": "float16", "bf16": "bfloat16", "f32": "float32", "f64": "float64"}


def plan_buckets(specs: Sequence[Tuple[Sequence[int], Sequence[int]]],
                 max_batch: int = ttals.MAX_BATCH) -> List[Tuple[tuple, tuple, List[int]]]:
    """Streams grouped into batches: one per distinct (dims, ranks) in order of first
    appearance, each holding at most `max_batch` stream indices (in input order).  Returns
    [(dims, ranks, members)]."""
    keys: Dict[tuple, List[int]] = {}
    for i, (d, r) in enumerate(specs):
        keys.setdefault((tuple(int(v) for v in d), tuple(int(v) for v in r)), []).append(i)
    out = []
    for (d, r), members in keys.items():
        for c0 in range(0, len(members), max_batch):
            out.append((d, r, members[c0:c0 + max_batch]))
    return out


class _Bucket:
    def __init__(self, dims, ranks, ingest, members, depth, schedule):
        import torch
        self.dims = tuple(dims)
        self.ranks = tuple(ranks)
        self.members = list(members)            # group stream indices, in slot order
        self.schedule = dict(schedule or {})
        n = len(self.members)
        from .tune import KEYS
        self.stream = Stream(dims, ranks, ingest=ingest, n_streams=n,
                             **{k: int(self.schedule.get(k, 0)) for k in KEYS})
        dt = getattr(torch, _TORCH_DT[ingest])
        self.inputs = torch.zeros((depth, n) + self.dims, dtype=dt, device="cuda")


class Group:
    """S streams given as (dims, ranks) pairs, 16-bit ingest (the fused path's batches)."""

    def __init__(self, specs: Sequence[Tuple[Sequence[int], Sequence[int]]], ingest: str = "f16",
                 depth: int = 2, tune: bool = True, tune_steps: int = 8):
        if ingest not in ("f16", "bf16"):
            raise ValueError("groups batch the fused path: FP16 or BF16 ingest")
        self.ingest = ingest
        self.depth = int(depth)
        self.specs = [(tuple(int(v) for v in d), tuple(int(v) for v in r)) for d, r in specs]
        self.buckets: List[_Bucket] = []
        self.where: Dict[int, Tuple[int, int]] = {}
        for d, r, part in plan_buckets(self.specs):
            sched = None
            if tune:
                from . import tune as _tune
                sched = _tune.best_schedule(d, r, len(part), ingest, steps=tune_steps)
            b = _Bucket(d, r, ingest, part, self.depth, sched)
            for slot, i in enumerate(part):
                self.where[i] = (len(self.buckets), slot)
            self.buckets.append(b)
        self._graph = None
        import torch
        self._side = [torch.cuda.Stream() for _ in self.buckets]

    # -- inputs and stepping
    def slot(self, i: int, p: int = 0):
        """Device tensor that receives stream i's slice for ring position p."""
        bi, slot = self.where[i]
        return self.buckets[bi].inputs[p, slot]

    def step(self, p: int = 0, active: Optional[set] = None, stream=None):
        """One step of every stream (or of the streams in `active`), slices from ring position p."""
        import torch
        main = stream or torch.cuda.current_stream()
        fork = torch.cuda.Event()
        fork.record(main)
        for b, side in zip(self.buckets, self._side):
            blk = b.inputs[p]
            mask = None
            if active is not None:
                mask = 0
                for slot, i in enumerate(b.members):
                    if i in active:
                        mask |= 1 << slot
                if not mask:
                    continue
            side.wait_event(fork)
            b.stream.push_batch_ptr(blk.data_ptr(), side.cuda_stream, mask)
            join = torch.cuda.Event()
            join.record(side)
            main.wait_event(join)

    def capture(self, positions: Sequence[int], stream):
        """Record one step per ring position in `positions` (an even count: the state's
        double buffers end where they started) into a CUDA graph on `stream`; replay() then
        performs them all.  Steps enqueued on `stream` before the capture fix the order."""
        import torch
        if len(positions) % 2:
            raise ValueError("capture an even number of steps")
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for p in positions:
                self.step(p, stream=torch.cuda.current_stream())
        self._graph = g
        return g

    def replay(self):
        self._graph.replay()

    # -- per-stream access
    def _sel(self, i):
        bi, slot = self.where[i]
        b = self.buckets[bi]
        b.stream.select(slot)
        return b.stream

    def set_cores(self, i, cores, g, t: int = 0):
        self._sel(i).set_cores(cores, g, t)

    def reconstruct(self, i, out, dtype: str = "f64", stream=None):
        self._sel(i).reconstruct(out, dtype, stream)

    def stats(self, i) -> np.ndarray:
        return self._sel(i).stats()

    def step_count(self, i) -> int:
        return self._sel(i).step()

    @property
    def launches_per_step(self) -> int:
        return 3 * len(self.buckets)

    def device_bytes(self) -> int:
        return sum(b.stream.device_bytes + b.inputs.numel() * b.inputs.element_size() for b in self.buckets)

    def close(self):
        for b in self.buckets:
            b.stream.close()
        self.buckets = []
