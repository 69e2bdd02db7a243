#!/usr/bin/env python
"""Online TT-ALS per-slice update benchmark (arXiv 2606.31061, Algorithm 1).

Workload: the video-shaped 4th-order stream, 1080 x 1920 x 3 slices of uint8-range
values (smooth TT field of ranks (32,32,3) plus integer noise, clipped to 0..255),
method ranks (32,32,3) clamped to (32,9,3), FP16 ingest (exact for 8-bit pixels) with
FP32 accumulation; FP32 ingest is timed alongside.  A step is one push of one slice
through the whole update.  Synthetic, seeded frames (synth.make_stream("video")): a
pool of 64 consecutive frames (796 MB in FP16, larger than the 126 MB L2) is played
forward and backward so that consecutive steps stay temporally smooth.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs an independent replica
stream on its own GPU (streams are independent: no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Online TT-ALS slices/s & HBM GB/s vs peak; p50/p99 per-slice latency"
DIMS = (1080, 1920, 3)
RANKS = (32, 32, 3)
WORKLOAD = "video 1080x1920x3 stream, TT ranks (32,32,3) clamped to (32,9,3), T=600-step recipe"


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "of measured"
    except Exception:
        return 6400.0, "of fallback"


def pingpong(t, n):
    if n == 1:
        return 0
    p = 2 * (n - 1)
    u = t % p
    return u if u < n else p - u


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, t0, t1):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        rows = [l for (ts, l) in self.lines if t0 - 0.15 <= ts <= t1 + 0.15] or [l for _, l in self.lines]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in rows:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1].split()[0]))
                mx.append(float(f[2].split()[0]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_pool(ingest, n):
    from paper_2606_31061_b300 import synth
    sp = synth.make_stream("video")
    frames = []
    for x in sp.frames(n):
        payload, _ = synth.round_to_ingest(x, ingest)
        frames.append(payload)
    return np.stack(frames)


def to_device(pool_np, ingest):
    import torch
    t = torch.from_numpy(pool_np)
    if ingest == "f16":
        t = t.view(torch.float16)
    elif ingest == "bf16":
        t = t.view(torch.bfloat16)
    return t.cuda()


# the sources of the fused kernels whose DRAM traffic profiles/traffic.json records
TRAFFIC_SOURCES = ("ttals_fast.cuh", "ttals_r64.cuh")


def traffic_sha256():
    import hashlib
    h = hashlib.sha256()
    src = os.path.join(ROOT, "paper_2606_31061_b300", "csrc")
    for name in TRAFFIC_SOURCES:
        h.update(open(os.path.join(src, name), "rb").read())
    return h.hexdigest()


def traffic_record(kernel, sub=None):
    """DRAM bytes per launch from a committed ncu capture, if the fused kernels' sources are
    unchanged (`sub`: the kernel within a batched record)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)
        digest = traffic_sha256()
        r = rec.get(kernel)
        if r and r.get("src_sha256") == digest:
            return r["kernel_bytes_per_launch"].get(sub) if sub else r.get("bytes_per_launch")
    except Exception:
        pass
    return None


def time_arm(ingest, steps, warmup, pool, dist_on, sampler_idx, factor="fp64", dims=None, ranks=None):
    """Device-timed throughput of `steps` pushes; per-kernel event timing on the launch stream."""
    import torch
    from paper_2606_31061_b300.ttals import Stream
    st = Stream(dims or DIMS, ranks or RANKS, ingest=ingest, factor=factor)
    P = pool.shape[0]
    stream = torch.cuda.current_stream()
    h = stream.cuda_stream
    for t in range(warmup):
        st.push_ptr(pool[pingpong(t, P)].data_ptr(), h)
    torch.cuda.synchronize()
    if dist_on:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = None
    sampler = ClockSampler(sampler_idx) if sampler_idx is not None else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    ptrs = [pool[i].data_ptr() for i in range(P)]
    order = [ptrs[pingpong(warmup + t, P)] for t in range(steps)]
    # host cost of one push: a short burst enqueued while the device is busy (the launch
    # queue does not fill, so no back-pressure is included)
    nb = 200
    burst = [ptrs[pingpong(t % warmup, P)] for t in range(nb)]   # slices seen in the warm-up (maps cached)
    host_us = float("inf")
    for _ in range(3):                                           # best of three bursts
        torch.cuda._sleep(int(1e9))
        h0 = time.perf_counter()
        for p in burst:
            st.push_ptr(p, h)
        host_us = min(host_us, (time.perf_counter() - h0) / nb * 1e6)
        torch.cuda.synchronize()
    n0 = st.launch_count
    w0 = time.time()
    e0.record(stream)
    for p in order:
        st.push_ptr(p, h)
    e1.record(stream)
    torch.cuda.synchronize()
    w1 = time.time()
    if dist_on:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        clocks = sampler.stop(w0, w1)
    ms = e0.elapsed_time(e1)
    launches = st.launch_count - n0
    # per-kernel timing: CUDA events recorded by the library on the launch stream around
    # the level-1 kernels (a separate pass, so the event records do not sit inside the
    # throughput region above)
    nprof = min(steps, 400)
    st.profile(True)
    # keep the device busy while the host enqueues the whole pass, so that no event pair
    # spans a gap in which the next kernel had not been submitted yet
    torch.cuda._sleep(int(2e8))
    for t in range(nprof):
        st.push_ptr(pool[pingpong(warmup + steps + t, P)].data_ptr(), h)
    ms_solve, ms_factor, ms_env, ms_push, npush = st.profile_read()
    st.profile(False)
    lat = []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(min(steps, 400))]
    torch.cuda._sleep(int(2e8))
    for t, (a, b) in enumerate(ev):
        a.record(stream)
        st.push_ptr(pool[pingpong(warmup + steps + nprof + t, P)].data_ptr(), h)
        b.record(stream)
    torch.cuda.synchronize()
    lat = sorted(a.elapsed_time(b) for a, b in ev)
    stats = st.stats()
    st.close()
    return dict(ms=ms, launches=launches, host_us=host_us, ms_solve=ms_solve, ms_factor=ms_factor, ms_env=ms_env,
                ms_push=ms_push, npush=npush,
                lat=lat, clocks=clocks, re=math.sqrt(stats[3] / stats[2]) if stats[2] > 0 else None)


def batched_arm(ingest, nstreams, steps, warmup, pool):
    """`nstreams` independent video streams stepped together (ttals_push_batch): each push
    carries one slice per stream, contiguous [nstreams][slice].  Stream b at step t reads
    pool frame o_t + b, with o_t walking the pool forward and backward, so that every
    stream stays temporally smooth.  Returns device time, per-kernel times, per-push latency
    and each stream's relative reconstruction error."""
    import torch
    from paper_2606_31061_b300.ttals import Stream
    st = Stream(DIMS, RANKS, ingest=ingest, n_streams=nstreams)
    P = pool.shape[0]
    W = P - nstreams + 1
    stream = torch.cuda.current_stream()
    h = stream.cuda_stream
    ptrs = [pool[o].data_ptr() for o in range(W)]
    for t in range(warmup):
        st.push_batch_ptr(ptrs[pingpong(t, W)], h)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda._sleep(int(2e8))
    n0 = st.launch_count
    e0.record(stream)
    for t in range(steps):
        st.push_batch_ptr(ptrs[pingpong(warmup + t, W)], h)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = st.launch_count - n0
    nprof = min(steps, 200)
    st.profile(True)
    torch.cuda._sleep(int(2e8))
    for t in range(nprof):
        st.push_batch_ptr(ptrs[pingpong(warmup + steps + t, W)], h)
    ms_solve, ms_factor, ms_env, ms_push, npush = st.profile_read()
    st.profile(False)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(min(steps, 200))]
    torch.cuda._sleep(int(2e8))
    for t, (a, b) in enumerate(ev):
        a.record(stream)
        st.push_batch_ptr(ptrs[pingpong(warmup + steps + nprof + t, W)], h)
        b.record(stream)
    torch.cuda.synchronize()
    lat = sorted(a.elapsed_time(b) for a, b in ev)
    res = []
    for b in range(nstreams):
        st.select(b)
        s = st.stats()
        res.append(math.sqrt(s[3] / s[2]) if s[2] > 0 else float("nan"))
    st.close()
    return dict(ms=ms, launches=launches, ms_solve=ms_solve, ms_factor=ms_factor, ms_env=ms_env,
                ms_push=ms_push, npush=npush, lat=lat, re=res)


def c4_specs(n=64, seed=1004):
    """Mixed-shape batched workload: n streams of s x s slices, s uniform on {128, 256, 512,
    1024}, ranks (r, r) with r uniform on {8, 16, 32, 64} (seeded)."""
    rng = np.random.default_rng(seed)
    sides = rng.choice([128, 256, 512, 1024], size=n)
    ranks = rng.choice([8, 16, 32, 64], size=n)
    return [((int(s), int(s)), (int(r), int(r))) for s, r in zip(sides, ranks)]


def c4_arm(steps, depth=4, tune=True):
    """64 streams of uneven shapes stepped together through paper_2606_31061_b300.group: one
    batch per distinct shape, schedules from the autotuner, a ring of `depth` input blocks
    (larger than L2 in total) filled with each stream's synthetic drifting low-rank frames.
    Times eager steps and replays of a CUDA graph holding `depth` steps."""
    import torch
    from paper_2606_31061_b300 import synth
    from paper_2606_31061_b300.group import Group
    specs = c4_specs()
    t0 = time.perf_counter()
    grp = Group(specs, depth=depth, tune=tune, tune_steps=6)
    tune_s = time.perf_counter() - t0
    in_bytes = 0
    for i, (d, r) in enumerate(specs):
        sp = synth.make_stream("square", s=d[0], r=r[0], seed=1004 * 100 + i)
        for p, x in enumerate(sp.take(depth)):
            grp.slot(i, p).copy_(torch.from_numpy(synth.round_to_ingest(x, "f16")[0]).view(torch.float16))
        in_bytes += 2 * d[0] * d[1]
    cs = torch.cuda.Stream()
    with torch.cuda.stream(cs):
        for t in range(2 * depth):
            grp.step(t % depth, stream=cs)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda._sleep(int(1e8))
        e0.record(cs)
        for t in range(steps):
            grp.step(t % depth, stream=cs)
        e1.record(cs)
        torch.cuda.synchronize()
        ms_eager = e0.elapsed_time(e1)
        grp.capture(list(range(depth)), cs)
        reps = max(1, steps // depth)
        grp.replay()
        torch.cuda.synchronize()
        e0.record(cs)
        for _ in range(reps):
            grp.replay()
        e1.record(cs)
        torch.cuda.synchronize()
        ms_graph = e0.elapsed_time(e1)
    n = len(specs)
    res = []
    for i in range(n):
        s_ = grp.stats(i)
        res.append(math.sqrt(s_[3] / s_[2]) if s_[2] > 0 else float("nan"))
    sched = {}
    for b in grp.buckets:
        key = f"{b.dims[0]}x{b.dims[1]} r{b.ranks[0]} n{len(b.members)}"
        sched[key] = {k: v for k, v in b.schedule.items() if k in ("env_kernel", "solve_kernel", "k1_split",
                                                                    "factor_cluster")}
    out = {
        "workload": "64 streams, s x s slices with s ~ U{128,256,512,1024}, ranks (r, r) with r ~ U{8,16,32,64} "
                    "(seed 1004), drifting low-rank TT fields + noise 0.01, FP16 ingest",
        "streams": n, "batches": len(grp.buckets), "launches_per_step": grp.launches_per_step,
        "slice_bytes_per_step": in_bytes,
        "value": steps * n / (ms_eager / 1000.0), "unit": "slices/s",
        "hbm_gbs_slices": steps * in_bytes / (ms_eager / 1000.0) / 1e9,
        "ms_per_step": ms_eager / steps,
        "graph": {"value": reps * depth * n / (ms_graph / 1000.0), "unit": "slices/s",
                  "ms_per_step": ms_graph / (reps * depth), "steps_per_graph": depth},
        "l2": f"ring of {depth} input blocks, {depth * in_bytes / 1e6:.0f} MB in total",
        "re_per_stream": {"min": min(res), "max": max(res)},
        "tuning_seconds": tune_s, "schedules": sched,
    }
    grp.close()
    return out


SERVE_SIZES = ((256, 256), (720, 1280, 3), (1080, 1920, 3))


def serve_specs(n=256, seed=1005):
    """Serving workload: n streams in equal thirds of the three frame sizes, ranks uniform
    on [8, 48] per bond (seeded)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        dims = SERVE_SIZES[i % 3]
        out.append((dims, tuple(int(v) for v in rng.integers(8, 49, size=len(dims)))))
    return out


def _serve_frames(nframes=6):
    """Pinned host 8-bit frames per size, the video recipe (C2-style content; 256 x 256 is
    the first channel of a 256 x 256 x 3 video frame)."""
    import torch
    from paper_2606_31061_b300 import synth
    pools = {}
    for dims in SERVE_SIZES:
        vd = dims if len(dims) == 3 else dims + (3,)
        sp = synth.make_stream("video", dims=vd, seed=1005)
        fr = [np.clip(np.rint(x), 0, 255).astype(np.uint8) for x in sp.take(nframes)]
        if len(dims) == 2:
            fr = [np.ascontiguousarray(x[..., 0]) for x in fr]
        pools[dims] = [torch.from_numpy(x).pin_memory() for x in fr]
    return pools


def serve_arm(seconds=2.0, n=256, lam=30.0, budget=150e9, slots=8, rank_step=16, quantum=0.002, check=True,
              fp64_compare=True):
    """Continuous-batching serving loop (paper_2606_31061_b300.serve) in real time: n streams,
    Poisson frame arrivals at `lam` frames/s each for `seconds`, admission by an HBM budget.
    Latency per frame = detection of its step's completion - arrival.  Ranks are rounded up
    to multiples of `rank_step` (pools of many streams) and the loop ticks every `quantum`
    seconds (several frames per pool step): per-step host cost, not the GPU, bounds a loop
    that steps one frame at a time.  Also: the drain rate
    with every frame already queued (capacity), and the per-stream FP64 path's capacity
    for the same mix of sizes."""
    import torch
    from paper_2606_31061_b300 import serve
    from paper_2606_31061_b300.ttals import Stream
    specs = serve_specs(n)
    frames = _serve_frames()
    rng = np.random.default_rng(1005)
    events = []
    for sid in range(n):
        t = np.cumsum(rng.exponential(1.0 / lam, size=int(lam * seconds * 2) + 8))
        events += [(float(tt), sid) for tt in t if tt <= seconds]
    events.sort()

    from oracle import ttals_oracle as O
    from paper_2606_31061_b300 import synth
    init = lambda sid, d, r: synth.init_cores(d, r, seed=20000 + sid)
    sample = [next(sid for sid in range(n) if specs[sid][0] == d) for d in SERVE_SIZES]
    checked = {}

    def run(evts, realtime, check=False):
        srv = serve.Server(int(budget), slots=slots, rank_step=rank_step, wire="u8", init_cores=init)
        admitted = sum(srv.connect(sid, d, r) for sid, (d, r) in enumerate(specs))
        # warm the pools (their first steps, over both input blocks and both state buffers,
        # pay one-time costs), then restart every stream
        for sid, (d, r) in enumerate(specs):
            if srv.admitted(sid):
                for j in range(4):
                    srv.submit(sid, frames[d][j % len(frames[d])], 0.0)
        while srv.backlog():
            srv.tick()
            torch.cuda.synchronize()
            srv.poll()
        srv.restart_streams()
        torch.cuda.synchronize()
        nxt = {sid: 0 for sid in range(n)}
        h2d = 0
        t0 = time.perf_counter()
        i = 0
        last_tick = -1.0
        while i < len(evts) or srv.backlog():
            now = time.perf_counter() - t0
            if realtime and now - last_tick < quantum:
                srv.poll()
                continue
            last_tick = now
            while i < len(evts) and (not realtime or evts[i][0] <= now):
                ta, sid = evts[i]
                d = specs[sid][0]
                f = frames[d][nxt[sid] % len(frames[d])]
                nxt[sid] += 1
                srv.submit(sid, f, t0 + (ta if realtime else 0.0))
                h2d += f.numel()
                i += 1
            srv.tick()
            srv.poll()
        t1 = time.perf_counter()
        if check:
            # sampled served streams (one per frame size) against the oracle on the frames they got
            for sid in sample:
                pool, slot = srv.where[sid]
                pool.batch.select(slot)
                s_ = pool.batch.stats()
                d, rr = specs[sid][0], tuple(pool.batch.ranks)
                fr = [frames[d][i % len(frames[d])].numpy().astype(np.float64) for i in range(pool.batch.step())]
                orc = O.OnlineTTALS(d, list(rr), *init(sid, d, rr))
                re_o = O.stream_relative_error(fr, [orc.step(x) for x in fr])
                re_g = math.sqrt(s_[3] / s_[2]) if s_[2] > 0 else float("nan")
                checked["x".join(map(str, d))] = {"ranks": rr, "frames": len(fr), "re_gpu": re_g,
                                                  "re_oracle": re_o, "abs_diff_re": abs(re_g - re_o)}
        out = {"frames": len(srv.latencies), "seconds": t1 - t0, "steps": srv.steps, "admitted": admitted,
               "pools": sum(len(v) for v in srv.pools.values()), "device_gb": srv.used / 1e9,
               "h2d_gbs": h2d / (t1 - t0) / 1e9, "latency_s": serve.percentiles(srv.latencies)}
        srv.close()
        torch.cuda.empty_cache()
        return out

    rt = run(events, True, check=check)
    half = [e for j, e in enumerate(events) if j % 2 == 0]     # every other arrival: lam / 2
    rt_half = run(half, True)
    cap_events = [(0.0, sid) for sid in range(n) for _ in range(4)]
    cap = run(cap_events, False)
    # per-stream FP64 path, one stream per size at the ranks its sampled served stream got, the
    # same 8-bit frames over the host link widened on the device (to FP64), wall time per frame
    from paper_2606_31061_b300.ttals import widen_u8
    fp64 = {}
    for dims in (SERVE_SIZES if fp64_compare else ()):
        rr = checked.get("x".join(map(str, dims)), {}).get("ranks") or serve.feasible_ranks(dims, (32,) * len(dims))
        st = Stream(dims, rr, ingest="f64")
        stage = torch.empty(dims, dtype=torch.uint8, device="cuda")
        x = torch.empty(dims, dtype=torch.float64, device="cuda")
        hf = frames[dims]

        def one(i):
            stage.copy_(hf[i % len(hf)], non_blocking=True)
            widen_u8(stage, x)
            st.push(x)

        for i in range(2):
            one(i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(6):
            one(i)
        torch.cuda.synchronize()
        fp64["x".join(map(str, dims))] = 6 / (time.perf_counter() - t0)
        st.close()
        del x, stage
    fp64_mix = 1.0 / sum((1.0 / 3) / v for v in fp64.values()) if fp64 else None
    lat = rt["latency_s"]
    return {
        "workload": f"{n} streams, sizes in thirds 256x256 / 720x1280x3 / 1080x1920x3, ranks U[8,48] per bond "
                    f"(rounded up to multiples of {rank_step} for pooling), Poisson arrivals {lam:g} frames/s each for "
                    f"{seconds:g} s, 8-bit frames over the host link widened to FP16 on the device, "
                    f"HBM budget {budget / 1e9:g} GB, pools of {slots} slots, ticks every {quantum * 1e3:g} ms",
        "offered_slices_s": len(events) / seconds,
        "served_slices_s": rt["frames"] / rt["seconds"],
        "latency_ms": {"p50": lat["p50"] * 1e3 if lat["p50"] is not None else None,
                       "p99": lat["p99"] * 1e3 if lat["p99"] is not None else None, "n": lat["n"],
                       "what": "frame arrival -> host detection of its step's completion event"},
        "realtime": rt,
        "half_load": {"offered_slices_s": len(half) / seconds, "served_slices_s": rt_half["frames"] / rt_half["seconds"],
                      "latency_ms": {"p50": rt_half["latency_s"]["p50"] * 1e3, "p99": rt_half["latency_s"]["p99"] * 1e3,
                                     "n": rt_half["latency_s"]["n"]}, "run": rt_half},
        "capacity_slices_s": cap["frames"] / cap["seconds"], "capacity_run": cap,
        "served_vs_oracle": checked,
        "fp64_plain_per_stream_slices_s": fp64, "fp64_plain_mix_capacity_slices_s": fp64_mix,
        "vs_fp64_plain_capacity": (cap["frames"] / cap["seconds"]) / fp64_mix if fp64_mix else None,
    }


PAPER_TABLE1_MS = {5: 15.21, 6: 545.5, 7: 17365.0}   # Online TT-ALS, ms per frame (their hardware)


def _tt_frames_gpu(dims, gen_rank, nframes, seed, decay=0.7, noise=1e-3):
    """Synthetic high-order frames built on the device (input generation only): a TT of
    ground-truth rank `gen_rank` whose cores have decaying column scales (decaying singular
    values of every unfolding), temporal weights drifting slowly, plus Gaussian noise."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    m = len(dims)
    scale = decay ** torch.arange(gen_rank, device="cuda", dtype=torch.float64)
    cores = []
    for k in range(m):
        a = 1 if k == 0 else gen_rank
        c = torch.randn((a, dims[k], gen_rank), generator=g, device="cuda", dtype=torch.float64) / math.sqrt(a * dims[k])
        cores.append(c * scale)
    w = torch.randn(gen_rank, generator=g, device="cuda", dtype=torch.float64)
    frames = []
    for t in range(nframes):
        w = 0.98 * w + 0.2 * torch.randn(gen_rank, generator=g, device="cuda", dtype=torch.float64)
        v = torch.tensordot(cores[-1], w, dims=([2], [0]))              # (r, I_m)
        for k in range(m - 2, -1, -1):
            v = torch.tensordot(cores[k], v, dims=([2], [0]))           # (a, I_k, ...)
        x = v.reshape(tuple(dims)).float()
        x = x / x.std()
        x += noise * torch.randn(x.shape, generator=g, device="cuda", dtype=torch.float32)
        frames.append(x.contiguous())
        del v
    return frames


def table1_arm(orders=(5, 6, 7), I=30, rank=8, steps=6):
    """Table-1-shaped scalability workload: slices of order n - 1 with I = 30 per mode, TT
    ranks `rank` on every bond (an assumption: the paper does not state them), FP32 ingest.
    ms per slice from CUDA events over `steps` pushes after two warm-up pushes."""
    import torch
    from paper_2606_31061_b300.ttals import Stream
    out = {}
    for n in orders:
        dims = (I,) * (n - 1)
        frames = _tt_frames_gpu(dims, rank, 4, seed=659 + n)
        st = Stream(dims, (rank,) * (n - 1), ingest="f32")
        for t in range(2):
            st.push(frames[t % 4])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for t in range(steps):
            st.push(frames[t % 4])
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        s_ = st.stats()
        nbytes = frames[0].numel() * 4
        out[f"n={n}"] = {"slice_elems": frames[0].numel(), "ms_per_slice": ms, "slices_s": 1000.0 / ms,
                         "slice_gbs": nbytes / (ms * 1e-3) / 1e9, "re": math.sqrt(s_[3] / s_[2]),
                         "paper_online_ttals_ms_per_frame": PAPER_TABLE1_MS.get(n),
                         "device_gb": st.device_bytes / 1e9}
        st.close()
        del frames
        torch.cuda.empty_cache()
    return {"workload": f"orders n = {orders}, I = {I} per mode, TT ranks {rank} on every bond (assumed), "
                        "synthetic TT fields with decaying singular values + noise 1e-3, FP32 ingest",
            "results": out,
            "paper_note": "the paper's times are on its own hardware: context, not a target"}


def e2e_arm(ingest, steps, pool_np, dist_on, wire="ingest"):
    """Same metric through the C ABI from pinned HOST buffers: per step an H2D copy of the
    slice (copy stream, double-buffered device slot), the push, and an async D2H read of
    the step's error statistics.  Copies overlap the previous step's update.
    wire = "u8": the video frames are 8-bit pixels; the host holds them as bytes, the copy
    moves bytes and ttals_widen_u8 widens them to the ingest type on the device (exact), on
    the copy stream, before the push."""
    import torch
    from paper_2606_31061_b300.ttals import Stream, widen_u8
    st = Stream(DIMS, RANKS, ingest=ingest)
    P = min(16, pool_np.shape[0])
    if wire == "u8":
        vals = torch.from_numpy(pool_np[:P])
        if ingest == "f16":
            vals = vals.view(torch.float16)
        elif ingest == "bf16":
            vals = vals.view(torch.bfloat16)
        host = vals.float().round().clamp(0, 255).to(torch.uint8).pin_memory()
        stage = [torch.empty(host.shape[1:], dtype=torch.uint8, device="cuda") for _ in range(2)]
    else:
        host = torch.from_numpy(pool_np[:P]).pin_memory()
        stage = None
    slot_shape = host.shape[1:]
    dev_dt = {"f16": torch.float16, "bf16": torch.bfloat16, "f32": torch.float32}[ingest]
    dev = [torch.empty(slot_shape, dtype=dev_dt if wire == "u8" else host.dtype, device="cuda") for _ in range(2)]
    out = torch.zeros((steps, 4), dtype=torch.float64).pin_memory()
    comp = torch.cuda.current_stream()
    copy = torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]
    for i in range(2):
        consumed[i].record(comp)

    def one(t):
        s = t % 2
        with torch.cuda.stream(copy):
            copy.wait_event(consumed[s])
            if stage is None:
                dev[s].copy_(host[pingpong(t, P)], non_blocking=True)
            else:
                stage[s].copy_(host[pingpong(t, P)], non_blocking=True)
                widen_u8(stage[s], dev[s], stream=copy)
            copied[s].record(copy)
        comp.wait_event(copied[s])
        st.push_ptr(dev[s].data_ptr(), comp.cuda_stream)
        consumed[s].record(comp)
        st.stats_async(out[t].data_ptr(), comp.cuda_stream)

    for t in range(min(3, steps)):
        one(t)
    torch.cuda.synchronize()
    if dist_on:
        import torch.distributed as dist
        dist.barrier()
    t0 = time.perf_counter()
    for t in range(steps):
        one(t)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    st.close()
    slice_bytes = int(np.prod(DIMS)) * host.element_size()
    return dict(seconds=t1 - t0, h2d=slice_bytes, d2h=4 * 8)


SENSOR_DIMS = (32, 32, 32, 32)
SENSOR_RANKS = (16, 32, 32, 16)


def sensor_arm(ingest, steps, warmup):
    """Sensor-shaped 5th-order stream (32^4 slices, ranks (16,32,32,16), abrupt change every 200
    steps), device-resident pool of frames larger than L2 played forward and backward."""
    import torch
    from paper_2606_31061_b300 import synth
    sp = synth.make_stream("sensor")
    es = 4 if ingest == "f32" else 2
    nfr = int(math.ceil(200e6 / (int(np.prod(SENSOR_DIMS)) * es)))
    pool_np = np.stack([synth.round_to_ingest(x, ingest)[0] for x in sp.frames(nfr)])
    pool = to_device(pool_np, ingest)
    r = time_arm(ingest, steps, warmup, pool, False, None, dims=SENSOR_DIMS, ranks=SENSOR_RANKS)
    sb = int(np.prod(SENSOR_DIMS)) * es
    out = {"value": steps / (r["ms"] / 1000.0), "unit": "slices/s", "ms_per_step": r["ms"] / steps,
           "slice_gbs": steps / (r["ms"] / 1000.0) * sb / 1e9, "re": r["re"], "gpu_launches": r["launches"],
           "pool_mb": pool.numel() * es / 1e6}
    del pool
    torch.cuda.empty_cache()
    return out


def oracle_check(name, dims, ranks, ingests, nframes, init_seed=7, **kw):
    """The FP64 oracle and the GPU path on the same first `nframes` frames of a stream, from the
    same initial cores, each ingest rounding the frames the way the GPU ingests them (ingests
    whose rounded frames coincide, as FP16 and FP32 do for 8-bit pixels, share one oracle
    run): per ingest the stream RE of both (Sec. 5.1), |RE_gpu - RE_oracle| and the largest
    per-slice relative difference of the reconstructions.  Also the oracle's time per slice."""
    import torch
    from oracle import ttals_oracle as O
    from paper_2606_31061_b300 import synth
    from paper_2606_31061_b300.ttals import Stream
    sp = synth.make_stream(name, **kw)
    frames = sp.take(nframes)
    r = O.clamp_ranks(dims, ranks)
    cores, g = synth.init_cores(dims, r, seed=init_seed)
    tdt = {"f64": torch.float64, "f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}
    groups = []                       # [(ingests sharing the rounded values)]
    for ing in ingests:
        e0 = synth.round_to_ingest(frames[0], ing)[1]
        for grp in groups:
            if np.array_equal(synth.round_to_ingest(frames[0], grp[0])[1], e0):
                grp.append(ing)
                break
        else:
            groups.append([ing])
    res, orc_s, orc_n = {}, 0.0, 0
    for grp in groups:
        sts = {}
        for ing in grp:
            sts[ing] = Stream(dims, ranks, ingest=ing)
            sts[ing].set_cores(cores, g)
        out = torch.empty(tuple(dims), dtype=torch.float64, device="cuda")
        orc = O.OnlineTTALS(dims, r, cores, g)
        acc = {ing: [0.0, 0.0] for ing in grp}      # [sum ||x - x^_gpu||^2, worst per-slice]
        num_o = den = 0.0
        for x in frames:
            exact = None
            for ing in grp:
                payload, exact = synth.round_to_ingest(x, ing)
                t = torch.from_numpy(np.ascontiguousarray(payload))
                if ing in ("f16", "bf16"):
                    t = t.view(tdt[ing])
                sts[ing].push(t.cuda())
            a = time.perf_counter()
            xo = orc.step(exact)
            orc_s += time.perf_counter() - a
            orc_n += 1
            nxo = max(float(np.linalg.norm(xo)), 1e-300)
            for ing in grp:
                sts[ing].reconstruct(out, "f64")
                xg = out.cpu().numpy()
                acc[ing][0] += float(np.sum((exact - xg) ** 2))
                acc[ing][1] = max(acc[ing][1], float(np.linalg.norm(xg - xo)) / nxo)
            num_o += float(np.sum((exact - xo) ** 2))
            den += float(np.sum(exact * exact))
        re_o = math.sqrt(num_o / den)
        for ing in grp:
            sts[ing].close()
            re_g = math.sqrt(acc[ing][0] / den)
            res[ing] = {"re_gpu": re_g, "re_oracle": re_o, "abs_diff_re": abs(re_g - re_o),
                        "max_rel_diff_per_slice": acc[ing][1]}
    return {"frames": nframes, "per_ingest": res, "oracle_s_per_slice": orc_s / max(1, orc_n)}


def ablation_arm(T=500, dims=(60, 80, 3), ranks=(30, 3, 3)):
    """Sec. 5.4 ablation (Table ablation_ortho): the relative error of the stream so far at
    t = 10, 100, 500 with orthogonalisation (literal) and without it (noortho: LQ/QR removed,
    Gram-inverse local solves), on the GPU in FP64 and FP32 ingest and in the oracle, for a
    colour-video-shaped stream with the paper's ranks (30,3,3) (synthetic stand-in for the
    paper's continuousPan sequence, which is not available)."""
    import torch
    from oracle import ttals_oracle as O
    from paper_2606_31061_b300 import synth
    from paper_2606_31061_b300.ttals import Stream
    sp = synth.make_stream("video", dims=dims)
    frames = sp.take(T)
    r = O.clamp_ranks(dims, ranks)
    cores, g = synth.init_cores(dims, r, seed=7)
    marks = (10, 100, 500)
    out = {}
    for mode in ("literal", "noortho"):
        for ingest in ("f64", "f32"):
            st = Stream(dims, ranks, ingest=ingest, mode=mode)
            st.set_cores(cores, g)
            dt = torch.float64 if ingest == "f64" else torch.float32
            curve = {}
            for t, x in enumerate(frames, 1):
                st.push(torch.from_numpy(x).to(dt).cuda())
                if t in marks:
                    s_ = st.stats()
                    curve[t] = math.sqrt(s_[3] / s_[2])
            st.close()
            out[f"gpu_{ingest}_{mode}"] = curve
        orc = O.OnlineTTALS(dims, r, cores, g, mode=mode)
        num = den = 0.0
        curve = {}
        for t, x in enumerate(frames, 1):
            xh = orc.step(x)
            num += float(np.sum((x - xh) ** 2))
            den += float(np.sum(x * x))
            if t in marks:
                curve[t] = math.sqrt(num / den)
        out[f"oracle_{mode}"] = curve
    return {"workload": f"colour-video-shaped stream {dims[0]}x{dims[1]}x{dims[2]}, ranks {ranks}, T = {T}",
            "re_at_t": out,
            "paper_continuousPan": {"w/o Ortho": {10: 0.097, 100: 0.147, 500: 0.203},
                                    "w/ Ortho": {10: 0.097, 100: 0.100, 500: 0.100}}}


def cpu_baseline_oracle(ingest, budget_s=15.0, max_steps=None):
    """The FP64 oracle (test infrastructure) on the host cores, on a bounded prefix of the
    same stream: returns (slices/s, steps, threads, seconds)."""
    from oracle import ttals_oracle as O
    from paper_2606_31061_b300 import synth
    try:
        from threadpoolctl import threadpool_info
        threads = max([d.get("num_threads", 1) for d in threadpool_info()] + [1])
    except Exception:
        threads = os.cpu_count() or 1
    sp = synth.make_stream("video")
    r = O.clamp_ranks(DIMS, RANKS)
    cores, g = synth.init_cores(DIMS, r, seed=7)
    orc = O.OnlineTTALS(DIMS, r, cores, g)
    gen = sp.frames(10_000)
    done, spent = 0, 0.0
    while spent < budget_s and (max_steps is None or done < max_steps):
        x = next(gen)
        _, exact = synth.round_to_ingest(x, ingest)
        a = time.perf_counter()
        orc.step(exact)
        spent += time.perf_counter() - a
        done += 1
    return done / spent, done, threads, spent


def run_reference(args, rank):
    if rank != 0:
        return
    budget = 120.0
    rate, done, threads, spent = cpu_baseline_oracle(args.ingest, budget_s=budget,
                                                     max_steps=max(1, args.steps))
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "slices/s", "n_gpus": args.gpus,
        "steps": done, "warmup": 0, "ms_per_step": 1000.0 / rate, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "ingest": args.ingest, "parallelism": "host cores"},
        "cpu_baseline": {"value": rate, "unit": "slices/s", "cores": threads, "kind": "oracle",
                         "sample": f"first {done} frames of the stream (of {args.steps} requested; "
                                   f"capped at {budget:.0f} s of oracle time), FP64 literal Algorithm 1"},
        "e2e": {"value": rate, "unit": "slices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def profile_case(args):
    """Untimed pushes for a profiler capture: one video stream (profile_case = "single"), a
    batch of args.batch video streams ("batched"), or one sensor-shaped stream in FP32 on the
    generic path ("sensor"), args.warmup + args.steps pushes."""
    import torch
    from paper_2606_31061_b300.ttals import Stream
    if args.profile_case == "sensor":
        from paper_2606_31061_b300 import synth
        sp = synth.make_stream("sensor")
        pool = to_device(np.stack([synth.round_to_ingest(x, "f32")[0] for x in sp.take(4)]), "f32")
        st = Stream(SENSOR_DIMS, SENSOR_RANKS, ingest="f32")
        h = torch.cuda.current_stream().cuda_stream
        for t in range(args.warmup + args.steps):
            st.push_ptr(pool[t % 4].data_ptr(), h)
        torch.cuda.synchronize()
        st.sync()
        st.close()
        return
    S = args.batch if args.profile_case == "batched" else 0
    pool = to_device(make_pool(args.ingest, max(8, S + 4)), args.ingest)
    st = Stream(DIMS, RANKS, ingest=args.ingest, n_streams=S)
    h = torch.cuda.current_stream().cuda_stream
    for t in range(args.warmup + args.steps):
        if S:
            st.push_batch_ptr(pool[t % 4].data_ptr(), h)
        else:
            st.push_ptr(pool[t % 8].data_ptr(), h)
    torch.cuda.synchronize()
    st.sync()
    st.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ingest", default="f16", choices=["f16", "f32", "bf16"])
    ap.add_argument("--pool", type=int, default=64)
    ap.add_argument("--no-f32", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=300)
    ap.add_argument("--batch", type=int, default=32, help="streams per batched push (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=400)
    ap.add_argument("--c4-steps", type=int, default=200, help="mixed-shape group steps (0: skip)")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="serving-loop traffic (0: skip)")
    ap.add_argument("--table1", type=int, default=1, help="high-order scalability arm (0: skip)")
    ap.add_argument("--sensor-steps", type=int, default=300, help="sensor-shaped stream arm (0: skip)")
    ap.add_argument("--ablation", type=int, default=1, help="Sec. 5.4 orthogonality ablation arm (0: skip)")
    ap.add_argument("--oracle-frames", type=int, default=40,
                    help="prefix on which the oracle is timed and compared with the GPU path")
    ap.add_argument("--profile-case", default=None, choices=["single", "batched", "sensor"],
                    help="for profilers: run --warmup + --steps pushes of one video stream, of a "
                         "batch of --batch video streams, or of one FP32 sensor-shaped stream, untimed, "
                         "and print no bench line")
    args = ap.parse_args()
    rank = env_int("RANK", 0)
    world = env_int("WORLD_SIZE", 1)
    local = env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.warmup < 3:
        args.warmup = 3
    import torch
    torch.cuda.set_device(local)
    dist_on = world > 1
    if dist_on:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2606_31061_b300 import build
    if rank == 0 or not dist_on:
        build.build()
    if args.profile_case:
        profile_case(args)
        return
    if dist_on:
        torch.distributed.barrier()
    pool_np = make_pool(args.ingest, args.pool)
    pool = to_device(pool_np, args.ingest)
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    smi_idx = int(vis.split(",")[local]) if vis else local
    r = time_arm(args.ingest, args.steps, args.warmup, pool, dist_on, smi_idx if rank == 0 else None)
    sec = r["ms"] / 1000.0
    if dist_on:
        t = torch.tensor([sec], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        sec = float(t.item())
    value = args.steps * world / sec
    es = pool.element_size()
    slice_bytes = int(np.prod(DIMS)) * es
    r1, rest1, i1 = 32, 1920 * 3, 1080
    # algorithmic bytes per launch: each operand read once, each result written once
    alg = {"solve": slice_bytes + r1 * rest1 * es + i1 * r1 * 4,          # X, C (ingest copy) -> Y
           "factor": i1 * r1 * 4 + i1 * r1 * (es + 4),                   # Y -> Q1 (ingest copy + FP32)
           "env": slice_bytes + i1 * r1 * es + r1 * rest1 * (4 + es)}    # X, Q1 -> C (FP32 + ingest copy)
    npush = max(1, r["npush"])
    per = {"solve": r["ms_solve"] / npush, "factor": r["ms_factor"] / npush, "env": r["ms_env"] / npush}
    dom = max(per, key=per.get)
    peak, peak_src = peaks()
    ach = {k: alg[k] / (per[k] * 1e-3) / 1e9 for k in per}
    knames = {"solve": "k_fast_solve: level-1 local solve Y = X_(1) B^_1^T (S4, slice contraction)",
              "factor": "k_fast_factor: level-1 r x r factor and basis Q1 = orth(Y) (S5)",
              "env": "k_fast_env1: level-1 environment E_2 = Q1^T X_(1) (S6, slice contraction)"}
    # the same stream with the FP32 r x r factor (the faster variant, for comparison)
    r32f = time_arm(args.ingest, args.steps, args.warmup, pool, dist_on, None, factor="fp32")
    factor_fp32 = {"value": args.steps * world / (r32f["ms"] / 1000.0), "unit": "slices/s",
                   "ms_per_step": r32f["ms"] / args.steps,
                   "ms_factor_per_launch": r32f["ms_factor"] / max(1, r32f["npush"]), "re": r32f["re"]}
    # end to end: 8-bit video frames over the host link, widened on the device (the pixels
    # are integers 0..255, exact in FP16); the FP16-frame variant is reported beside it
    wire = "u8" if args.ingest in ("f16", "bf16") else "ingest"
    e2e = e2e_arm(args.ingest, args.e2e_steps, pool_np, dist_on, wire=wire)
    e2e16 = e2e_arm(args.ingest, args.e2e_steps, pool_np, dist_on) if wire == "u8" else None
    e2e_sec = e2e["seconds"]
    if dist_on:
        t = torch.tensor([e2e_sec], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_sec = float(t.item())
    batched = None
    if args.batch > 0:
        S = min(args.batch, args.pool)
        rb = batched_arm(args.ingest, S, args.batch_steps, args.warmup, pool)
        bsec = rb["ms"] / 1000.0
        if dist_on:
            t = torch.tensor([bsec], device="cuda")
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            bsec = float(t.item())
        nb = max(1, rb["npush"])
        bper = {"solve": rb["ms_solve"] / nb, "factor": rb["ms_factor"] / nb, "env": rb["ms_env"] / nb}
        bdom = max(bper, key=bper.get)
        blat = rb["lat"]
        bach = {k: S * alg[k] / (bper[k] * 1e-3) / 1e9 for k in bper}
        batched = {
            "streams": S, "steps": args.batch_steps,
            "value": args.batch_steps * S * world / bsec, "unit": "slices/s",
            "ms_per_step": rb["ms"] / args.batch_steps,
            "hbm_gbs": args.batch_steps * S * world / bsec * slice_bytes / 1e9,
            "gpu_launches": rb["launches"],
            "latency_ms": {"p50": blat[len(blat) // 2], "p99": blat[min(len(blat) - 1, int(0.99 * len(blat)))],
                           "n": len(blat), "what": "one batched push (every stream's slice of that step)"},
            "re_per_stream": {"min": min(rb["re"]), "max": max(rb["re"])},
            "roofline": {"bound": "hbm", "kernel": bdom, "achieved": bach[bdom], "peak": peak,
                         "peak_source": peak_src, "unit": "GB/s", "frac": bach[bdom] / peak,
                         "traffic": traffic_record(f"batched{S}", {"solve": "solve", "env": "env_stream",
                                                                   "factor": "factor"}[bdom]),
                         "algorithmic_bytes": S * alg[bdom], "ms_per_launch": bper[bdom],
                         "achieved_all": bach, "ms_per_launch_all": bper},
            "inputs": f"stream b at step t reads pool frame o_t + b; one push reads {S * slice_bytes / 1e6:.0f} MB",
        }
    c4 = c4_arm(args.c4_steps) if args.c4_steps > 0 else None
    ablation = ablation_arm() if args.ablation and world == 1 else None
    sensor = None
    if args.sensor_steps > 0 and world == 1:
        sensor = {ing: sensor_arm(ing, args.sensor_steps, args.warmup) for ing in ("f32", "bf16")}
    served = serve_arm(args.serve_seconds) if args.serve_seconds > 0 and world == 1 else None
    table1 = table1_arm() if args.table1 and world == 1 else None
    f32 = None
    if not args.no_f32 and args.ingest != "f32":
        del pool
        torch.cuda.empty_cache()
        pool32_np = make_pool("f32", min(args.pool, 48))
        pool32 = to_device(pool32_np, "f32")
        r32 = time_arm("f32", args.steps, args.warmup, pool32, dist_on, None)
        f32 = {"value": args.steps * world / (r32["ms"] / 1000.0), "unit": "slices/s",
               "ms_per_step": r32["ms"] / args.steps, "re": r32["re"],
               "hbm_gbs": args.steps * world / (r32["ms"] / 1000.0) * int(np.prod(DIMS)) * 4 / 1e9}
        del pool32
    cpu = None
    checks = {}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on a bounded prefix of the headline stream, the GPU path in lockstep on the
        # same frames (FP16 and FP32 ingest share the oracle run: the frames are integers); its
        # time per slice is the CPU baseline
        vc = oracle_check("video", DIMS, RANKS, [args.ingest, "f32"], args.oracle_frames)
        checks["video"] = vc
        try:
            from threadpoolctl import threadpool_info
            threads = max([d.get("num_threads", 1) for d in threadpool_info()] + [1])
        except Exception:
            threads = os.cpu_count() or 1
        cpu = {"value": 1.0 / vc["oracle_s_per_slice"], "unit": "slices/s", "cores": threads, "kind": "oracle",
               "sample": f"first {vc['frames']} frames of the same stream "
                         f"({vc['frames'] * vc['oracle_s_per_slice']:.1f} s), FP64 literal Algorithm 1"}
        if sensor is not None:
            checks["sensor"] = oracle_check("sensor", SENSOR_DIMS, SENSOR_RANKS, ["f32", "bf16"],
                                            args.oracle_frames)
    bat_roof = {}
    if batched is not None:
        bro = batched["roofline"]
        b_alg = S * alg["solve"]
        bat_roof = {"batched_streams": S,
                    "batched_solve_frac": bro["achieved_all"]["solve"] / peak,
                    "batched_env_frac": bro["achieved_all"]["env"] / peak,
                    "batched_step_gbs_slice_once": batched["hbm_gbs"],
                    "batched_step_frac_slice_once": batched["hbm_gbs"] / peak}
        del b_alg
    lat = r["lat"]
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "slices/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.ingest, "data": "synthetic",
            "config": {"workload": WORKLOAD, "ingest": args.ingest,
                       "precision": (f"{args.ingest.upper()} ingest, FP32 accumulation and state; FP64 r x r factor "
                                     "of each local solve's Gram (fraction-free LDL^T, Gram summed in FP64 from FP32 "
                                     "partials); FP32 tall apply rounded to the ingest type with an exact projector "
                                     "correction for the rounded basis") if args.ingest != "f32" else
                                    "FP32 ingest and state; Cholesky-QR (FP32 factor, FP64 sums) + FP64 polar pass",
                       "oracle_check": "; ".join(
                           f"{k} first {v['frames']} frames: " + ", ".join(
                               f"{ing} |RE_gpu - RE_oracle| {d['abs_diff_re']:.2e} (RE {d['re_oracle']:.5f}), "
                               f"max per-slice rel diff {d['max_rel_diff_per_slice']:.2e}"
                               for ing, d in v["per_ingest"].items()) for k, v in checks.items()),
                       "l2": f"inputs larger than L2: {args.pool}-frame pool "
                             f"({args.pool * slice_bytes / 1e6:.0f} MB), played forward and backward",
                       "parallelism": f"replicas x{world}" if world > 1 else "single stream"},
            "hbm_gbs": value * slice_bytes / 1e9,
            "host_enqueue_us_per_step": r["host_us"],
            "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                           "n": len(lat)},
            "re": r["re"],
            "roofline": dict({"bound": "hbm", "kernel": knames["solve"], "achieved": ach["solve"], "peak": peak,
                              "peak_source": peak_src, "unit": "GB/s", "frac": ach["solve"] / peak,
                              "traffic": traffic_record("solve"),
                              "algorithmic_bytes": alg["solve"], "ms_per_launch": per["solve"],
                              "env_kernel": knames["env"], "env_achieved": ach["env"], "env_frac": ach["env"] / peak,
                              "env_ms_per_launch": per["env"],
                              "dominant_kernel": knames[dom], "dominant_achieved": ach[dom],
                              "dominant_frac": ach[dom] / peak, "dominant_ms_per_launch": per[dom],
                              "dominant_step_share": per[dom] / (r["ms_push"] / npush),
                              "factor_ms_per_launch": per["factor"]}, **bat_roof),
            "factor_fp32": factor_fp32,
            "sensor": sensor,
            "ablation_ortho": ablation,
            "oracle_checks": checks,
            "e2e": {"value": args.e2e_steps * world / e2e_sec, "unit": "slices/s",
                    "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"],
                    "wire": "8-bit pixels, widened to the ingest type on the device (ttals_widen_u8)"
                            if wire == "u8" else args.ingest},
            "e2e_f16_wire": ({"value": args.e2e_steps / e2e16["seconds"], "unit": "slices/s",
                              "h2d_bytes_per_step": e2e16["h2d"], "d2h_bytes_per_step": e2e16["d2h"]}
                             if e2e16 else None),
            "gpu_launches": r["launches"],
            "clocks": r["clocks"],
            "batched": batched,
            "c4_mixed_shapes": c4,
            "serving": served,
            "table1_high_order": table1,
            "f32_ingest": f32,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist_on:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
