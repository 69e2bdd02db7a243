"""Serving loop on the GPU (paper_2606_31061_b300.serve): every stream served in the mix --
frames of many streams arriving interleaved, masked batch steps, slots reused after a
stream leaves -- ends within the FP16 ingest tolerance of the same stream run alone
(every reconstructed slice within 1e-3 relative, RE within 1e-3 absolute), with the same
number of steps."""
import numpy as np
import pytest

from paper_2606_31061_b300 import synth

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    from paper_2606_31061_b300 import build
    build.build()
    return torch


def _init(sid, dims, ranks):
    return synth.init_cores(dims, ranks, seed=500 + sid)


def _frames(torch, name, kw, sid, T):
    sp = synth.make_stream(name, seed=8000 + 11 * sid, **kw)
    xs = [synth.round_to_ingest(x, "f16")[0] for x in sp.take(T)]
    return [torch.from_numpy(x).view(torch.float16).pin_memory() for x in xs]


def _alone(torch, dims, ranks, sid, frames):
    from paper_2606_31061_b300.ttals import Stream
    st = Stream(dims, ranks, ingest="f16")
    st.set_cores(*_init(sid, dims, st.ranks))
    out = torch.empty(tuple(dims), dtype=torch.float64, device="cuda")
    for f in frames:
        st.push(f.cuda())
    st.reconstruct(out, "f64")
    res = out.cpu().numpy().copy(), np.array(st.stats()), st.step()
    st.close()
    return res


def _served(torch, server, sid, dims):
    st = server.stream(sid)
    out = torch.empty(tuple(dims), dtype=torch.float64, device="cuda")
    st.reconstruct(out, "f64")
    return out.cpu().numpy().copy(), np.array(st.stats()), st.step()


def _close(a, b, what):
    rel = np.linalg.norm(a[0] - b[0]) / np.linalg.norm(b[0])
    assert rel <= 1e-3, (what, rel)
    ra, rb = np.sqrt(a[1][3] / a[1][2]), np.sqrt(b[1][3] / b[1][2])
    assert abs(ra - rb) <= 1e-3, (what, ra, rb)
    assert a[2] == b[2], what


def _drain(server):
    import torch
    while server.backlog():
        server.tick()
        torch.cuda.synchronize()
        server.poll()


def test_serving_mix_matches_alone():
    torch = _torch()
    from paper_2606_31061_b300 import serve
    shapes = [("video", {"dims": (96, 128, 3)}, (20, 10, 3)), ("square", {"s": 128, "r": 8}, (8, 8))]
    srv = serve.Server(8 << 30, slots=4, rank_step=16, init_cores=_init)
    rng = np.random.default_rng(5)
    streams = {}
    for sid in range(6):
        name, kw, ranks = shapes[sid % 2]
        dims = kw["dims"] if "dims" in kw else (kw["s"], kw["s"])
        T = 3 + sid % 3
        streams[sid] = (dims, srv.key(dims, ranks)[1], _frames(torch, name, kw, sid, T))
        assert srv.connect(sid, dims, ranks)
    # Poisson-like interleaved arrivals, served tick by tick as they come
    events = []
    for sid, (_, _, fr) in streams.items():
        t = np.cumsum(rng.exponential(1.0 / 30, size=len(fr)))
        events += [(float(t[k]), sid, k) for k in range(len(fr))]
    events.sort()
    last = {}
    for ta, sid, k in events:
        assert last.get(sid, -1) == k - 1
        last[sid] = k
        srv.submit(sid, streams[sid][2][k], ta)
        if rng.random() < 0.5:
            srv.tick()
    _drain(srv)
    assert len(srv.latencies) == len(events) and srv.steps < len(events)
    for sid, (dims, ranks, fr) in streams.items():
        _close(_served(torch, srv, sid, dims), _alone(torch, dims, ranks, sid, fr), sid)
    srv.close()


def test_serving_budget_queues_then_reuses_slot():
    torch = _torch()
    from paper_2606_31061_b300 import serve
    dims, ranks = (128, 128), (16, 16)
    srv = serve.Server(1 << 40, slots=2, rank_step=16, init_cores=_init)
    frames = {sid: _frames(torch, "square", {"s": 128, "r": 16}, sid, 3) for sid in range(3)}
    assert srv.connect(0, dims, ranks)
    srv.budget = srv.used                       # room for exactly this one pool of two slots
    assert srv.connect(1, dims, ranks)
    assert not srv.connect(2, dims, ranks) and list(srv.waiting) == [2]
    for k in range(3):
        for sid in (0, 1):
            srv.submit(sid, frames[sid][k], 0.0)
    _drain(srv)
    first = _served(torch, srv, 0, dims)
    srv.disconnect(0)                           # stream 2 takes slot 0, reset to its own cores
    assert srv.admitted(2) and srv.where[2][1] == 0
    for k in range(3):
        srv.submit(2, frames[2][k], 0.0)
    _drain(srv)
    _close(first, _alone(torch, dims, srv.key(dims, ranks)[1], 0, frames[0]), 0)
    _close(_served(torch, srv, 1, dims), _alone(torch, dims, srv.key(dims, ranks)[1], 1, frames[1]), 1)
    _close(_served(torch, srv, 2, dims), _alone(torch, dims, srv.key(dims, ranks)[1], 2, frames[2]), 2)
    srv.close()


def test_u8_wire_bitwise_equals_f16_wire():
    """8-bit frames widened on the device (ttals_widen_u8) give bitwise the results of the
    same frames sent as FP16 (the widening is exact)."""
    torch = _torch()
    from paper_2606_31061_b300 import serve
    from paper_2606_31061_b300.ttals import widen_u8
    dims, ranks = (96, 128, 3), (20, 10, 3)
    sp = synth.make_stream("video", dims=dims, seed=4242)
    raw = [np.clip(np.rint(x), 0, 255).astype(np.uint8) for x in sp.take(3)]
    u8 = [torch.from_numpy(x).pin_memory() for x in raw]
    f16 = [torch.from_numpy(x.astype(np.float16)).pin_memory() for x in raw]
    # the widening itself, with a ragged tail (n % 16 != 0)
    src = torch.from_numpy(raw[0].reshape(-1)[:1000 - 3].copy()).cuda()
    for dt in (torch.float16, torch.bfloat16, torch.float32):
        dst = torch.empty(src.numel(), dtype=dt, device="cuda")
        widen_u8(src, dst)
        torch.cuda.synchronize()
        assert torch.equal(dst.cpu().float(), src.cpu().float()), dt
    out = []
    for wire, fr in (("u8", u8), ("f16", f16)):
        srv = serve.Server(8 << 30, slots=2, rank_step=16, init_cores=_init, wire=wire)
        assert srv.connect(0, dims, ranks)
        for f in fr:
            srv.submit(0, f, 0.0)
        _drain(srv)
        out.append(_served(torch, srv, 0, dims))
        srv.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_seed_cores_matches_create_seed():
    """ttals_seed_cores draws the library's own default initial cores: a batch slot seeded with
    x steps bitwise like a fresh stream created with cfg.seed = x (the serving loop seeds every
    admitted stream this way, without the test-input generator)."""
    torch = _torch()
    from paper_2606_31061_b300.ttals import Stream
    dims, ranks = (96, 128, 3), (32, 9, 3)
    frames = [f.cuda() for f in _frames(torch, "video", {"dims": dims}, 3, 3)]
    out_a = torch.empty(dims, dtype=torch.float64, device="cuda")
    out_b = torch.empty_like(out_a)
    a = Stream(dims, ranks, ingest="f16", seed=777)
    b = Stream(dims, ranks, ingest="f16", seed=123)
    for f in frames[:2]:
        b.push(f)                                  # some history that the reseed must erase
    b.seed_cores(777)
    assert b.step() == 0
    for f in frames:
        a.push(f)
        b.push(f)
    a.reconstruct(out_a, "f64")
    b.reconstruct(out_b, "f64")
    assert torch.equal(out_a, out_b)
    assert np.array_equal(a.stats(), b.stats()) and a.step() == b.step() == 3


def test_host_ingest_matches_masked_push():
    """ttals_batch_push_host (the library copies the frames, widens 8-bit pixels, steps the
    streams given a frame) computes bitwise what ttals_push_batch_masked computes on the same
    values, and its tickets complete in order."""
    torch = _torch()
    from paper_2606_31061_b300.ttals import Stream
    dims, ranks = (96, 128, 3), (32, 9, 3)
    fr = {sid: _frames(torch, "video", {"dims": dims}, sid, 3) for sid in range(3)}
    u8 = {sid: [torch.from_numpy(f.view(torch.float16).float().numpy().astype("uint8")).pin_memory() for f in fr[sid]]
          for sid in fr}
    a = Stream(dims, ranks, ingest="f16", n_streams=3)
    b = Stream(dims, ranks, ingest="f16", n_streams=3)
    a.ingest_init(u8=True)
    for q in range(3):
        for st in (a, b):
            st.select(q)
            st.set_cores(*_init(q, dims, st.ranks))
    plan = [{0: 0, 1: 0, 2: 0}, {0: 1, 2: 1}, {1: 1, 2: 2}]      # slot -> frame index
    tickets = []
    for step in plan:
        slots = sorted(step)
        tickets.append(a.push_host(slots, [u8[q][step[q]].data_ptr() for q in slots]))
        blk = torch.zeros((3,) + dims, dtype=torch.float16, device="cuda")
        mask = 0
        for q in slots:
            blk[q] = fr[q][step[q]].cuda()
            mask |= 1 << q
        b.push_batch(blk, active=mask)
    torch.cuda.synchronize()
    assert tickets == [0, 1, 2] and all(a.ticket_done(t) for t in tickets)
    for q in range(3):
        oa, ob = (torch.empty(dims, dtype=torch.float64, device="cuda") for _ in range(2))
        a.select(q)
        b.select(q)
        a.reconstruct(oa, "f64")
        b.reconstruct(ob, "f64")
        assert torch.equal(oa, ob) and np.array_equal(a.stats(), b.stats()) and a.step() == b.step()
