"""Request server (fb_fft_server_*): every result is the same alone and in the
mix (batched or not), matches the FP64 oracle, admission respects the
device-memory budget, cancellation and rejection behave as documented."""
import math

import numpy as np
import pytest

import oracle
from paper_2004_09883_gb300 import inputs

pytestmark = pytest.mark.gpu

FWD, INV = -1, 1


def tol(n: int) -> float:
    return 2e-6 * math.log2(n) if n > 1 else 1e-7


# 5 ** 9 has no split into two factors <= 2048: it runs per request, through its plan
MIX = [(4096,), (256,), (1 << 20,), (1 << 22,), (6000,), (3 * 5 ** 6,), (60, 45), (512, 512), (16, 250),
       (128, 128, 128), (8, 100, 27), (1,), (2,), (1000, 1), (80000,), (96, 96), (8, 8, 8), (45, 64, 125),
       (5 ** 9,), (1, 8), (6, 4, 1)]


def _mix(seed, copies=3):
    shapes = [s for _ in range(copies) for s in MIX]
    rng = np.random.default_rng(seed)
    rng.shuffle(shapes)
    dirs = [FWD if rng.random() < 0.6 else INV for _ in shapes]
    return shapes, dirs


def _alone(fb, torch, shape, direction, x):
    """The request on its own through the per-call API."""
    with fb.Plan(list(shape), 1) as p:
        y = p.exec(x, None, direction)
        torch.cuda.synchronize()
        p.check()
    return y


def _served_alone(fb, torch, shape, direction, x, scale=False):
    """The request on its own through a fresh batching server (a batch of one)."""
    y = torch.empty_like(x)
    with fb.Server(slots=1, hbm_cap_bytes=1 << 30) as srv:
        srv.submit_ptr(tuple(shape), x.data_ptr(), y.data_ptr(), 0, direction, scale_inv_n=scale)
        srv.drain()
        assert [r[:2] for r in srv.poll()] == [(0, 0)]
    return y


@pytest.mark.parametrize("slots,max_batch", [(1, 1), (8, 1), (1, 256), (8, 256)])
def test_mix_equals_alone_and_oracle(fb, slots, max_batch):
    """Without batching every result has the per-call plan's bits; with it,
    the bits of the same request served alone."""
    import torch
    from paper_2004_09883_gb300 import serving
    shapes, dirs = _mix(1200 + slots)
    w = serving.Workload(shapes, 7000, dirs)
    arrivals = serving.poisson_arrivals(len(shapes), 20000.0, 5)
    with fb.Server(slots=slots, hbm_cap_bytes=1 << 30, max_batch=max_batch) as srv:
        serving.run_served(srv, w, arrivals)
        st = srv.stats()
    assert st["completed"] == len(shapes) and st["rejected"] == 0
    assert st["max_busy_slots"] <= slots
    assert st["arena_peak"] <= st["arena_bytes"]
    if max_batch == 1:
        assert st["batches"] == 0 and st["max_in_flight"] <= slots
    else:
        assert st["batched_requests"] == sum(1 for s in shapes if s != (5 ** 9,))
    checked = set()
    for i, (s, d) in enumerate(zip(shapes, dirs)):
        if max_batch == 1 or s == (5 ** 9,):
            y_alone = _alone(fb, torch, s, d, w.x[i])
        else:
            y_alone = _served_alone(fb, torch, s, d, w.x[i])
        assert torch.equal(w.y[i], y_alone), f"request {i} {s}: mix result differs from alone"
        if (s, d) not in checked:  # each distinct request kind once against the oracle
            checked.add((s, d))
            ref = oracle.fft(w.x[i].cpu().numpy().astype(np.complex128).reshape(s), list(s), d)
            err = oracle.rel_l2(w.y[i].cpu().numpy().reshape(1, -1), ref.reshape(1, -1))[0]
            assert err <= tol(int(np.prod(s))), f"{s} dir {d}: rel L2 {err:.3e}"


@pytest.mark.parametrize("max_batch", [1, 256])
def test_host_arrays_through_staging(fb, max_batch):
    """Host arrays, all queued at once (so batches form): each result equals
    the same request on device arrays alone."""
    import torch
    from paper_2004_09883_gb300 import serving
    shapes, dirs = _mix(1300, copies=1)
    w = serving.Workload(shapes, 7100, dirs, host=True)
    with fb.Server(slots=4, hbm_cap_bytes=256 << 20, max_batch=max_batch) as srv:
        serving.run_served(srv, w, np.zeros(len(shapes)), host_io=True)
        st = srv.stats()
    assert st["arena_in_use"] == 0 and 0 < st["arena_peak"] <= 256 << 20
    if max_batch > 1:
        assert st["largest_batch"] > 1
    for i, (s, d) in enumerate(zip(shapes, dirs)):
        if max_batch == 1 or s == (5 ** 9,):
            y_alone = _alone(fb, torch, s, d, w.x[i]).cpu()
        else:
            y_alone = _served_alone(fb, torch, s, d, w.x[i]).cpu()
        assert torch.equal(w.hy[i], y_alone), f"request {i} {s}"


def test_in_place_host_request(fb):
    x = inputs.uniform_c64((3, 4096), 77)
    import torch
    h = torch.from_numpy(x.copy()).pin_memory()
    with fb.Server(slots=2, hbm_cap_bytes=64 << 20) as srv:
        srv.submit_ptr([4096], h.data_ptr(), h.data_ptr(), 1, FWD, batch=3, host_io=True)
        srv.drain()
        (tag, st, *_), = srv.poll()
    assert (tag, st) == (1, 0)
    ref = oracle.fft(x.astype(np.complex128), [4096], FWD)
    err = oracle.rel_l2(h.numpy().reshape(3, -1), ref.reshape(3, -1))
    assert err.max() <= tol(4096)


def test_budget_holds_requests_back(fb):
    """Arena for one host request at a time: the others wait in FIFO order."""
    import torch
    n = 1 << 20
    need = n * 8 + n * 8  # staging + four-step scratch
    xs = [torch.from_numpy(inputs.uniform_c64((n,), 80 + i)).pin_memory() for i in range(4)]
    ys = [torch.empty_like(v).pin_memory() for v in xs]
    with fb.Server(slots=4, hbm_cap_bytes=need + need // 2) as srv:
        for i in range(4):
            srv.submit_ptr([n], xs[i].data_ptr(), ys[i].data_ptr(), i, FWD, host_io=True)
        srv.drain()
        done = srv.poll()
        st = srv.stats()
    assert [d[0] for d in sorted(done, key=lambda d: d[4])] == [0, 1, 2, 3]  # admitted in FIFO order
    assert st["max_in_flight"] == 1 and st["arena_peak"] <= need + need // 2
    for i in range(4):
        ref = oracle.fft(xs[i].numpy().astype(np.complex128), [n], FWD)
        assert oracle.rel_l2(ys[i].numpy().reshape(1, -1), ref.reshape(1, -1))[0] <= tol(n)


def test_over_budget_and_bad_requests_rejected(fb):
    import torch
    x = torch.zeros(1 << 16, dtype=torch.complex64, device="cuda")
    h = torch.zeros(1 << 18, dtype=torch.complex64).pin_memory()
    with fb.Server(slots=2, hbm_cap_bytes=1 << 20) as srv:
        with pytest.raises(fb.FFTError) as e:  # 2 MiB staging + 2 MiB four-step scratch > 1 MiB
            srv.submit_ptr([1 << 18], h.data_ptr(), h.data_ptr(), 0, FWD, host_io=True)
        assert e.value.status == -9
        with pytest.raises(fb.FFTError) as e:
            srv.submit_ptr([7], x.data_ptr(), x.data_ptr(), 1, FWD)
        assert e.value.status == -2
        with pytest.raises(fb.FFTError) as e:
            srv.submit_ptr([64], x.data_ptr(), x.data_ptr(), 2, 0)
        assert e.value.status == -1
        with pytest.raises(fb.FFTError) as e:  # partial overlap of device in/out
            srv.submit_ptr([64], x.data_ptr(), x.data_ptr() + 8, 3, FWD)
        assert e.value.status == -1
        srv.submit_ptr([64], x.data_ptr(), x.data_ptr(), 4, FWD)  # in place is fine
        srv.drain()
        assert [d[:2] for d in srv.poll()] == [(4, 0)]
        st = srv.stats()
    assert st["rejected"] == 4 and st["completed"] == 1


def test_cancel_pending_request(fb):
    """Two host requests that each need most of the arena: the second waits
    while the first (a 128 MiB copy each way) runs, and can be cancelled."""
    import torch
    n = 1 << 24
    a = torch.zeros(n, dtype=torch.complex64).pin_memory()
    b = torch.from_numpy(inputs.uniform_c64((4096,), 3)).pin_memory()
    bo = torch.empty_like(b).pin_memory()
    with fb.Server(slots=2, hbm_cap_bytes=n * 8 * 2 + (1 << 20)) as srv:
        srv.submit_ptr([n], a.data_ptr(), a.data_ptr(), 0, FWD, host_io=True)
        srv.submit_ptr([n], a.data_ptr(), a.data_ptr(), 1, FWD, host_io=True)  # waits for the arena
        srv.cancel(1)
        with pytest.raises(fb.FFTError):
            srv.cancel(1)  # no longer queued
        srv.submit_ptr([4096], b.data_ptr(), bo.data_ptr(), 2, FWD, host_io=True)
        srv.drain()
        done = {d[0]: d for d in srv.poll()}
        st = srv.stats()
    assert done[1][1] == -8 and done[1][2] == -1
    assert done[0][1] == 0 and done[2][1] == 0
    assert st["cancelled"] == 1 and st["completed"] == 2
    ref = oracle.fft(b.numpy().astype(np.complex128), [4096], FWD)
    assert oracle.rel_l2(bo.numpy().reshape(1, -1), ref.reshape(1, -1))[0] <= tol(4096)


def test_plan_cache_eviction_keeps_results(fb):
    """At most max_plans idle plans stay resident; evicted shapes are rebuilt."""
    import torch
    from paper_2004_09883_gb300 import serving
    shapes = [(64,), (128,), (3000,), (64,), (27, 27), (128,), (5 ** 5,), (64,)] * 3
    w = serving.Workload(shapes, 7300)
    with fb.Server(slots=3, hbm_cap_bytes=16 << 20, max_plans=2) as srv:
        for i, s in enumerate(shapes):  # one at a time, so earlier plans are idle
            srv.submit_ptr(s, w.x[i].data_ptr(), w.y[i].data_ptr(), i, FWD)
            srv.drain()
            assert [d[:2] for d in srv.poll()] == [(i, 0)]
            assert srv.stats()["plans"] <= 2
        st = srv.stats()
    assert st["plan_builds"] > 5
    for i, s in enumerate(shapes):
        assert torch.equal(w.y[i], _served_alone(fb, torch, s, FWD, w.x[i]))


def test_server_handle_errors(fb):
    import ctypes
    assert fb.lib.fb_fft_server_destroy(None) == 0
    assert fb.lib.fb_fft_server_drain(None) == -6
    assert fb.lib.fb_fft_server_clock(None) == -1.0
    h = ctypes.c_void_p()
    assert fb.lib.fb_fft_server_create(ctypes.byref(h), 0, 0, 1) == -1
    assert fb.lib.fb_fft_server_create(ctypes.byref(h), 65, 0, 1) == -1
    assert fb.lib.fb_fft_server_create(ctypes.byref(h), 1, -1, 1) == -1
    with fb.Server(slots=1, hbm_cap_bytes=0) as srv:
        assert srv.poll(wait=True) == []  # nothing queued: returns at once
        with pytest.raises(fb.FFTError) as e:  # four-step scratch cannot fit a zero budget
            import torch
            x = torch.zeros(1 << 16, dtype=torch.complex64, device="cuda")
            srv.submit_ptr([1 << 16], x.data_ptr(), x.data_ptr(), 0, FWD)
        assert e.value.status == -9


def test_requests_overlap_on_the_device(fb):
    """Continuous batching means requests run at the same time on the GPU:
    with 8 slots, more than one request is in flight at once, and the device
    intervals [t_dev_start, t_dev_end] of requests on different slots
    intersect (CUDA event timestamps on the slots' streams).  Every result
    still matches the oracle."""
    import torch
    n, batch, count = 1 << 22, 2, 12
    xs = [torch.from_numpy(inputs.uniform_c64((batch * n,), 7300 + i)).cuda() for i in range(count)]
    ys = [torch.empty_like(x) for x in xs]
    torch.cuda.synchronize()
    with fb.Server(slots=8, hbm_cap_bytes=2 << 30) as srv:
        srv.prepare([n], batch)
        for i in range(count):
            srv.submit_ptr([n], xs[i].data_ptr(), ys[i].data_ptr(), i, FWD, batch=batch)
        srv.drain()
        recs = srv.poll(device_times=True)
        st = srv.stats()
    assert sorted(r[0] for r in recs) == list(range(count)) and all(r[1] == 0 for r in recs)
    assert st["max_in_flight"] > 1
    iv = [(r[6], r[7], r[2]) for r in recs]
    assert all(0.0 <= a < b for a, b, _ in iv), iv
    overlapping = sum(1 for i in range(count) for j in range(i + 1, count)
                      if iv[i][2] != iv[j][2] and iv[i][0] < iv[j][1] and iv[j][0] < iv[i][1])
    assert overlapping > 0, iv
    for i in (0, count - 1):
        ref = oracle.fft(xs[i].cpu().numpy().astype(np.complex128), [n], FWD, False, 8)
        err = oracle.rel_l2(ys[i].cpu().numpy().reshape(batch, n), ref.reshape(batch, n))
        assert err.max() <= tol(n)


HOLD_TAG = 10 ** 6


def _hold_slot(srv, torch):
    """Occupy a slot for about a millisecond: a 2^24-point host-array request
    (128 MiB copied each way; its factors exceed 2048, so it runs alone
    through its plan).  Returns its buffers (keep them alive until drained)."""
    n = 1 << 24
    h = torch.zeros(n, dtype=torch.complex64).pin_memory()
    srv.submit_ptr((n,), h.data_ptr(), h.data_ptr(), HOLD_TAG, FWD, host_io=True)
    return h


def test_batches_form_under_load(fb):
    """One slot held busy while the whole mix is queued: the queue then runs
    as batches (fewer launches than requests), forward and scaled inverse
    requests in the same batch, with a per-request shape (5^9) in the FIFO;
    every result equals the request served alone and matches the oracle."""
    import torch
    from paper_2004_09883_gb300 import serving
    shapes, dirs = _mix(1400, copies=4)
    w = serving.Workload(shapes, 7400, dirs)
    scale = [d == INV and i % 2 == 0 for i, d in enumerate(dirs)]
    with fb.Server(slots=1, hbm_cap_bytes=1 << 30) as srv:
        for s in set(shapes):
            srv.prepare(list(s))
            srv.prepare(list(s), scale_inv_n=True)
        srv.prepare([1 << 24])
        hold = _hold_slot(srv, torch)
        l0 = fb.launch_count()
        for i, s in enumerate(shapes):
            srv.submit_ptr(s, w.x[i].data_ptr(), w.y[i].data_ptr(), i, dirs[i], scale_inv_n=scale[i])
        srv.drain()
        torch.cuda.synchronize()
        launches = fb.launch_count() - l0
        done = srv.poll()
        st = srv.stats()
    del hold
    done = [d for d in done if d[0] != HOLD_TAG]
    assert sorted(d[0] for d in done) == list(range(len(shapes))) and all(d[1] == 0 for d in done)
    assert st["largest_batch"] > 4 and st["batches"] < st["batched_requests"]
    assert launches < len(shapes)
    checked = set()
    for i, (s, d) in enumerate(zip(shapes, dirs)):
        if s == (5 ** 9,):
            continue
        y_alone = _served_alone(fb, torch, s, d, w.x[i], scale=scale[i])
        assert torch.equal(w.y[i], y_alone), f"request {i} {s}"
        if (s, d, scale[i]) not in checked:
            checked.add((s, d, scale[i]))
            ref = oracle.fft(w.x[i].cpu().numpy().astype(np.complex128).reshape(s), list(s), d, scale[i])
            err = oracle.rel_l2(w.y[i].cpu().numpy().reshape(1, -1), ref.reshape(1, -1))[0]
            assert err <= tol(int(np.prod(s))), f"{s} dir {d} scale {scale[i]}: rel L2 {err:.3e}"


def test_batched_requests_with_batch_dimension_and_in_place(fb):
    """Requests with batch > 1 (1-D single job, four-step, 2-D, 3-D) and in
    place (in == out) inside one batch, against the oracle."""
    import torch
    cases = [((4096,), 3), ((1000,), 5), ((6000,), 2), ((24, 40), 3), ((8, 12, 20), 2), ((1,), 4)]
    xs = [torch.from_numpy(inputs.uniform_c64((b * int(np.prod(s)),), 7500 + i)).cuda()
          for i, (s, b) in enumerate(cases)]
    x0 = [x.clone() for x in xs]
    with fb.Server(slots=1, hbm_cap_bytes=1 << 30) as srv:
        for s, b in cases:
            srv.prepare(list(s), b)
        srv.prepare([1 << 24])
        hold = _hold_slot(srv, torch)  # the others queue behind it
        for i, (s, b) in enumerate(cases):
            srv.submit_ptr(s, xs[i].data_ptr(), xs[i].data_ptr(), i, FWD, batch=b)
        srv.drain()
        done = srv.poll()
        st = srv.stats()
    del hold
    assert all(d[1] == 0 for d in done) and len(done) == len(cases) + 1
    assert st["largest_batch"] == len(cases)
    for i, (s, b) in enumerate(cases):
        n = int(np.prod(s))
        ref = oracle.fft(x0[i].cpu().numpy().astype(np.complex128), list(s), FWD)
        err = oracle.rel_l2(xs[i].cpu().numpy().reshape(b, n), ref.reshape(b, n))
        assert err.max() <= tol(max(2, n)), f"{s} x {b}: {err.max():.3e}"


def test_submit_many_queues_the_valid_and_reports_the_rest(fb):
    """submit_many: every request's status as submit would give it; the valid
    ones are queued (in order) and run, a rejected one is not."""
    import torch
    shapes = [(4096,), (7,), (24, 40), (1 << 20,), (96, 96)]
    xs = [torch.from_numpy(inputs.uniform_c64((int(np.prod(s)),), 7700 + i)).cuda() for i, s in enumerate(shapes)]
    ys = [torch.empty_like(x) for x in xs]
    with fb.Server(slots=2, hbm_cap_bytes=1 << 30) as srv:
        reqs = srv.requests([(s, xs[i].data_ptr(), ys[i].data_ptr(), i, FWD) for i, s in enumerate(shapes)])
        st = srv.submit_many(reqs)
        srv.drain()
        done = sorted(srv.poll())
        stats = srv.stats()
    assert st == [0, -2, 0, 0, 0]
    assert [d[:2] for d in done] == [(0, 0), (2, 0), (3, 0), (4, 0)]
    assert stats["rejected"] == 1 and stats["completed"] == 4
    for i, s in enumerate(shapes):
        if i == 1:
            continue
        ref = oracle.fft(xs[i].cpu().numpy().astype(np.complex128), list(s), FWD)
        err = oracle.rel_l2(ys[i].cpu().numpy().reshape(1, -1), ref.reshape(1, -1))[0]
        assert err <= tol(int(np.prod(s))), f"{s}: {err:.3e}"


def test_replay_together_equals_one_by_one(fb):
    """The replay that hands over every arrived request in one call and the
    one that submits them one by one give the same bits."""
    import torch
    from paper_2004_09883_gb300 import serving
    shapes, dirs = _mix(1500, copies=2)
    w = serving.Workload(shapes, 7800, dirs)
    with fb.Server(slots=4, hbm_cap_bytes=1 << 30) as srv:
        serving.run_served(srv, w, np.zeros(len(shapes)), together=True)
        y1 = [y.clone() for y in w.y]
        st = srv.stats()
        serving.run_served(srv, w, np.zeros(len(shapes)), together=False)
    assert st["largest_batch"] > 1
    for i in range(len(shapes)):
        assert torch.equal(y1[i], w.y[i]), f"request {i} {shapes[i]}"


def test_wait_returns_on_completion_or_deadline(fb):
    """fb_fft_server_wait: returns once a request has finished (it is then
    ready for poll), at once with nothing running, and at the deadline."""
    import time
    import torch
    x = torch.from_numpy(inputs.uniform_c64((1 << 20,), 7900)).cuda()
    y = torch.empty_like(x)
    with fb.Server(slots=2, hbm_cap_bytes=1 << 30) as srv:
        t0 = time.perf_counter()
        srv.wait(srv.clock() + 0.05)  # nothing running: at once
        assert time.perf_counter() - t0 < 0.04
        srv.submit_ptr((1 << 20,), x.data_ptr(), y.data_ptr(), 5, FWD)
        srv.wait(srv.clock() + 10.0)
        done = srv.poll()
        assert [d[:2] for d in done] == [(5, 0)]
        t0 = time.perf_counter()
        srv.wait(srv.clock() + 0.01)  # idle again
        assert time.perf_counter() - t0 < 0.04
    ref = oracle.fft(x.cpu().numpy().astype(np.complex128), [1 << 20], FWD)
    assert oracle.rel_l2(y.cpu().numpy().reshape(1, -1), ref.reshape(1, -1))[0] <= tol(1 << 20)
