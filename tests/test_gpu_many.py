"""Batched uneven lengths (fb_fft_plan_many) against the FP64 oracle: every
transform of a packed batch, graph replay vs direct launches, repeats,
in place, inverse with 1/N, host arrays."""
import math

import numpy as np
import pytest

import oracle
from paper_2004_09883_gb300 import inputs

pytestmark = pytest.mark.gpu


def tol(n: int) -> float:
    return 2e-6 * math.log2(n) if n > 1 else 1e-7


def _batch(lengths, seed):
    return [inputs.uniform_c64((int(n),), seed + i) for i, n in enumerate(lengths)]


def _check(plan, xs, ys, direction, scale=False):
    for x, y, n in zip(xs, ys, plan.lengths):
        ref = oracle.fft(x.astype(np.complex128), [int(n)], direction, scale)
        err = oracle.rel_l2(y.reshape(1, -1), ref.reshape(1, -1))[0]
        assert err <= tol(int(n)), f"n={n}: rel L2 {err:.3e}"


LENGTHS = ([64, 4096, 100, 75, 4096, 6000, 64, 1 << 16, 81, 2, 3125, 8192, 65536, 4096, 1000, 45000, 4, 96]
           + list(inputs.uneven_lengths(40, 64, 65536, inputs.seed_for(inputs.WORKLOAD_UNEVEN_4096))))


@pytest.mark.parametrize("graph", [True, False])
def test_many_matches_oracle(fb, graph):
    import torch
    xs = _batch(LENGTHS, 900)
    with fb.PlanMany(LENGTHS) as p:
        p.set_graph(graph)
        d = torch.from_numpy(p.pack(xs)).cuda()
        out = p.exec(d, None, -1)
        out2 = p.exec(d, None, -1)  # second exec replays the cached graph
        p.check()
        ys = p.unpack(out.cpu().numpy())
        # the packed layout pads odd lengths to even: compare the transforms, not the padding
        for a, b in zip(p.unpack(out.cpu().numpy()), p.unpack(out2.cpu().numpy())):
            assert np.array_equal(a, b)
    _check(p, xs, ys, -1)


def test_many_graph_equals_direct_and_inverse_scaled(fb):
    import torch
    xs = _batch(LENGTHS, 901)
    with fb.PlanMany(LENGTHS, scale_inv_n=True) as p:
        d = torch.from_numpy(p.pack(xs)).cuda()
        p.set_graph(True)
        g = p.exec(d, None, 1)
        p.set_graph(False)
        direct = p.exec(d, None, 1)
        p.check()
        for a, b in zip(p.unpack(g.cpu().numpy()), p.unpack(direct.cpu().numpy())):
            assert np.array_equal(a, b)
        ys = p.unpack(g.cpu().numpy())
    _check(p, xs, ys, 1, scale=True)


def test_many_in_place_and_host_arrays(fb):
    import torch
    lens = [4096] * 7 + [128] * 33 + [65536, 1 << 20, 3 * 5 ** 6]
    xs = _batch(lens, 902)
    with fb.PlanMany(lens) as p:
        packed = p.pack(xs)
        d = torch.from_numpy(packed).cuda()
        p.exec(d, d, -1)
        p.check()
        dev = p.unpack(d.cpu().numpy())
        host = p.unpack(p.exec_host(packed, None, -1))
    _check(p, xs, dev, -1)
    for a, b in zip(dev, host):
        assert np.array_equal(a, b)


def test_many_single_transform_and_empty(fb):
    import torch
    with fb.PlanMany([]) as p:
        assert p.total == 0
    with fb.PlanMany([12]) as p:
        x = inputs.uniform_c64((12,), 3)
        y = p.exec(torch.from_numpy(p.pack([x])).cuda(), None, -1)
        _check(p, [x], p.unpack(y.cpu().numpy()), -1)


@pytest.mark.parametrize("opts", [dict(streams=1, use_graph=0, chunk_bytes=8 << 20, odd_radices_first=1, max_lines=4,
                                       per_length=1),
                                  dict(streams=16, use_graph=1, chunk_bytes=1 << 20, odd_radices_first=0, max_lines=16)])
def test_many_knobs_keep_results(fb, opts):
    import torch
    xs = _batch(LENGTHS, 903)
    with fb.PlanMany(LENGTHS, opts=opts) as p:
        out = p.exec(torch.from_numpy(p.pack(xs)).cuda(), None, -1)
        p.check()
        ys = p.unpack(out.cpu().numpy())
    _check(p, xs, ys, -1)


def test_autotuner_returns_a_working_setting(fb):
    import torch
    lens = LENGTHS[:30]
    xs = _batch(lens, 904)
    offs, total = fb.many_layout(lens)
    buf = np.zeros(total, np.complex64)
    for o, x in zip(offs, xs):
        buf[o:o + len(x)] = x
    d = torch.from_numpy(buf).cuda()
    out = torch.empty_like(d)
    best, ms = fb.autotune_many(lens, d, out, -1, reps=2)
    assert ms > 0 and 1 <= best.streams <= 32 and best.chunk_bytes > 0
    with fb.PlanMany(lens, opts=best) as p:
        y = p.exec(d, None, -1)
        p.check()
        _check(p, xs, p.unpack(y.cpu().numpy()), -1)


@pytest.mark.parametrize("direction,scale", [(-1, False), (1, True)])
def test_merged_launches_equal_per_length_launches(fb, direction, scale):
    """Engine 1: merged mixed-kernel launches and one launch per length agree,
    with far fewer launches."""
    import torch
    lens = list(inputs.uneven_lengths(300, 64, 65536, inputs.seed_for(inputs.WORKLOAD_UNEVEN_4096, 7)))
    lens += [75, 6000, 45000, 3 * 5 ** 6, 2, 3, 3000, 2187, 3125, 4050, 64, 128, 512, 2048, 4096, 8192, 65536]
    xs = _batch(lens, 950)
    with fb.PlanMany(lens, scale_inv_n=scale, opts={"engine": 1}) as pm, \
            fb.PlanMany(lens, scale_inv_n=scale, opts={"per_length": 1}) as pl:
        d = torch.from_numpy(pm.pack(xs)).cuda()
        l0 = fb.launch_count()
        ym = pm.exec(d, None, direction)
        torch.cuda.synchronize()
        l1 = fb.launch_count()
        yl = pl.exec(d, None, direction)
        torch.cuda.synchronize()
        l2 = fb.launch_count()
        pm.check()
        pl.check()
        assert (l1 - l0) < (l2 - l1)
        ys = pm.unpack(ym.cpu().numpy())
        yls = pl.unpack(yl.cpu().numpy())
    # same kernel, same bits for single-pass lengths with a factor 3 or 5 (both
    # plans run them in the mixed kernel); the merged plan runs lengths
    # 2049..4096 with such a factor as two passes, which the oracle check covers
    for n, a, b in zip(lens, ys, yls):
        if n & (n - 1) and n <= 2048:
            assert np.array_equal(a, b), n
    _check(pm, xs, ys, direction, scale)
    _check(pl, xs, yls, direction, scale)


ENGINE0_LENGTHS = ([1, 2, 3, 4, 5, 8, 9, 16, 27, 64, 100, 125, 243, 1000, 1024, 2000, 2048, 2187, 3000, 4096,
                    4050, 6000, 8192, 45000, 59049, 65536, 1 << 20]
                   + list(inputs.uneven_lengths(200, 64, 65536, inputs.seed_for(inputs.WORKLOAD_UNEVEN_4096, 9))))


@pytest.mark.parametrize("direction,scale", [(-1, False), (1, True)])
def test_one_kernel_engine_matches_oracle_in_one_launch(fb, direction, scale):
    """Engine 0 (the default): every pass of the batch -- single passes,
    four-step columns and the rows that wait for them -- in one launch per
    exec (a replayed graph); lengths 1 to 2^20, one-radix schedules, odd
    lengths, every result against the oracle, in place and out of place, and
    repeated and graph-free execs give the same bits."""
    import torch
    xs = _batch(ENGINE0_LENGTHS, 960)
    with fb.PlanMany(ENGINE0_LENGTHS, scale_inv_n=scale) as p:
        assert p.info()["passes"] == 1
        d = torch.from_numpy(p.pack(xs)).cuda()
        l0 = fb.launch_count()
        y = p.exec(d, None, direction)
        torch.cuda.synchronize()
        assert fb.launch_count() - l0 == 1
        y2 = p.exec(d, None, direction)
        z = d.clone()
        p.exec(z, z, direction)
        p.set_graph(False)
        y3 = p.exec(d, None, direction)
        p.check()
        ys, ys2, ys3, zs = (p.unpack(t.cpu().numpy()) for t in (y, y2, y3, z))
    for a, b, c, e in zip(ys, ys2, zs, ys3):
        assert np.array_equal(a, b) and np.array_equal(a, c) and np.array_equal(a, e)
    _check(p, xs, ys, direction, scale)


def test_one_launch_and_two_launch_forms_give_identical_bits(fb):
    """Engine 2 runs the same jobs as two launches (all single passes and
    four-step columns, then all rows): the same bits as the one launch."""
    import torch
    xs = _batch(ENGINE0_LENGTHS, 960)
    with fb.PlanMany(ENGINE0_LENGTHS) as p1, fb.PlanMany(ENGINE0_LENGTHS, opts={"engine": 2}) as p2:
        assert p1.info()["passes"] == 1 and p2.info()["passes"] == 2
        d = torch.from_numpy(p1.pack(xs)).cuda()
        l0 = fb.launch_count()
        y2 = p2.exec(d, None, -1)
        torch.cuda.synchronize()
        assert fb.launch_count() - l0 == 2
        y1 = p1.exec(d, None, -1)
        p1.check()
        p2.check()
        # transforms only: the pad value after an odd length is never written
        for a, b in zip(p1.unpack(y1.cpu().numpy()), p2.unpack(y2.cpu().numpy())):
            assert np.array_equal(a, b)


def test_one_launch_beside_other_work_on_the_gpu(fb):
    """The one-launch exec while another stream keeps part of the GPU busy (so
    not every CTA of it is resident at once): a row tile only ever waits for
    column tiles that running CTAs hold, so it finishes, with the same bits."""
    import torch
    lens = list(inputs.uneven_lengths(300, 64, 65536, inputs.seed_for(inputs.WORKLOAD_UNEVEN_4096, 13)))
    xs = _batch(lens, 990)
    with fb.PlanMany(lens) as p:
        d = torch.from_numpy(p.pack(xs)).cuda()
        want = p.unpack(p.exec(d, None, -1).cpu().numpy())
        side = torch.cuda.Stream()
        a = torch.randn(4096, 4096, device="cuda")
        for it in range(6):
            with torch.cuda.stream(side):
                for _ in range(8):
                    a = torch.tanh(a @ a * 1e-3)
            got = p.exec(d, None, -1)
            torch.cuda.synchronize()
            p.check()
            # transforms only: the pad value after an odd length is never written
            for n, g, w in zip(lens, p.unpack(got.cpu().numpy()), want):
                assert np.array_equal(g, w), f"exec {it}, n={n}"
    _check(p, xs, want, -1)


def test_one_launch_reports_a_dependency_wait_that_runs_out(fb):
    """The test hook raises every four-step row's dependency target out of
    reach: the waits give up after about a second (the first one to run out
    ends the others), the plan reports FB_FFT_ERR_TIMEOUT, and the next exec
    without the hook is correct again (the counters were zeroed)."""
    import torch
    lens = [8192, 64, 45000, 100, 65536]
    xs = _batch(lens, 995)
    with fb.PlanMany(lens) as p:
        d = torch.from_numpy(p.pack(xs)).cuda()
        p.debug_inject_timeout(True)
        p.exec(d, None, -1)
        with pytest.raises(fb.FFTError) as e:
            p.check()
        assert e.value.status == -5
        p.debug_inject_timeout(False)
        y = p.exec(d, None, -1)
        p.check()
        ys = p.unpack(y.cpu().numpy())
    _check(p, xs, ys, -1)


def test_both_engines_agree_with_the_oracle(fb):
    import torch
    lens = list(inputs.uneven_lengths(120, 64, 65536, inputs.seed_for(inputs.WORKLOAD_UNEVEN_4096, 11)))
    xs = _batch(lens, 970)
    with fb.PlanMany(lens) as p0, fb.PlanMany(lens, opts={"engine": 1}) as p1:
        d = torch.from_numpy(p0.pack(xs)).cuda()
        y0 = p0.unpack(p0.exec(d, None, -1).cpu().numpy())
        y1 = p1.unpack(p1.exec(d, None, -1).cpu().numpy())
        p0.check()
        p1.check()
    _check(p0, xs, y0, -1)
    _check(p1, xs, y1, -1)
