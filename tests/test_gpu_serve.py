"""Served form on the GPU: requests of different sizes, constants, iteration
limits, slice frames and both FP32 modes (plain, and FP32 + FP64 recheck) run
together in the persistent launch (other precisions and modes as frames on the
serving stream).  Every result must be
identical to rendering the same request alone with dqj_render, whatever else was
in the mix.  Budget-limited admission and a long stream of small requests are
covered too."""
import time

import numpy as np
import pytest

from paper_2303_14827_gb300 import binding, scenes
from parity import to_numpy

pytestmark = pytest.mark.gpu


def run_served(ctx, reqs, timeout=60.0):
    import torch
    outs = [binding.alloc_outputs(s["width"], s["height"]) for s in reqs]
    torch.cuda.synchronize()  # the library writes outputs from its own streams
    tickets = [binding.dqj_submit(ctx, s, binding.outputs_of(o)) for s, o in zip(reqs, outs)]
    pending = set(range(len(reqs)))
    status = {}
    t0 = time.time()
    while pending:
        for i in list(pending):
            done, st = binding.dqj_poll(ctx, tickets[i])
            if done:
                status[i] = st
                pending.discard(i)
        assert time.time() - t0 < timeout, f"{len(pending)} requests not done"
        time.sleep(0.0005)
    return outs, status


def assert_same(a, b, s, what):
    x, y = to_numpy(a, s["width"], s["height"]), to_numpy(b, s["width"], s["height"])
    for k in ("iter", "depth", "normal", "rgba"):
        assert np.array_equal(x[k], y[k]), (what, k)
    assert binding.stats_dict(a["stats"]) == binding.stats_dict(b["stats"]), what


def mixed_requests():
    reqs = [scenes.default_scene()]
    reqs += scenes.batch_scenes(seed=1, n=5)
    for s in reqs[1:]:
        if s["width"] * s["height"] > 600_000:
            s.update(width=640, height=360)
    for name in ("highres", "test2_f", "test2_c"):
        reqs.append(scenes.default_scene(c=list(scenes.PAPER_C_VALUES[name]), width=300, height=200, max_iter=15))
    reqs.append(scenes.full_hd_scene(3))
    for k, (t, s) in enumerate(scenes.serving_stream(seed=2, n=6)):
        s.update(width=min(s["width"], 512), height=min(s["height"], 512))
        reqs.append(s)
    reqs.append(scenes.default_scene(width=1, height=1))
    reqs.append(scenes.default_scene(width=37, height=19))
    # the contract-accurate mode in the same launch: FP32 + FP64 recheck of an
    # axis frame, general slices and the 1080p workload frame
    for i in (0, 2, 4, 9):
        reqs.append(dict(reqs[i], precision=scenes.PRECISION_FP32_RECHECK))
    reqs.append(dict(scenes.default_scene(width=300, height=200, max_iter=16, march_steps=512, bisect_steps=10),
                     precision=scenes.PRECISION_FP32_RECHECK))
    return reqs


@pytest.mark.parametrize("policy", [binding.DQJ_SERVE_FIFO, binding.DQJ_SERVE_SHORTEST])
def test_served_equals_alone(policy):
    import torch
    reqs = mixed_requests()
    with binding.Renderer(0) as rdr:
        ctx = binding.dqj_create(0)
        try:
            binding.dqj_serve_policy(ctx, policy)
            outs, status = run_served(ctx, reqs)
            assert all(v == binding.DQJ_OK for v in status.values()), status
            # every request ran in the persistent launch, the launch served
            # several at once, and their device executions overlapped
            stats = binding.dqj_serve_stats(ctx)
            assert stats["packed"] == len(reqs) and stats["plain"] == 0, stats
            assert stats["launches"] < len(reqs), stats
            assert stats["max_active"] >= 2, stats
            assert stats["overlapped"] >= 1, stats
            for i, s in enumerate(reqs):
                alone = rdr.render(s)
                assert_same(outs[i], alone, s, f"request {i} precision {s['precision']}")
        finally:
            binding.dqj_destroy(ctx)
    torch.cuda.synchronize()


def test_shortest_policy_lets_small_requests_overtake():
    """DQJ_SERVE_SHORTEST: eight 128x128 requests submitted just after a
    1920x1080 request with 2048 march steps (several ms) all finish before it;
    the results still equal the requests rendered alone."""
    import torch
    big = dict(scenes.full_hd_scene(0), march_steps=2048)
    small = [scenes.default_scene(width=128, height=128, c=[-0.2, 0.6, 0.2, 0.2, 0.1, 0.0, 0.0, 0.01 * k])
             for k in range(8)]
    reqs = [big] + small
    ctx = binding.dqj_create(0)
    try:
        binding.dqj_serve_policy(ctx, binding.DQJ_SERVE_SHORTEST)
        run_served(ctx, [small[0]])  # scheduler thread and persistent launch running
        outs = [binding.alloc_outputs(s["width"], s["height"]) for s in reqs]
        torch.cuda.synchronize()
        tickets = [binding.dqj_submit(ctx, s, binding.outputs_of(o)) for s, o in zip(reqs, outs)]
        order, pending, t0 = [], set(range(len(reqs))), time.time()
        while pending:
            for i in sorted(pending):
                done, st = binding.dqj_poll(ctx, tickets[i])
                if done:
                    assert st == binding.DQJ_OK
                    order.append(i)
                    pending.discard(i)
            assert time.time() - t0 < 60.0
        assert order[-1] == 0, order
        with binding.Renderer(0) as rdr:
            for i, s in enumerate(reqs):
                assert_same(outs[i], rdr.render(s), s, f"request {i}")
    finally:
        binding.dqj_destroy(ctx)


def test_served_other_modes_equal_alone():
    reqs = [scenes.default_scene(width=96, height=80, precision=scenes.PRECISION_FP64),
            scenes.default_scene(width=96, height=80, precision=scenes.PRECISION_FP32_RECHECK),
            scenes.default_scene(width=96, height=80, square_mode=scenes.SQUARE_PAPER_COMPONENTWISE),
            scenes.default_scene(width=96, height=80, modulus_mode=scenes.MODULUS_DUALNUM),
            scenes.default_scene(width=128, height=128)]
    with binding.Renderer(0) as rdr:
        ctx = binding.dqj_create(0)
        try:
            outs, status = run_served(ctx, reqs)
            assert all(v == binding.DQJ_OK for v in status.values()), status
            for i, s in enumerate(reqs):
                assert_same(outs[i], rdr.render(s), s, f"mode request {i}")
        finally:
            binding.dqj_destroy(ctx)


def test_budget_limited_admission_and_many_small_requests():
    s0 = scenes.default_scene(width=128, height=96)
    px = 128 * 96
    budget = 3 * (px * 40 + 4096)  # about three requests resident at a time
    reqs = []
    rng = np.random.default_rng(5)
    for k in range(60):
        s = dict(s0)
        s["c"] = (np.array(scenes.C_DEFAULT) + rng.normal(0, 0.02, 8)).tolist()
        s["max_iter"] = int(rng.integers(8, 20))
        reqs.append(s)
    with binding.Renderer(0) as rdr:
        ctx = binding.dqj_create(0, mem_budget_bytes=budget)
        try:
            outs, status = run_served(ctx, reqs)
            assert all(v == binding.DQJ_OK for v in status.values())
            for i in (0, 17, 59):
                assert_same(outs[i], rdr.render(reqs[i]), reqs[i], f"small request {i}")
        finally:
            binding.dqj_destroy(ctx)


def test_destroy_with_requests_in_flight():
    import torch
    ctx = binding.dqj_create(0)
    outs = []
    for k in range(8):
        s = scenes.full_hd_scene(k % 5)
        o = binding.alloc_outputs(s["width"], s["height"])
        torch.cuda.synchronize()
        outs.append(o)
        binding.dqj_submit(ctx, s, binding.outputs_of(o))
    binding.dqj_destroy(ctx)  # waits (bounded) for admitted requests, cancels queued ones


def test_waves_with_idle_gaps_keep_full_speed():
    """Requests arriving in waves separated by about the kernel's idle limit: a
    launch must end as a whole, never leaving a few warps to serve the next wave."""
    import torch
    s = scenes.default_scene(width=256, height=256, max_iter=12)
    ctx = binding.dqj_create(0)
    try:
        outs = [binding.alloc_outputs(256, 256) for _ in range(8)]
        torch.cuda.synchronize()
        t0 = time.time()
        for wave in range(40):
            tickets = [binding.dqj_submit(ctx, s, binding.outputs_of(o)) for o in outs]
            for t in tickets:
                while True:
                    done, st = binding.dqj_poll(ctx, t)
                    if done:
                        assert st == binding.DQJ_OK
                        break
                    assert time.time() - t0 < 20.0, f"wave {wave} stalled"
                    time.sleep(0.0002)
            time.sleep(0.0015 + 0.0001 * (wave % 10))
        assert time.time() - t0 < 20.0
        stats = binding.dqj_serve_stats(ctx)
        assert stats["completed"] == 320 and stats["packed"] == 320
    finally:
        binding.dqj_destroy(ctx)
