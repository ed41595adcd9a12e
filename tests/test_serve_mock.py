"""Serving scheduler on the CPU-only mock device (no GPU): tickets, admission by
the memory budget in arrival order, the bounded host queue (BUSY), injected
allocation failure (NOMEM), a device that never completes (TIMEOUT at destroy)
and requests larger than the budget."""
import time

import pytest

from paper_2303_14827_gb300 import binding, scenes

MOCK = -1


def footprint(s):
    # output planes (24 B/px) + counters and hit list (256 + 16 B/px) + one device slot
    px = s["width"] * s["height"]
    return px * 24 + 256 + px * 16 + 2048


def wait_all(ctx, tickets, timeout=10.0):
    done_order, results = [], {}
    t0 = time.time()
    while len(results) < len(tickets):
        for t in tickets:
            if t in results:
                continue
            done, st = binding.dqj_poll(ctx, t)
            if done:
                results[t] = st
                done_order.append(t)
        assert time.time() - t0 < timeout
        time.sleep(0.001)
    return done_order, results


@pytest.fixture
def mock_env(monkeypatch):
    monkeypatch.setenv("DQJ_MOCK_DELAY_US", "2000")
    monkeypatch.delenv("DQJ_MOCK_FAIL", raising=False)
    return monkeypatch


def test_tickets_complete_and_are_consumed(mock_env):
    ctx = binding.dqj_create(MOCK)
    s = scenes.default_scene(width=32, height=32)
    tickets = [binding.dqj_submit(ctx, s, binding.make_outputs(pitch_px=32)) for _ in range(20)]
    assert len(set(tickets)) == 20
    _, res = wait_all(ctx, tickets)
    assert all(v == binding.DQJ_OK for v in res.values())
    with pytest.raises(binding.DqjError) as ei:
        binding.dqj_poll(ctx, tickets[0])
    assert ei.value.status == binding.DQJ_ERR_NOT_FOUND
    with pytest.raises(binding.DqjError):
        binding.dqj_poll(ctx, 987654)
    binding.dqj_destroy(ctx)


def test_budget_admits_in_arrival_order(mock_env):
    mock_env.setenv("DQJ_MOCK_DELAY_US", "20000")
    s = scenes.default_scene(width=64, height=64)
    ctx = binding.dqj_create(MOCK, mem_budget_bytes=int(footprint(s) * 1.5))  # one at a time
    t0 = time.time()
    tickets = [binding.dqj_submit(ctx, s, binding.make_outputs(pitch_px=64)) for _ in range(4)]
    order, res = wait_all(ctx, tickets)
    assert order == tickets
    assert time.time() - t0 >= 4 * 0.020
    assert all(v == binding.DQJ_OK for v in res.values())
    binding.dqj_destroy(ctx)


def test_host_queue_bound_gives_busy(mock_env):
    mock_env.setenv("DQJ_MOCK_DELAY_US", "300000")
    s = scenes.default_scene(width=64, height=64)
    ctx = binding.dqj_create(MOCK, mem_budget_bytes=int(footprint(s) * 1.5), max_pending=2)
    first = binding.dqj_submit(ctx, s, binding.make_outputs(pitch_px=64))
    time.sleep(0.05)  # admitted: the budget is now full
    queued = [binding.dqj_submit(ctx, s, binding.make_outputs(pitch_px=64)) for _ in range(2)]
    with pytest.raises(binding.DqjError) as ei:
        binding.dqj_submit(ctx, s, binding.make_outputs(pitch_px=64))
    assert ei.value.status == binding.DQJ_ERR_BUSY
    for t in [first] + queued:
        assert binding.dqj_poll(ctx, t) == (False, 0)
    _, res = wait_all(ctx, [first] + queued)
    assert all(v == binding.DQJ_OK for v in res.values())
    binding.dqj_destroy(ctx)


def test_request_larger_than_budget_is_refused(mock_env):
    s = scenes.default_scene(width=512, height=512)
    ctx = binding.dqj_create(MOCK, mem_budget_bytes=footprint(s) // 2)
    with pytest.raises(binding.DqjError) as ei:
        binding.dqj_submit(ctx, s, binding.make_outputs(pitch_px=512))
    assert ei.value.status == binding.DQJ_ERR_NOMEM
    binding.dqj_destroy(ctx)


def test_injected_allocation_failure(mock_env):
    mock_env.setenv("DQJ_MOCK_FAIL", "nomem")
    ctx = binding.dqj_create(MOCK)
    t = binding.dqj_submit(ctx, scenes.default_scene(width=16, height=16), binding.make_outputs(pitch_px=16))
    _, res = wait_all(ctx, [t])
    assert res[t] == binding.DQJ_ERR_NOMEM
    binding.dqj_destroy(ctx)


def test_host_exception_at_serve_start_becomes_nomem(mock_env):
    # no C++ exception crosses the C ABI: a host allocation that fails inside
    # dqj_submit comes back as DQJ_ERR_NOMEM with a message
    mock_env.setenv("DQJ_MOCK_FAIL", "throw_start")
    ctx = binding.dqj_create(MOCK)
    with pytest.raises(binding.DqjError) as ei:
        binding.dqj_submit(ctx, scenes.default_scene(width=16, height=16), binding.make_outputs(pitch_px=16))
    assert ei.value.status == binding.DQJ_ERR_NOMEM and "allocation" in binding.last_error()
    binding.dqj_destroy(ctx)


def test_host_exception_in_the_scheduler_thread(mock_env):
    # the scheduler thread survives a throwing admission: the admitted request
    # stays unfinished (its device work might still run), queued ones end with
    # DQJ_ERR_NOMEM, new submits are refused, and destroy reports TIMEOUT
    mock_env.setenv("DQJ_MOCK_FAIL", "throw_admit")
    mock_env.setenv("DQJ_DESTROY_TIMEOUT_MS", "200")
    s = scenes.default_scene(width=64, height=64)
    ctx = binding.dqj_create(MOCK, mem_budget_bytes=int(footprint(s) * 1.5))
    tickets = [binding.dqj_submit(ctx, s, binding.make_outputs(pitch_px=64))]
    for _ in range(2):  # queued behind the first, or refused once the thread has stopped
        try:
            tickets.append(binding.dqj_submit(ctx, s, binding.make_outputs(pitch_px=64)))
        except binding.DqjError as e:
            assert e.status == binding.DQJ_ERR_NOMEM
    time.sleep(0.05)
    states = [binding.dqj_poll(ctx, t) for t in tickets]
    assert states[0] == (False, 0)
    assert all(st == (True, binding.DQJ_ERR_NOMEM) for st in states[1:]), states
    with pytest.raises(binding.DqjError) as ei:
        binding.dqj_submit(ctx, s, binding.make_outputs(pitch_px=64))
    assert ei.value.status == binding.DQJ_ERR_NOMEM
    with pytest.raises(binding.DqjError) as ei:
        binding.dqj_destroy(ctx)
    assert ei.value.status == binding.DQJ_ERR_TIMEOUT


def test_never_completing_device_times_out_at_destroy(mock_env):
    mock_env.setenv("DQJ_MOCK_FAIL", "hang")
    mock_env.setenv("DQJ_DESTROY_TIMEOUT_MS", "200")
    ctx = binding.dqj_create(MOCK)
    s = scenes.default_scene(width=16, height=16)
    tickets = [binding.dqj_submit(ctx, s, binding.make_outputs(pitch_px=16)) for _ in range(3)]
    time.sleep(0.02)
    for t in tickets:
        assert binding.dqj_poll(ctx, t) == (False, 0)
    t0 = time.time()
    with pytest.raises(binding.DqjError) as ei:
        binding.dqj_destroy(ctx)
    assert ei.value.status == binding.DQJ_ERR_TIMEOUT
    assert time.time() - t0 < 2.0


def test_destroy_does_not_wait_for_queued_requests(mock_env):
    mock_env.setenv("DQJ_MOCK_DELAY_US", "100000")
    s = scenes.default_scene(width=64, height=64)
    ctx = binding.dqj_create(MOCK, mem_budget_bytes=int(footprint(s) * 1.5))
    for _ in range(6):
        binding.dqj_submit(ctx, s, binding.make_outputs(pitch_px=64))
    time.sleep(0.01)
    t0 = time.time()
    binding.dqj_destroy(ctx)  # one admitted request (0.1 s) is waited for; five queued ones are cancelled
    assert time.time() - t0 < 0.45


def test_mock_context_cannot_render(mock_env):
    ctx = binding.dqj_create(MOCK)
    with pytest.raises(binding.DqjError) as ei:
        binding.dqj_render(ctx, scenes.default_scene(width=8, height=8), binding.make_outputs(pitch_px=8), 0)
    assert ei.value.status == binding.DQJ_ERR_INVALID
    binding.dqj_destroy(ctx)


def test_serve_stats_count_admissions_and_completions(mock_env):
    ctx = binding.dqj_create(MOCK)
    assert binding.dqj_serve_stats(ctx) == {k: 0 for k in binding.SERVE_STAT_NAMES}
    s = scenes.default_scene(width=16, height=16)
    tickets = [binding.dqj_submit(ctx, s, binding.make_outputs(pitch_px=16)) for _ in range(7)]
    wait_all(ctx, tickets)
    st = binding.dqj_serve_stats(ctx)
    assert st["completed"] == 7 and st["plain"] == 7 and st["packed"] == 0  # the mock runs no persistent launch
    assert 1 <= st["batches"] <= 7 and st["launches"] == 0 and st["loops"] >= st["batches"]
    # seven requests submitted together, each running 1 ms on the mock, were resident together
    assert 2 <= st["max_active"] <= 7 and st["overlapped"] == 0, st
    binding.dqj_destroy(ctx)


def test_shortest_policy_orders_the_host_queue(mock_env):
    """DQJ_SERVE_SHORTEST also orders the host queue: with the budget taken by a
    running request, a 1920x1080 request and two 16x16 requests submitted just
    after it are admitted smallest estimated finish first (FIFO: arrival order)."""
    mock_env.setenv("DQJ_MOCK_DELAY_US", "20000")
    big = scenes.default_scene(width=1920, height=1080, march_steps=512)
    small = scenes.default_scene(width=16, height=16, march_steps=512)
    orders = {}
    for policy in (binding.DQJ_SERVE_FIFO, binding.DQJ_SERVE_SHORTEST):
        ctx = binding.dqj_create(MOCK, mem_budget_bytes=footprint(big) + 2 * footprint(small))
        binding.dqj_serve_policy(ctx, policy)
        blocker = binding.dqj_submit(ctx, big, binding.make_outputs(pitch_px=1920))
        time.sleep(0.005)  # the blocker is admitted and holds the budget
        a = binding.dqj_submit(ctx, big, binding.make_outputs(pitch_px=1920))
        b = binding.dqj_submit(ctx, small, binding.make_outputs(pitch_px=16))
        c = binding.dqj_submit(ctx, small, binding.make_outputs(pitch_px=16))
        order, res = wait_all(ctx, [blocker, a, b, c])
        assert all(v == binding.DQJ_OK for v in res.values())
        orders[policy] = [{blocker: "blocker", a: "big", b: "small1", c: "small2"}[t] for t in order]
        binding.dqj_destroy(ctx)
    assert orders[binding.DQJ_SERVE_FIFO] == ["blocker", "big", "small1", "small2"], orders
    assert orders[binding.DQJ_SERVE_SHORTEST][0] == "blocker", orders
    assert orders[binding.DQJ_SERVE_SHORTEST][-1] == "big", orders


@pytest.mark.parametrize("policy", [binding.DQJ_SERVE_FIFO, binding.DQJ_SERVE_SHORTEST])
def test_tight_polling_does_not_starve_the_scheduler(mock_env, policy):
    """A client that polls every in-flight ticket in a loop without sleeping
    (the benchmark's pattern) while requests keep arriving: dqj_poll does not
    take the scheduler's lock, so admissions and completions keep going."""
    import numpy as np
    mock_env.setenv("DQJ_MOCK_DELAY_US", "200")
    ctx = binding.dqj_create(MOCK)
    binding.dqj_serve_policy(ctx, policy)
    sizes = [(16, 16), (64, 64), (256, 256)]
    reqs = [scenes.default_scene(width=w, height=h) for w, h in sizes]
    rng = np.random.default_rng(3)
    n = 3000
    arrivals = np.cumsum(rng.exponential(50e-6, n))
    kinds = rng.integers(0, len(sizes), n)
    t0 = time.perf_counter()
    nxt, inflight, done_n = 0, {}, 0
    while nxt < n or inflight:
        now = time.perf_counter() - t0
        while nxt < n and arrivals[nxt] <= now:
            k = int(kinds[nxt])
            t = binding.dqj_submit(ctx, reqs[k], binding.make_outputs(pitch_px=sizes[k][0]))
            inflight[t] = k
            nxt += 1
        for t in list(inflight):
            done, st = binding.dqj_poll(ctx, t)
            if done:
                assert st == binding.DQJ_OK
                inflight.pop(t)
                done_n += 1
        assert time.perf_counter() - t0 < 20.0, (nxt, len(inflight), binding.dqj_serve_stats(ctx))
    assert done_n == n
    st = binding.dqj_serve_stats(ctx)
    assert st["completed"] == n and st["loops"] > 0
    binding.dqj_destroy(ctx)
