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
    binding.dqj_destroy(ctx)
