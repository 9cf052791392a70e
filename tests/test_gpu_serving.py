"""The request loop (rtm_submit / rtm_poll): continuous batching under a
memory budget.  Each served result must equal the direct rtm_migrate result
bit for bit, alone or in a mix; failures stay with their own request."""
import time

import numpy as np
import pytest

from paper_2001_06444_gb300 import inputs, rtm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _request(nx, nz, nshot, nt, seed, f=15.0):
    s = inputs.scaled_survey(nx, nz, nshot, nt, f, seed)
    v = torch.from_numpy(s.vel.astype(np.float32)).cuda()
    rng = inputs.normal(seed, nshot * nt * s.nrec).reshape(nshot, nt, s.nrec) * 1e-3
    seis = torch.from_numpy(rng.astype(np.float32)).cuda()
    img = torch.zeros((nz, nx), dtype=torch.float32, device="cuda")
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    grid = rtm.make_grid(*s.grid_tuple())
    opts = rtm.Opts(4, rtm.SNAP_F16, 1e-6, 1)
    req = rtm.Request(grid, v.data_ptr(), acq, seis.data_ptr(), opts, img.data_ptr())
    return dict(req=req, keep=keep, v=v, seis=seis, img=img, grid=grid, acq=acq, opts=opts)


def _direct(ctx, r):
    out = torch.zeros_like(r["img"])
    ctx.migrate(r["grid"], r["v"], r["acq"], r["seis"], r["opts"], out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _wait(ctx, tickets, timeout_s=300):
    states = {}
    t0 = time.time()
    pending = set(tickets)
    while pending and time.time() - t0 < timeout_s:
        for t in list(pending):
            st, rc = ctx.poll(t, 50)
            if st in (rtm.REQ_DONE, rtm.REQ_FAILED):
                states[t] = st
                pending.discard(t)
    assert not pending, "requests did not finish"
    return states


def test_mixed_requests_match_direct_migration():
    ctx = rtm.Context(0)
    try:
        reqs = [_request(201, 101, 3, 400, 1), _request(330, 120, 5, 300, 2),
                _request(160, 64, 1, 500, 3), _request(201, 101, 2, 250, 4)]
        want = [_direct(ctx, r) for r in reqs]
        tickets = [ctx.submit(r["req"]) for r in reqs]
        states = _wait(ctx, tickets)
        torch.cuda.synchronize()
        for t, r, w in zip(tickets, reqs, want):
            assert states[t] == rtm.REQ_DONE
            assert np.array_equal(r["img"].cpu().numpy(), w)
        # the requests ran side by side (each on its own stream), not one
        # after another
        assert ctx.stats()["requests_peak_running"] >= 2
    finally:
        ctx.close()


def test_admission_runs_one_at_a_time_under_a_small_budget():
    probe = _request(201, 101, 2, 300, 5)
    call_b, item_b = rtm.plan_bytes(probe["grid"], probe["acq"], probe["opts"])
    # room for one 2-shot request with both shots in flight, not for a second
    # request's minimum (call + one item)
    ctx = rtm.Context(0, budget_bytes=call_b + 2 * item_b + item_b // 2)
    try:
        reqs = [probe, _request(201, 101, 2, 300, 6), _request(201, 101, 2, 300, 7)]
        want = [_direct(ctx, r) for r in reqs]
        for r in reqs:
            r["img"].zero_()
        torch.cuda.synchronize()
        tickets = [ctx.submit(r["req"]) for r in reqs]
        running_seen = 0
        t0 = time.time()
        done = set()
        while len(done) < len(tickets) and time.time() - t0 < 300:
            now_running = 0
            for t in tickets:
                if t in done:
                    continue
                st, _ = ctx.poll(t, 0)
                if st == rtm.REQ_RUNNING:
                    now_running += 1
                if st in (rtm.REQ_DONE, rtm.REQ_FAILED):
                    assert st == rtm.REQ_DONE
                    done.add(t)
            running_seen = max(running_seen, now_running)
            time.sleep(0.005)
        assert len(done) == len(tickets)
        assert running_seen <= 1
        assert ctx.stats()["requests_peak_running"] <= 1
        torch.cuda.synchronize()
        for r, w in zip(reqs, want):
            assert np.array_equal(r["img"].cpu().numpy(), w)
    finally:
        ctx.close()


def test_backfill_admits_a_small_request_past_a_waiting_head():
    """A long request holds most of the budget; the next one in the queue
    cannot start until it ends, but a small one behind it fits in what is
    left.  The small one is admitted past the waiting head and finishes while
    the long one still runs; every image equals the direct call's."""
    long_r = _request(201, 101, 4, 24000, 21)
    head = _request(601, 301, 2, 2000, 22)
    small = _request(161, 81, 1, 300, 23)
    cb = {}
    for name, r in (("long", long_r), ("head", head), ("small", small)):
        call_b, item_b = rtm.plan_bytes(r["grid"], r["acq"], r["opts"])
        cb[name] = (call_b, item_b)
    want_long = cb["long"][0] + 4 * cb["long"][1]
    need_head = cb["head"][0] + cb["head"][1]
    need_small = cb["small"][0] + cb["small"][1]
    assert need_head > need_small
    ctx = rtm.Context(0, budget_bytes=want_long + need_small + (need_head - need_small) // 2)
    try:
        reqs = [long_r, head, small]
        want = [_direct(ctx, r) for r in reqs]
        for r in reqs:
            r["img"].zero_()
        torch.cuda.synchronize()
        ctx.stats(reset=True)
        tickets = [ctx.submit(r["req"]) for r in reqs]
        st, _ = ctx.poll(tickets[2], 120000)
        assert st == rtm.REQ_DONE
        st_long, _ = ctx.poll(tickets[0], 0)
        assert st_long == rtm.REQ_RUNNING  # the small request overtook the head
        states = _wait(ctx, tickets[:2])
        assert all(v == rtm.REQ_DONE for v in states.values())
        assert ctx.stats()["requests_backfilled"] >= 1
        torch.cuda.synchronize()
        for r, w in zip(reqs, want):
            assert np.array_equal(r["img"].cpu().numpy(), w)
    finally:
        ctx.close()


def test_request_errors():
    ctx = rtm.Context(0, budget_bytes=64 << 20)
    try:
        big = _request(1701, 351, 2, 5000, 8)
        with pytest.raises(rtm.RTMError) as e:
            ctx.submit(big["req"])
        assert e.value.code == rtm.RTM_ERR_NOMEM
        r = _request(120, 60, 1, 200, 9)
        host = np.zeros((60, 120), np.float32)
        bad = rtm.Request(r["grid"], r["v"].data_ptr(), r["acq"], r["seis"].data_ptr(), r["opts"],
                          host.ctypes.data)
        with pytest.raises(rtm.RTMError) as e:
            ctx.submit(bad)
        assert e.value.code == rtm.RTM_ERR_ARG
        with pytest.raises(rtm.RTMError) as e:
            ctx.poll(123456789, 0)
        assert e.value.code == rtm.RTM_ERR_STATE
        # a request that fails on the device side (CFL) reports FAILED; a
        # request submitted next to it still completes
        fast = _request(120, 60, 1, 200, 10)
        fast["v"].fill_(1.05 * rtm.cfl_limit() * 10.0 / 1e-3)
        ok = _request(120, 60, 1, 200, 11)
        t_bad = ctx.submit(fast["req"])
        t_ok = ctx.submit(ok["req"])
        states = _wait(ctx, [t_bad, t_ok])
        assert states[t_bad] == rtm.REQ_FAILED
        assert states[t_ok] == rtm.REQ_DONE
        assert "CFL" in ctx.last_error() or states[t_bad] == rtm.REQ_FAILED
    finally:
        ctx.close()
