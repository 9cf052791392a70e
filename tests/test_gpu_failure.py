"""Failure detection on the device without a GPU fault: a bounded wait that
runs out raises a flag the host reads, and the context keeps working."""
import time

import numpy as np
import pytest

from paper_2001_06444_gb300 import inputs, rtm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_context_survives():
    with rtm.Context(0) as ctx:
        t = time.perf_counter()
        assert ctx.selftest_wait(200) is True
        dt = time.perf_counter() - t
        assert 0.15 < dt < 5.0, dt
        # the context is still usable: a small modelling call succeeds
        nx, nz, nt = 60, 40, 50
        v = np.full((nz, nx), 2000.0, np.float32)
        keep = rtm._Keep()
        acq = rtm.make_acq(keep, [30], [5], np.arange(nx), np.full(nx, 5), inputs.ricker(20.0, 1e-3, nt))
        out = torch.zeros((nt, nx), dtype=torch.float32, device="cuda")
        ctx.model(rtm.make_grid(nx, nz, 10, 10.0, 10.0, 1e-3, nt), torch.from_numpy(v).cuda(), acq, 0, out)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all() and out.abs().max() > 0


def _small(seed):
    nx, nz, nt = 140, 70, 240
    s = inputs.scaled_survey(nx, nz, 2, nt, 18.0, seed)
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    seis = (inputs.normal(seed, 2 * nt * s.nrec).reshape(2, nt, s.nrec) * 1e-3).astype(np.float32)
    return dict(s=s, keep=keep, acq=acq, grid=rtm.make_grid(*s.grid_tuple()),
                v=torch.from_numpy(s.vel.astype(np.float32)).cuda(),
                seis=torch.from_numpy(seis).cuda(), opts=rtm.Opts(2, rtm.SNAP_F32, 1e-6, 1))


def test_raised_wait_flag_is_reported_by_its_own_call():
    """A migration whose wait-timeout flag is raised (injected on the host, as
    if a bounded device-side wait had given up) is reported by that call when
    it synchronises, else by the next call on the context, and by no other."""
    p = _small(3)
    s = p["s"]
    with rtm.Context(0) as ctx:
        ok = np.zeros((s.nz, s.nx), np.float32)
        ctx.migrate(p["grid"], p["v"], p["acq"], p["seis"], p["opts"], ok)  # host image: syncs
        ctx.inject_wait_timeout(1)
        host = np.zeros_like(ok)
        with pytest.raises(rtm.RTMError) as e:
            ctx.migrate(p["grid"], p["v"], p["acq"], p["seis"], p["opts"], host)
        assert e.value.code == rtm.RTM_ERR_TIMEOUT and "this call" in str(e.value)
        ctx.migrate(p["grid"], p["v"], p["acq"], p["seis"], p["opts"], host)  # reported once
        assert np.array_equal(host, ok)
        # device buffers: the call does not synchronise; the next call reports
        img = torch.zeros((s.nz, s.nx), dtype=torch.float32, device="cuda")
        ctx.inject_wait_timeout(1)
        ctx.migrate(p["grid"], p["v"], p["acq"], p["seis"], p["opts"], img)
        torch.cuda.synchronize()
        with pytest.raises(rtm.RTMError) as e:
            ctx.migrate(p["grid"], p["v"], p["acq"], p["seis"], p["opts"], img)
        assert e.value.code == rtm.RTM_ERR_TIMEOUT and "earlier call" in str(e.value)
        ctx.migrate(p["grid"], p["v"], p["acq"], p["seis"], p["opts"], img)
        torch.cuda.synchronize()
        assert np.array_equal(img.cpu().numpy(), ok)


def test_raised_wait_flag_fails_only_its_own_request():
    """Two requests in flight at once, one of them started with its flag
    raised: exactly that one ends FAILED with RTM_ERR_TIMEOUT and its own
    error text; the other ends DONE with the direct call's image."""
    a, b = _small(5), _small(6)
    with rtm.Context(0) as ctx:
        want = []
        for p in (a, b):
            out = torch.zeros((p["s"].nz, p["s"].nx), dtype=torch.float32, device="cuda")
            ctx.migrate(p["grid"], p["v"], p["acq"], p["seis"], p["opts"], out)
            want.append(out)
        torch.cuda.synchronize()
        imgs = [torch.zeros_like(w) for w in want]
        reqs = [rtm.Request(p["grid"], p["v"].data_ptr(), p["acq"], p["seis"].data_ptr(), p["opts"],
                            im.data_ptr()) for p, im in zip((a, b), imgs)]
        ctx.inject_wait_timeout(1)
        tickets = [ctx.submit(r) for r in reqs]
        states = {}
        t0 = time.time()
        while len(states) < 2 and time.time() - t0 < 120:
            for t in tickets:
                if t in states:
                    continue
                st, rc = _poll_keep_error(ctx, t)
                if st in (rtm.REQ_DONE, rtm.REQ_FAILED):
                    states[t] = (st, rc)
        assert len(states) == 2
        torch.cuda.synchronize()
        failed = [k for k, t in enumerate(tickets) if states[t][0] == rtm.REQ_FAILED]
        assert len(failed) == 1, states
        k = failed[0]
        assert "device-side wait gave up in this request" in states[tickets[k]][1]
        other = 1 - k
        assert states[tickets[other]][0] == rtm.REQ_DONE
        assert torch.equal(imgs[other], want[other])


def _poll_keep_error(ctx, ticket):
    """(state, error text of a FAILED request)."""
    st, rc = ctx.poll(ticket, 20)
    return st, (ctx.last_error() if st == rtm.REQ_FAILED else "")
