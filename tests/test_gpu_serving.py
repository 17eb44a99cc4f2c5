"""Serving: continuous batching of range-count and membership requests.

The bar is exact: every result must be the same when the request runs alone
and when it runs mixed with others (counts are integers), and equal to the
CPU oracle's, also when long walks inside a batch are handed to the
giant-step kernel.  Failure handling is exercised on the host only: a full
queue refuses submits (EIS_EBUSY), a wait can time out, a queued request can
be cancelled, a step-limit error in a batch reaches its requests as
EIS_ESTEPS, and a batch launch that fails (faked before anything is
enqueued) fails its requests with EIS_EDEVICE.
"""
import numpy as np
import pytest

import paper_2507_06579_gb300 as E
from paper_2507_06579_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    E.build()
    c = E.Context(0)
    yield c
    c.close()


def _stream(n, rate, seed, len_range=(1e2, 1e5), d_max=1e11):
    return W.serving_stream(n, rate, seed=seed, len_range=len_range, d_max=d_max,
                            a_range=(1e6, 1e11))


def _alone(ctx, kind, lo, hi):
    if kind == "count":
        return E.EIS_OK, ctx.count_range(lo, hi)
    try:
        return E.EIS_OK, int(ctx.is_eisenstein(lo))
    except E.EisError as e:
        return e.code, 0


def test_results_alone_equal_results_in_mix(ctx):
    reqs = _stream(400, 1e3, seed=31)
    alone = [_alone(ctx, k, lo, hi) for _, k, lo, hi in reqs]
    with E.Server(ctx, slots=3) as srv:
        ids = []
        for _, k, lo, hi in reqs:  # all at once: batches mix many requests
            ids.append(srv.submit_member(lo) if k == "member" else srv.submit_count(lo, hi))
        got = [srv.wait(i)[:2] for i in ids]
        st = srv.stats()
    for (rc, res), (rc_a, res_a) in zip(got, alone):
        assert rc == rc_a
        if rc == E.EIS_OK:
            assert res == res_a
    assert st["batches"] < len(reqs)          # requests really were batched together
    assert st["max_batch_parts"] > 1


def test_replay_poisson_matches_alone(ctx):
    reqs = _stream(600, 3e3, seed=32)
    t = [r[0] for r in reqs]
    kinds = [E.EIS_REQ_MEMBER if r[1] == "member" else E.EIS_REQ_COUNT for r in reqs]
    los = [r[2] for r in reqs]
    his = [r[3] for r in reqs]
    with E.Server(ctx) as srv:
        out = srv.replay(t, kinds, los, his)
    assert out["rc"] == E.EIS_OK
    for i, (_, k, lo, hi) in enumerate(reqs):
        rc_a, res_a = _alone(ctx, k, lo, hi)
        assert out["status"][i] == rc_a
        if rc_a == E.EIS_OK:
            assert int(out["results"][i]) == res_a
    lat = out["latency_us"]
    assert np.all(lat > 0) and np.percentile(lat, 50) < 1e6


def test_large_request_split_into_parts(ctx):
    lo, hi = 10**9, 10**9 + 8 * 200_000 + 3
    with E.Server(ctx, slots=2, slot_candidates=1 << 16) as srv:
        rid = srv.submit_count(lo, hi)
        rc, res, _ = srv.wait(rid)
        st = srv.stats()
    assert rc == E.EIS_OK and res == ctx.count_range(lo, hi)
    assert st["parts"] >= 4


def test_member_queries_not_in_D(ctx):
    with E.Server(ctx) as srv:
        a = srv.submit_member(45)        # 45 = 9 * 5: == 5 mod 8, not square-free
        b = srv.submit_member(10**9)     # not == 5 mod 8: answered without the GPU
        c = srv.submit_member(1901)      # Section 2.3 example, in E
        assert srv.wait(a)[0] == E.EIS_ENOTD
        assert srv.wait(b)[0] == E.EIS_ENOTD
        rc, res, _ = srv.wait(c)
        assert rc == E.EIS_OK and res == 1


def test_admission_refusal_timeout_and_cancel(ctx):
    heavy = (10**11, 10**11 + 8 * (1 << 22))      # one full slot of long walks
    with E.Server(ctx, slots=1, slot_candidates=1 << 22, max_pending=3) as srv:
        h = srv.submit_count(*heavy)
        # the dispatcher picks `h` up; the next submits queue behind it
        queued, busy = [], 0
        for i in range(20):
            try:
                queued.append(srv.submit_count(10**7 + 1000 * i, 10**7 + 1000 * i + 500))
            except E.EisError as e:
                assert e.code == E.EIS_EBUSY
                busy += 1
        assert busy > 0 and srv.stats()["rejected"] == busy
        # a zero-length wait on the heavy request times out and leaves it queued
        rc, _, _ = srv.wait(h, timeout_ms=0.0)
        assert rc in (E.EIS_ETIMEOUT, E.EIS_OK)
        if rc == E.EIS_ETIMEOUT:
            rc, res, _ = srv.wait(h)
            assert rc == E.EIS_OK and res == ctx.count_range(*heavy)
        # cancel one queued request
        srv.cancel(queued[-1])
        rc_c = srv.wait(queued[-1])[0]
        assert rc_c in (E.EIS_ECANCELED, E.EIS_OK)
        for q in queued[:-1]:
            rc, res, _ = srv.wait(q)
            assert rc == E.EIS_OK


def test_step_limit_error_reaches_requests():
    E.build()
    with E.Context(0) as c:
        c.set_option(E.EIS_OPT_STEP_LIMIT, 40)
        with E.Server(c) as srv:
            a = srv.submit_count(10**10, 10**10 + 80_000)
            rc, _, _ = srv.wait(a)
            assert rc == E.EIS_ESTEPS
        c.set_option(E.EIS_OPT_STEP_LIMIT, 1 << 26)
        with E.Server(c) as srv:  # the context still works
            b = srv.submit_count(10**6, 10**6 + 8000)
            rc, res, _ = srv.wait(b)
            assert rc == E.EIS_OK and res == c.count_range(10**6, 10**6 + 8000)


def test_server_memory_admission():
    E.build()
    with E.Context(0, mem_budget_bytes=64 << 20) as c:
        with pytest.raises(E.EisError) as ei:
            E.Server(c, slots=8, slot_candidates=1 << 24)
        assert ei.value.code == E.EIS_ENOMEM
        with E.Server(c, slots=2, slot_candidates=1 << 20) as srv:
            rid = srv.submit_count(5, 10**6 + 1)
            rc, res, _ = srv.wait(rid)
            assert rc == E.EIS_OK and res == c.count_range(5, 10**6 + 1)


def _oracle_answer(orc, kind, lo, hi):
    """(status, result) the server must return, from the CPU oracle."""
    if kind == "count":
        _, nE, _ = orc.count_range(lo, hi)
        return E.EIS_OK, nE
    rc, theta, _ = orc.walk_mod2(lo)
    if rc == orc.ORC_ENOTD:
        return E.EIS_ENOTD, 0
    assert rc == 0
    return E.EIS_OK, int(theta == 1)


@pytest.mark.parametrize("giant_after", [600, 0xffffffff], ids=["giant_handover", "walk_only"])
def test_server_results_match_oracle(ctx, orc, giant_after):
    """Every answer of a seeded mixed stream (range counts and membership
    queries) equals the oracle's.  With giant_after = 600 most range walks
    pass 600 baby steps inside a batch and are handed to the giant-step
    kernel (checked through the server's deferred counter); with 0xffffffff
    none is, and the same answers come from the baby walk alone."""
    reqs = W.serving_stream(200, 1e3, seed=41, len_range=(1e2, 2e4), d_max=1e10,
                            a_range=(1e6, 1e10))
    want = [_oracle_answer(orc, k, lo, hi) for _, k, lo, hi in reqs]
    with E.Server(ctx, slots=3, giant_after=giant_after, giant_max=1 << 16) as srv:
        ids = [srv.submit_member(lo) if k == "member" else srv.submit_count(lo, hi)
               for _, k, lo, hi in reqs]
        got = [srv.wait(i)[:2] for i in ids]
        st = srv.stats()
    for (rc, res), (rc_o, res_o), r in zip(got, want, reqs):
        assert rc == rc_o, r
        if rc == E.EIS_OK:
            assert res == res_o, r
    if giant_after == 600:
        assert st["deferred"] > 100
    else:
        assert st["deferred"] == 0


def test_failed_launch_fails_its_requests(ctx):
    """A batch whose launch fails (faked on the host by the fail_launches
    hook, before anything is enqueued) completes every request it held, and
    every request still queued, with EIS_EDEVICE: none returns EIS_OK with
    counts that were never written.  The context itself stays usable."""
    with E.Server(ctx, slots=1, fail_launches=1) as srv:
        ids = [srv.submit_count(10**6 + 1000 * i, 10**6 + 1000 * i + 800) for i in range(12)]
        ids.append(srv.submit_member(1901))
        rcs = [srv.wait(i)[0] for i in ids]
    assert all(rc == E.EIS_EDEVICE for rc in rcs), rcs
    assert ctx.count_range(10**6, 10**6 + 800) == ctx.count_range(10**6, 10**6 + 800)
    assert ctx.is_eisenstein(1901) is True
