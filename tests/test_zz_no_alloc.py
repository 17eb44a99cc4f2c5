"""The no-allocation entry point eis_classify_range_noalloc.

It is for callers that may not allocate device memory (allocator hooks, which
would recurse into themselves, processes whose GPU memory belongs to another
framework's pool, loops that forbid allocation after start-up).  Its scratch
is a fixed array inside the library, shared by every call.  The test calls it
through the C-ABI twice in a row -- first the largest range it accepts, then
a smaller one, so stale scratch from the first call would show up in the
second -- and compares both with eis_classify_range bit for bit.  A third
test compares its output with the CPU oracle candidate by candidate.  It runs
alone or after the rest of the suite (this file is collected last).
"""
import ctypes

import numpy as np
import pytest

import paper_2507_06579_gb300 as E

pytestmark = pytest.mark.gpu


def _range_with(n, top):
    """[lo, hi) holding exactly n candidates, ending near `top`."""
    d0 = top - 8 * n
    d0 += (13 - d0 % 8) % 8
    return d0, d0 + 8 * (n - 1) + 1


def _call(torch, lo, hi, with_sqfree=True):
    n, _ = E.num_candidates(lo, hi)
    nw = max((n + 31) // 32, 1)
    # outputs start as garbage: the call must clear what it ORs into
    f = torch.full((nw,), -1, dtype=torch.int32, device="cuda")
    s = torch.full((nw,), -1, dtype=torch.int32, device="cuda") if with_sqfree else None
    cnt = ctypes.c_uint64(12345)
    rc = E.lib().eis_classify_range_noalloc(0, lo, hi, f.data_ptr(),
                                            s.data_ptr() if s is not None else None,
                                            ctypes.byref(cnt), None)
    torch.cuda.synchronize()
    fn = f.cpu().numpy().view(np.uint32)[: (n + 31) // 32]
    sn = s.cpu().numpy().view(np.uint32)[: (n + 31) // 32] if s is not None else None
    return rc, fn, sn, int(cnt.value)


def test_noalloc_matches_classify_range_twice():
    torch = pytest.importorskip("torch")
    E.build()
    cases = [_range_with(E.EIS_NOALLOC_MAX_CANDIDATES, 10**11),   # the largest accepted
             _range_with(70_001, 10**7)]                          # then a smaller one
    with E.Context(0) as ctx:
        refs = [ctx.classify_range(lo, hi) for lo, hi in cases]
        for (lo, hi), (f_ref, s_ref, c_ref) in zip(cases, refs):
            rc, f, s, c = _call(torch, lo, hi)
            assert rc == E.EIS_OK, E.lib().eis_strerror(rc)
            assert c == c_ref
            assert np.array_equal(f, f_ref)
            assert np.array_equal(s, s_ref)
        # without a square-free output the bitmap goes to the internal scratch
        lo, hi = cases[1]
        rc, f, _, c = _call(torch, lo, hi, with_sqfree=False)
        assert rc == E.EIS_OK and c == refs[1][2] and np.array_equal(f, refs[1][0])


def _unpack(words, n):
    return np.unpackbits(words.view(np.uint8), bitorder="little")[:n]


def test_noalloc_matches_oracle():
    """10^5 candidates near 10^7 (several sieve tiles and a ragged last word),
    each code (not in D / D minus E / E) equal to the oracle's."""
    torch = pytest.importorskip("torch")
    import oracle
    E.build()
    lo, hi = _range_with(100_001, 10**7)
    rc, f, s, c = _call(torch, lo, hi)
    assert rc == E.EIS_OK, E.lib().eis_strerror(rc)
    n, _ = E.num_candidates(lo, hi)
    codes = np.where(_unpack(f, n) == 1, 2, _unpack(s, n)).astype(np.uint8)
    ref = oracle.classify_range(lo, hi)["codes"]
    assert np.array_equal(codes, ref)
    assert c == int((ref == 2).sum())


def test_noalloc_allocates_nothing_after_setup():
    torch = pytest.importorskip("torch")
    E.build()
    lo, hi = _range_with(200_000, 10**10)
    rc, *_ = _call(torch, lo, hi)          # first call on the device: set-up
    assert rc == E.EIS_OK
    n, _ = E.num_candidates(lo, hi)
    nw = (n + 31) // 32
    f = torch.zeros(nw, dtype=torch.int32, device="cuda")
    s = torch.zeros(nw, dtype=torch.int32, device="cuda")
    cnt = ctypes.c_uint64()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        rc = E.lib().eis_classify_range_noalloc(0, lo, hi, f.data_ptr(), s.data_ptr(),
                                                ctypes.byref(cnt), None)
        assert rc == E.EIS_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_oversized_and_bad_arguments():
    torch = pytest.importorskip("torch")
    E.build()
    lo, hi = _range_with(E.EIS_NOALLOC_MAX_CANDIDATES + 1, 10**9)
    f = torch.full((4,), -1, dtype=torch.int32, device="cuda")
    cnt = ctypes.c_uint64(7)
    rc = E.lib().eis_classify_range_noalloc(0, lo, hi, f.data_ptr(), None, ctypes.byref(cnt), None)
    assert rc == E.EIS_ETOOLARGE
    assert "2^20" in E.lib().eis_strerror(rc).decode()
    torch.cuda.synchronize()
    assert cnt.value == 7 and bool((f == -1).all())   # nothing written
    assert E.lib().eis_classify_range_noalloc(0, 10, 5, f.data_ptr(), None, None, None) == E.EIS_EINVAL
    assert E.lib().eis_classify_range_noalloc(0, 5, 100, None, None, None, None) == E.EIS_EINVAL
    assert E.lib().eis_classify_range_noalloc(0, 5, E.EIS_D_LIMIT + 1, f.data_ptr(), None, None,
                                              None) == E.EIS_ERANGE
