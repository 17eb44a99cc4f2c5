"""The lane-per-d infrastructure search of the batch path (eis_bsgs.cuh), run
on the host against the oracle.

The host model (bsgs_host.cu) walks baby steps in plain integers and uses
the library's own table, index, marking threshold and giant steps.  Its
answers must equal the oracle's log eps_d for every d, with the lean product,
NUCOMP and the general textbook composition,
with every giant cycle ending one step after its first marked state (the
kernel's order), or walking on for a while (as lanes of a warp that wait
for each other would).  With
`verify` the model walks the whole period first and checks that every hit is
at position l - j (mirror key) or l + j (direct key) of the first period,
the claim the search's window argument makes (also with the wide stride
reduce(a_jl a_j'), which nearly fills the window)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bsgs_host(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("bsgs") / "bsgs_host")
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I", os.path.join(ROOT, "include"),
                        "-I", os.path.join(ROOT, "paper_2507_06579_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "bsgs_host.cu"), "-o", exe],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    return exe


def _run(exe, rows, wide=1):
    """rows: (d, N, tau, compose, extra, verify) -> list of output tuples;
    wide = 1: the wide stride reduce(a_jl a_j'), 0: a_jl."""
    inp = "".join("%d %d %.9g %d %d %d %d\n" % (r + (wide,)) for r in rows)
    r = subprocess.run([exe], input=inp, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr
    out = [tuple(int(x) for x in ln.split()) for ln in r.stdout.strip().split("\n")]
    assert len(out) == len(rows)
    return out


def _ds(orc, rng, lo, hi, k):
    out = []
    while len(out) < k:
        d = int(rng.integers(lo // 8, hi // 8)) * 8 + 5
        if orc.in_D(d):
            out.append(d)
    return out


def _check(orc, rows, out, want_verified):
    searched = 0
    for (d, N, tau, comp, extra, verify), (status, g, baby, cycles, walked, k, jl, hit) in zip(rows, out):
        rc, theta, _ = orc.walk_mod2(d)
        assert rc == 0
        if status == 2:      # too few marked states: the search declines the d
            assert jl < 256
            continue
        assert status in (0, 1), (d, N, tau, comp, status)
        assert g == theta - 1, (d, N, tau, comp, extra, status, g, theta)
        if status == 1:
            searched += 1
            assert jl >= 256 and k >= 2
            if want_verified:
                assert hit == 1, (d, N, tau, comp, extra, hit)
    return searched


@pytest.mark.parametrize("wide", [1, 0], ids=["wide_stride", "stride_a_jl"])
@pytest.mark.parametrize("compose", [0, 1, 2, 3], ids=["lean", "lean_nucomp", "textbook", "nucomp"])
def test_hits_lie_in_the_first_period_window(bsgs_host, orc, compose, wide):
    """d up to 1e10 (whole periods walkable): every hit at l - j or l + j,
    with the stride a_jl and with the wide stride reduce(a_jl a_j')."""
    rng = np.random.default_rng(71 + compose)
    rows = []
    for lo, hi in ((10**8, 10**9), (10**9, 10**10)):
        for d in _ds(orc, rng, lo, hi, 24):
            for N, m in ((300, 8), (640, 16), (1200, 32)):
                for extra in (-1, 0, 50):
                    rows.append((d, N, 1.39 / m, compose, extra, 1))
    out = _run(bsgs_host, rows, wide)
    assert _check(orc, rows, out, True) > len(rows) // 2


@pytest.mark.parametrize("compose", [0, 1, 2, 3], ids=["lean", "lean_nucomp", "textbook", "nucomp"])
def test_search_matches_oracle_near_1e11_1e12_and_2p44(bsgs_host, orc, compose):
    rng = np.random.default_rng(83 + compose)
    rows = []
    top = 2**44
    for lo, hi, n in ((10**11 - 10**9, 10**11, 24), (10**12 - 10**9, 10**12, 12),
                      (top - 10**9, top, 6), (4389000000000, 4391000000000, 6)):
        for d in _ds(orc, rng, lo, hi, n):
            for N, m in ((1024, 16), (2048, 16)):
                rows.append((d, N, 1.39 / m, compose, (-1, 0, 64)[d % 3], 0))
    out = _run(bsgs_host, rows)
    assert _check(orc, rows, out, False) > len(rows) // 2


def test_a_full_table_ends_the_baby_walk_early(bsgs_host, orc):
    """Dense marks (1 state in 3) fill the 128-entry table after ~380 steps:
    the baby walk stops there and the search still finds every unit."""
    rng = np.random.default_rng(97)
    rows = [(d, 4096, 1.39 / 3, c, 0, 1) for d in _ds(orc, rng, 10**9, 10**10, 20) for c in (0, 1, 2)]
    out = _run(bsgs_host, rows)
    assert _check(orc, rows, out, True) > 0
    for (status, g, baby, *_rest), (_, _, _, _, _, _) in zip(out, rows):
        if status == 1:
            assert baby < 4096                      # stopped at the full table
    assert any(o[5] == 128 for o in out)


def test_sparse_marks_fall_back(bsgs_host, orc):
    """With very sparse marks (1 in 4096) the last marked state is usually
    too close to the start: the search declines rather than risk a gap."""
    rng = np.random.default_rng(101)
    rows = [(d, 300, 1.39 / 4096, 0, 0, 0) for d in _ds(orc, rng, 10**10, 10**11, 20)]
    out = _run(bsgs_host, rows)
    _check(orc, rows, out, False)
    assert sum(o[0] == 2 for o in out) > 0
