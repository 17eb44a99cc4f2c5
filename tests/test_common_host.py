"""isqrt44 (eis_common.cuh), the kernels' floor(sqrt d) for d < 2^44 without
the FP64 unit, built for the host from the same source and checked against
Python's exact math.isqrt: squares and their neighbours up to the top of the
range, values either side of fp32 rounding boundaries, and random d."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def common_host(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("common") / "common_host")
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I", os.path.join(ROOT, "paper_2507_06579_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "common_host.cu"), "-o", exe],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    return exe


def test_isqrt44_is_exact(common_host):
    rng = np.random.default_rng(17)
    top = 2**44
    ds = list(range(0, 2000))
    ks = [int(k) for k in rng.integers(1, 2**22, size=3000)] + [2**22 - 1, 2**22 - 2, 2**21, 3037000]
    for k in ks:
        for e in (-2, -1, 0, 1, 2):
            v = k * k + e
            if 0 <= v < top:
                ds.append(v)
    ds += [int(x) for x in rng.integers(0, top, size=20000)]
    # just above and below multiples of 2^21 (where float(d) rounds)
    for m in rng.integers(1, 2**23, size=2000):
        for e in (-1, 0, 1):
            v = int(m) * 2**21 + e
            if 0 <= v < top:
                ds.append(v)
    ds.append(top - 1)
    r = subprocess.run([common_host], input="\n".join(map(str, ds)) + "\n", capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    got = [int(x) for x in r.stdout.split()]
    assert len(got) == len(ds)
    bad = [(d, g) for d, g in zip(ds, got) if g != math.isqrt(d)]
    assert not bad, bad[:5]
