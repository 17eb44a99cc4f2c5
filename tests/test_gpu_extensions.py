"""Prime subsequence (Section 3.2) and the class of eps_d in F_4*, on the GPU,
against the oracle."""
import numpy as np
import pytest

import paper_2507_06579_gb300 as E

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    E.build()
    c = E.Context(0)
    yield c
    c.close()


def _bits(words, n):
    return np.unpackbits(np.asarray(words, dtype=np.uint32).view(np.uint8), bitorder="little")[:n]


WINDOWS = [(5, 400_001), (10**6, 10**6 + 8 * 70_001 + 3), (10**9, 10**9 + 120_000),
           (10**11 - 16_000, 10**11 + 1), (10**12 - 5_000, 10**12)]


@pytest.mark.parametrize("lo,hi", WINDOWS)
def test_prime_mode_matches_oracle(ctx, orc, lo, hi):
    ref = orc.classify_range_primes(lo, hi, thetas=True)
    n = len(ref["codes"])
    plan = ctx.plan_create([lo], [hi], E.EIS_MODE_PERSISTENT, E.EIS_PLAN_PRIMES | E.EIS_PLAN_CLASSES)
    plan.launch()
    f, s = plan.copy_bitmaps()
    nE, nP, cls = int(plan.counts()[0]), int(plan.counts_D()[0]), plan.class_counts()[0]
    plan.destroy()
    assert np.array_equal(_bits(s, n), (ref["codes"] > 0).astype(np.uint8))
    assert np.array_equal(_bits(f, n), (ref["codes"] == 2).astype(np.uint8))
    assert nP == int((ref["codes"] > 0).sum()) and nE == int((ref["codes"] == 2).sum())
    th = ref["thetas"][ref["codes"] > 0]
    assert [int(x) for x in cls] == [int((th == 1).sum()), int((th == 2).sum()), int((th == 3).sum())]


@pytest.mark.parametrize("lo,hi", WINDOWS[:4])
def test_class_counts_match_oracle(ctx, orc, lo, hi):
    ref = orc.classify_range(lo, hi, thetas=True)["thetas"]
    got = ctx.class_counts(lo, hi)
    assert got == [int((ref == 1).sum()), int((ref == 2).sum()), int((ref == 3).sum())]
    gp = ctx.class_counts(lo, hi, primes_only=True)
    refp = orc.classify_range_primes(lo, hi, thetas=True)["thetas"]
    assert gp == [int((refp == 1).sum()), int((refp == 2).sum()), int((refp == 3).sum())]
    # the E class is the Eisenstein count
    assert got[0] == ctx.count_range(lo, hi)


def test_c_program_through_the_abi(tmp_path):
    """A plain C program (no Python in the loop) counts pi_E(10^8) and asks
    for 1901 through include/eis.h."""
    import os
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    E.build()
    src = tmp_path / "prog.c"
    src.write_text(
        "#include <stdio.h>\n"
        '#include "eis.h"\n'
        "int main(void) {\n"
        "    eis_ctx *ctx;\n"
        "    int rc = eis_create(&ctx, 0, 0);\n"
        "    if (rc != EIS_OK) { printf(\"create %d\\n\", rc); return 1; }\n"
        "    uint64_t n = 0;\n"
        "    int r = -1;\n"
        "    rc = eis_count_range(ctx, 0, 100000001ull, &n);\n"
        "    if (rc == EIS_OK) rc = eis_is_eisenstein(ctx, 1901, &r);\n"
        "    printf(\"%d %llu %d\\n\", rc, (unsigned long long)n, r);\n"
        "    eis_destroy(ctx);\n"
        "    return rc == EIS_OK ? 0 : 2;\n"
        "}\n")
    exe = tmp_path / "prog"
    libdir = os.path.dirname(E.LIB_PATH)
    cc = subprocess.run(["gcc", "-std=c11", "-Wall", "-I", os.path.join(root, "include"), str(src),
                         "-L", libdir, "-leis_gb300", "-Wl,-rpath," + libdir, "-o", str(exe)],
                        capture_output=True, text=True, timeout=120)
    assert cc.returncode == 0, cc.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0, run.stdout + run.stderr
    assert run.stdout.split() == ["0", "3259668", "1"]
