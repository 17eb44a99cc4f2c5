"""The single-query command line (paper_2507_06579_gb300.query)."""
import contextlib
import io
import json
import subprocess
import sys

import pytest


def test_help_runs_without_a_device():
    r = subprocess.run([sys.executable, "-m", "paper_2507_06579_gb300.query", "--help"],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "--near" in r.stdout


@pytest.mark.gpu
@pytest.mark.parametrize("plain", [False, True])
def test_answers_match_oracle(orc, plain):
    from paper_2507_06579_gb300 import query
    ds = [37, 1901, 7053, 5, 45, 13, 10**12 - 3, 10**12 + 5]
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert query.main([str(d) for d in ds] + (["--plain"] if plain else [])) == 0
    rows = [json.loads(x) for x in buf.getvalue().splitlines()]
    assert [r["d"] for r in rows] == ds
    for r in rows:
        d = r["d"]
        if d % 8 != 5 or not orc.in_D(d):
            assert r["in_D"] is False
            continue
        rc, theta, _ = orc.walk_mod2(d)
        assert rc == 0
        assert r["in_D"] is True and r["in_E"] == (theta == 1), d
