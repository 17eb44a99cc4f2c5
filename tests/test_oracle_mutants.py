"""Planted mistakes: each mutant of the oracle must fail at least one pin.

A copy of oracle.c with one plausible mistake (a dropped term, a wrong index,
an off-by-one, a wrong constant) is compiled into a temporary library and the
quick pins below run against it in a child process.  The real oracle passes
the same pins (first case).  Everything runs on the CPU.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "none": None,
    "omega_sq_const": ("const int c = (int)(((d - 1) / 4) & 1);", "const int c = 0;"),
    "factor_old_P": ("int fx = (int)(((Pn - 1) / 2) & 1);", "int fx = (int)(((P - 1) / 2) & 1);"),
    "factor_drop_omega": ("int factor = fx | (1 << 1);", "int factor = fx | (fx << 1) | 1;"),
    "floor_off_by_one": ("int64_t q = (P + s) / Q;\n        int64_t Pn = q * Q - P;          /*",
                         "int64_t q = (P + s + 1) / Q;\n        int64_t Pn = q * Q - P;          /*"),
    "period_early_exit": ("} while (Q != 2); /* the first", "} while (Q != 2 && n < 3); /* the first"),
    "f4_drop_yy": ("int y = (x1 & y2) ^ (x2 & y1) ^ yy;", "int y = (x1 & y2) ^ (x2 & y1);"),
    "sieve_wrong_class": ("for (; x <= dhi; x += k2) {\n                    if (x % 8 == 5)",
                          "for (; x <= dhi; x += k2) {\n                    if (x % 8 == 1)"),
    "sieve_skip_k": ("for (uint64_t k = 2; k <= dhi / k; k++) {\n            if (J->primes)",
                     "for (uint64_t k = 2; k <= dhi / k; k += 2) {\n            if (J->primes)"),
    "prime_marks_k_itself": ("if (x < k * k) x = k * k;", "if (x < k) x = k;"),
    "prime_step_k2": ("for (; x <= dhi; x += k) {", "for (; x <= dhi; x += k * k) {"),
    "unitA_old_P": ("bn_lincomb(&Xn, &X, (uint64_t)Pn, &Y, d)", "bn_lincomb(&Xn, &X, (uint64_t)P, &Y, d)"),
    "unitA_flag_coord": ("int u_par = u.n ? (int)(u.w[0] & 1) : 0;", "int u_par = x_par;"),
    "forms_rho_sign": ("int64_t bp = r - (((r + b) % m) + m) % m;", "int64_t bp = r - (((r - b) % m) + m) % m;"),
}

QUICK_PINS = r'''
import math, sys, json
sys.path.insert(0, %(root)r)
sys.path.insert(0, %(tests)r)
import oracle as orc
from test_oracle import TEXTBOOK_UNITS, count_D_mobius
fails = []
def check(name, cond):
    if not cond:
        fails.append(name)
try:
    for d, (x0, y0, nrm) in TEXTBOOK_UNITS.items():
        u = orc.unit_exact(d)
        check("unit%%d" %% d, (u["x0"], u["y0"], u["norm"]) == (x0, y0, nrm))
        inE = ((x0 - y0) // 2) %% 2 == 1 and y0 %% 2 == 0
        rc, th, per = orc.walk_mod2(d)
        check("walk%%d" %% d, rc == 0 and (th == 1) == inE and per == u["period"])
    for d in (1901, 7053):
        rc, th, _ = orc.walk_mod2(d)
        check("paper%%d" %% d, rc == 0 and th == 1 and orc.unit_exact(d)["flag"])
    for d in range(5, 3000, 8):
        if orc.in_D(d):
            u = orc.unit_exact(d)
            rc, th, per = orc.walk_mod2(d)
            check("AB%%d" %% d, rc == 0 and th == u["theta"] and per == u["period"])
            h1, h4 = orc.narrow_classno(d), orc.narrow_classno(4 * d)
            check("iv%%d" %% d, h4 == (3 * h1 if th == 1 else h1))
    _, nD = orc.sqfree_range(0, 10**5)
    check("mobius", nD == count_D_mobius(0, 10**5))
    sieve = bytearray([1]) * 100000
    sieve[0] = sieve[1] = 0
    for i in range(2, 317):
        if sieve[i]:
            sieve[i * i::i] = bytearray(len(sieve[i * i::i]))
    nP = sum(1 for i in range(5, 100000, 8) if sieve[i])
    check("primes", orc.count_range_primes(0, 10**5)[0] == nP)
    nD, nE, _ = orc.count_range(0, 10**6 + 1)
    fit = 1e6 / (3 * math.pi**2) - 0.024 * 1e6 ** (5 / 6)
    check("fit", abs(nE - fit) / fit < 0.02)
except Exception as e:  # an oracle error is a caught mistake too
    fails.append("exception: %%r" %% (e,))
print(json.dumps(fails[:5]))
sys.exit(1 if fails else 0)
'''


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    src = open(SRC).read()
    mut = MUTANTS[name]
    if mut is not None:
        assert src.count(mut[0]) == 1, "mutation anchor not unique: %s" % name
        src = src.replace(mut[0], mut[1])
    cfile = tmp_path / "oracle.c"
    cfile.write_text(src)
    (tmp_path / "oracle.h").write_text(open(os.path.join(ROOT, "oracle", "oracle.h")).read())
    so = tmp_path / "liboracle_mut.so"
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                    str(cfile), "-o", str(so)], check=True)
    script = QUICK_PINS % {"root": ROOT, "tests": os.path.join(ROOT, "tests")}
    env = dict(os.environ, ORACLE_LIB=str(so))
    p = subprocess.run([sys.executable, "-c", script], env=env, capture_output=True,
                       text=True, timeout=600)
    if mut is None:
        assert p.returncode == 0, p.stdout + p.stderr
    else:
        assert p.returncode != 0, "mutant %s passed every pin" % name
