"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports exactly the entry points include/eis.h declares; argument errors are
rejected on the host before any device work."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2507_06579_gb300 as E

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "eis.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(eis_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libeis():
    E.build()
    return E.lib()


def test_header_declarations_are_exported(libeis):
    out = subprocess.run(["nm", "-D", "--defined-only", E.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = sorted(l.split()[-1] for l in out.splitlines() if re.search(r" T eis_", l))
    decl = declared_functions()
    assert decl, "no declarations parsed"
    missing = [f for f in decl if f not in exported]
    assert not missing, missing
    # every declared function is bound in the Python layer, with the same name
    bound = {name for name, _, _ in E.SIGNATURES}
    assert set(decl) <= bound, sorted(set(decl) - bound)
    for name in decl:
        assert getattr(libeis, name) is not None


def test_library_targets_sm103a():
    # the build passes exactly one -gencode: compute_103a -> sm_103a
    from paper_2507_06579_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    cuobj = subprocess.run(["cuobjdump", "--list-elf", E.LIB_PATH], capture_output=True, text=True)
    if cuobj.returncode == 0:
        assert "sm_103a" in cuobj.stdout


def test_strerror_names_every_code(libeis):
    for code in range(0, -10, -1):
        s = libeis.eis_strerror(code).decode()
        assert s and s != "unknown error", code
    assert libeis.eis_strerror(-1234).decode() == "unknown error"


def test_null_and_range_arguments_rejected_without_device(libeis):
    out = ctypes.c_uint64()
    assert libeis.eis_count_range(None, 0, 10, ctypes.byref(out)) == E.EIS_EINVAL
    assert libeis.eis_is_eisenstein(None, 5, None) == E.EIS_EINVAL
    assert libeis.eis_plan_launch(None, None) == E.EIS_EINVAL
    assert libeis.eis_plan_destroy(None) == E.EIS_OK
    assert libeis.eis_destroy(None) == E.EIS_OK
    assert libeis.eis_create(None, 0, 0) == E.EIS_EINVAL
    st = E.Stats()
    assert libeis.eis_get_stats(None, ctypes.byref(st)) == E.EIS_EINVAL


def test_product_path_has_no_cpu_fallback(monkeypatch, tmp_path):
    # Without the built library the binding raises instead of computing.
    monkeypatch.setattr(E, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(E, "_lib", None)
    with pytest.raises(RuntimeError):
        E.lib()


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2507_06579_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "oracle.h" not in txt, f
                assert "from oracle" not in txt, f


def test_header_is_plain_c_and_links(libeis, tmp_path):
    """A C11 program that includes only eis.h compiles without warnings and
    links against the library (it is not run: that needs a device)."""
    src = tmp_path / "use.c"
    src.write_text(
        '#include "eis.h"\n'
        "int main(void) {\n"
        "    eis_ctx *ctx;\n"
        "    uint64_t n = 0;\n"
        "    int r = 0;\n"
        "    if (eis_create(&ctx, 0, 0) != EIS_OK) return 1;\n"
        "    eis_count_range(ctx, 0, 1000001ull, &n);\n"
        "    eis_is_eisenstein(ctx, 1901, &r);\n"
        "    eis_destroy(ctx);\n"
        "    return (int)(n & 1) + r;\n"
        "}\n")
    exe = tmp_path / "use"
    libdir = os.path.dirname(E.LIB_PATH)
    r = subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-I",
                        os.path.join(ROOT, "include"), str(src), "-L", libdir, "-leis_gb300",
                        "-o", str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
