"""The C ABI library builds for sm_103a, loads, and exports every entry point of include/tdvp.h."""
import os
import re

import pytest

import paper_1907_12044_b300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(tdvp_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    path = pkg.build()
    assert os.path.exists(path)
    lib = pkg.load_library()
    declared = _declared()
    assert len(declared) >= 17
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(pkg.EXPORTED_SYMBOLS) == declared


def test_no_cpu_fallback_without_library(monkeypatch, tmp_path):
    import paper_1907_12044_b300._lib as L
    monkeypatch.setattr(L, "_LIB", None)
    monkeypatch.setattr(L, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        L.load_library()


def test_stats_struct_layout_matches_the_header(tmp_path):
    """The ctypes mirror of tdvp_stats_t has the C struct's size and field offsets."""
    import ctypes
    import shutil
    import subprocess
    from paper_1907_12044_b300._lib import StatsC
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f for f, _ in StatsC._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"tdvp.h\"\nint main(void){\n"
                   "printf(\"%zu\\n\", sizeof(tdvp_stats_t));\n"
                   + "".join(f"printf(\"%zu\\n\", offsetof(tdvp_stats_t, {f}));\n" for f in fields)
                   + "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert out[0] == ctypes.sizeof(StatsC)
    assert out[1:] == [getattr(StatsC, f).offset for f in fields]


def test_noalloc_lq_rejects_overlapping_buffers_before_touching_the_device():
    """X, Q and L of tdvp_lq_noalloc must be disjoint; the host check runs before any CUDA call,
    so it needs no GPU (the pointers are never dereferenced)."""
    n, m = 4, 8
    xb, lb = 16 * n * m, 16 * n * n
    base = 1 << 20
    cases = [(base, base + xb - 16, base + 4 * xb),        # X and Q share 16 bytes
             (base, base + 2 * xb, base + xb - 16),        # X and L
             (base, base + 2 * xb, base + 3 * xb - 16),    # Q and L
             (base, base, base + 4 * xb)]                  # in place
    for x, q, l in cases:
        with pytest.raises(pkg.TDVPError) as e:
            pkg.lq_noalloc(n, m, x, q, l, 0)
        assert e.value.code == -1
    assert lb < xb
