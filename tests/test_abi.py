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


def test_ozaki_gemm_rejects_bad_arguments_before_touching_the_device():
    """tdvp_zgemm_ozaki checks sizes, slice count, workspace size and alignment, 16-byte operand
    alignment and overlap on the host before any CUDA call (the pointers are never dereferenced)."""
    assert pkg.zgemm_ozaki_workspace(0, 4, 4, 8) == 0
    assert pkg.zgemm_ozaki_workspace(4, 4, 4, 0) == 0 and pkg.zgemm_ozaki_workspace(4, 4, 4, 9) == 0
    assert pkg.zgemm_ozaki_workspace(4, 4, (1 << 21) + 1, 8) == 0
    m, n, k = 40, 30, 20
    wsb = pkg.zgemm_ozaki_workspace(m, n, k, 8)
    assert wsb > 0 and wsb % 1024 == 0
    A, B, C, W = 1 << 24, 1 << 25, 1 << 26, 1 << 30
    cases = [
        dict(slices=0), dict(slices=9), dict(ws_bytes=wsb - 1), dict(a=0), dict(w=0),
        dict(w=W + 512),                       # workspace not 1024-byte aligned
        dict(a=A + 8),                         # operand not 16-byte aligned
        dict(c=A + 16),                        # C overlaps A
        dict(w=B),                             # workspace overlaps B
    ]
    for cs in cases:
        with pytest.raises(pkg.TDVPError) as e:
            pkg.zgemm_ozaki(m, n, k, cs.get("a", A), cs.get("b", B), cs.get("c", C), cs.get("slices", 8),
                            cs.get("w", W), cs.get("ws_bytes", wsb), 0)
        assert e.value.code == -1, cs
