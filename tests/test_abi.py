"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "kde.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"KDE_API\s+[\w\s\*]+?\b(kde_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1505_02100_gb300 import build
    build.build()
    import paper_1505_02100_gb300 as kde
    return kde.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("kde_psi", "kde_plugin_h", "kde_plugin_h_batch", "kde_server_create",
                     "kde_server_submit", "kde_server_poll", "kde_server_destroy", "kde_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_only_declared_symbols_are_exported(lib):
    from paper_1505_02100_gb300.build import LIB
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    ours = {s for s in exported if s.startswith("kde_")}
    assert ours == set(_declared())


def test_binding_covers_the_header():
    import paper_1505_02100_gb300 as kde
    assert set(kde.SIGNATURES) == set(_declared())


def test_result_struct_layout():
    import ctypes

    import paper_1505_02100_gb300 as kde
    assert ctypes.sizeof(kde.KdeResult) == 8 * 8 + 8
    assert kde.KdeResult.status.offset == 64


def test_struct_layouts_match_the_header(tmp_path):
    """sizeof and every field offset of the public structs, as gcc lays them out
    from include/kde.h, against the ctypes mirrors of the binding."""
    import ctypes
    import subprocess

    import paper_1505_02100_gb300 as kde
    mirrors = {"kde_result": kde.KdeResult, "kde_stage_result": kde.KdeStageResult,
               "kde_server_config": kde.KdeServerConfig, "kde_request_times": kde.KdeRequestTimes}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{os.path.join(ROOT, "include", "kde.h")}"',
             "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {(a, b): int(c) for a, b, c in (ln.split() for ln in out if ln.strip())}
    for cname, py in mirrors.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_errors_without_compute(lib):
    """Argument validation happens before any device work."""
    import ctypes

    import paper_1505_02100_gb300 as kde
    res = kde.KdeResult()
    x = (ctypes.c_double * 1)(1.0)
    assert lib.kde_plugin_h(ctypes.addressof(x), 1, kde.KDE_FP32, ctypes.addressof(res), None) == kde.KDE_ERR_INVALID
    assert "n < 2" in kde.kde_last_error()
    assert lib.kde_plugin_h(None, 5, kde.KDE_FP32, ctypes.addressof(res), None) == kde.KDE_ERR_INVALID
    out = ctypes.c_double()
    assert lib.kde_psi(ctypes.addressof(x), 8, 5, 1.0, kde.KDE_FP32, ctypes.addressof(out), None) == kde.KDE_ERR_INVALID
    assert lib.kde_psi(ctypes.addressof(x), 8, 4, -1.0, kde.KDE_FP32, ctypes.addressof(out), None) == kde.KDE_ERR_INVALID


def test_product_does_not_touch_the_oracle():
    """The CUDA path and the oracle share no code and neither imports the other."""
    pkg = os.path.join(ROOT, "paper_1505_02100_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                for bad in ("import oracle", "from oracle", "liboracle", "kde_oracle"):
                    assert bad not in text, (f, bad)
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_1505_02100_gb300" not in text and "kde.h" not in text, f
