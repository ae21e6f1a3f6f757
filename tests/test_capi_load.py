"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/xfft.h declares
(no GPU calls)."""
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "xfft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(xfft_[a-z_0-9]+)\s*\(", src)))


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_library_builds_loads_and_exports_header_symbols():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_02172_gb300 import capi
    L = capi.lib()
    names = _declared()
    assert len(names) >= 14
    for nm in names:
        assert hasattr(L, nm), nm
    assert set(names) == set(capi.EXPORTED)
    # host-only entry points work without a GPU
    o = capi.Options()
    assert L.xfft_default_options(o) == 0 and o.tol == 1e-10 and o.poll_every == 8
    assert o.scheme == 0 and o.cut_cache == 0 and o.enr_precond == 0 and o.inner_tol == 1e-5
    assert L.xfft_status_string(4).decode() == "not converged"


def test_product_path_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2601_02172_gb300 import capi
    monkeypatch.setattr(capi, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(capi, "_lib", None)
    with pytest.raises(RuntimeError):
        capi.lib()


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes structures of the binding have the C header's size and field offsets (a field
    appended on one side only would shift every later argument)."""
    import ctypes as C
    import subprocess
    from paper_2601_02172_gb300 import capi
    cases = {"xfft_grid": capi.Grid, "xfft_options": capi.Options, "xfft_stats": capi.Stats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "xfft.h"', "int main(void) {"]
    for cname, cls in cases.items():
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in cls._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in cases.items():
        assert got[(cname, "size")] == C.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
