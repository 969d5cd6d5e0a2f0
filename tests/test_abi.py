"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/opmm.h declares; the ctypes structs match the C layout.  No compute is
launched here (no GPU)."""
import os
import re
import subprocess
import ctypes

import pytest

import paper_2007_09884_gb300 as G
from paper_2007_09884_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "opmm.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(opmm_\w+)\s*\(", txt, re.M)))


def test_library_builds_and_exports_every_declared_symbol():
    B.build()
    lib = ctypes.CDLL(G.LIB_PATH)
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(G.EXPORTS) <= set(names)


def test_struct_layouts_match_c(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "opmm.h"
int main(void) {
  printf("%zu %zu %zu\\n", sizeof(opmm_saccade), sizeof(opmm_fit_opts), sizeof(opmm_fit_result));
  printf("%zu %zu %zu %zu\\n", offsetof(opmm_fit_result, f), offsetof(opmm_fit_result, rms_deg),
         offsetof(opmm_fit_result, status), offsetof(opmm_fit_opts, init_opc));
  printf("%zu %zu %zu %zu\\n", sizeof(opmm_ivt_event), sizeof(opmm_ivt_opts), sizeof(opmm_refine_opts),
         offsetof(opmm_refine_opts, centre_opc));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    a, b, c = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")[:3]
    sizes = [int(x) for x in a.split()]
    offs = [int(x) for x in b.split()]
    assert sizes == [ctypes.sizeof(G.opmm_saccade), ctypes.sizeof(G.opmm_fit_opts),
                     ctypes.sizeof(G.opmm_fit_result)]
    assert offs == [G.opmm_fit_result.f.offset, G.opmm_fit_result.rms_deg.offset,
                    G.opmm_fit_result.status.offset, G.opmm_fit_opts.init_opc.offset]
    assert [int(x) for x in c.split()] == [G.IVT_EVENT_DTYPE.itemsize, ctypes.sizeof(G.opmm_ivt_opts),
                                           ctypes.sizeof(G.opmm_refine_opts), G.opmm_refine_opts.centre_opc.offset]


def test_no_device_fails_loudly():
    """Without a usable GPU the product path refuses: there is no CPU fallback."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(G.OpmmError):
        G.opmm_create(0)


def test_product_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2007_09884_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "opmm_oracle" not in txt, f
