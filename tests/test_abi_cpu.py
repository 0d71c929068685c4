"""The C ABI library builds, loads without a GPU, and matches include/ipt.h.

No compute call is made here: the checks are that every function the header
declares is exported, and that the ctypes mirrors of the option/result
structs have the layout a C compiler gives the header's structs.
"""

import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ipt.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ipt_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2012_14702_gb300 import build_lib
    return build_lib.build()


def test_header_declares_the_solver_calls():
    names = declared_functions()
    for f in ["ipt_create", "ipt_destroy", "ipt_solve_dense", "ipt_solve_dense_host",
              "ipt_step_dense", "ipt_solve_csr", "ipt_status_string", "ipt_options_default"]:
        assert f in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name
    nm = shutil.which("nm")
    if nm:
        out = subprocess.run([nm, "-D", "--defined-only", libpath], capture_output=True,
                             text=True).stdout
        exported = set(re.findall(r" T (ipt_\w+)", out))
        assert set(declared_functions()) <= exported


def test_status_strings_and_defaults_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.ipt_status_string.restype = ctypes.c_char_p
    assert lib.ipt_status_string(0) == b"IPT_OK"
    assert lib.ipt_status_string(3) == b"IPT_DEGENERATE_THETA"
    from paper_2012_14702_gb300 import ipt
    o = ipt.Options()
    ipt.lib.ipt_options_default(ctypes.byref(o))
    assert o.precision == ipt.PRECISION["staged"] and o.stop == ipt.STOP["residual"]
    assert o.diverge_bound == 1e8 and o.z0 is None
    assert o.csr_window == 1 and o.epilogue_operand == 1


def test_struct_layout_matches_header(libpath, tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stddef.h>
#include <stdio.h>
#include "ipt.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(ipt_options), offsetof(ipt_options, z0),
         sizeof(ipt_result), offsetof(ipt_result, hist_stage),
         offsetof(ipt_options, epilogue_operand), offsetof(ipt_result, epilogue_operands));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    from paper_2012_14702_gb300 import ipt
    assert vals == [ctypes.sizeof(ipt.Options), ipt.Options.z0.offset,
                    ctypes.sizeof(ipt.Result), ipt.Result.hist_stage.offset,
                    ipt.Options.epilogue_operand.offset, ipt.Result.epilogue_operands.offset]


def test_product_path_has_no_oracle_import():
    """The package never reaches for the CPU oracle."""
    pkg = os.path.join(ROOT, "paper_2012_14702_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
