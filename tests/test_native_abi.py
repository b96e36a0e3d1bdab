"""The C-ABI library builds, loads and exports every entry point include/transit.h declares
(no GPU needed: only symbol lookup, no compute call)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "transit.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tr_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1912_07759_gb300 import build
    return build.build()


def test_library_exports_every_declared_entry_point(lib_path):
    lib = ctypes.CDLL(lib_path)
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_covers_the_header(lib_path):
    from paper_1912_07759_gb300 import _native
    assert set(_native.exported_names()) == set(declared_functions())
    _native.load(lib_path)


def test_binding_struct_sizes_match_the_header(lib_path):
    """The ctypes mirrors have the C layout: compile a probe that prints sizeof/offsetof."""
    import subprocess
    import tempfile
    from paper_1912_07759_gb300 import _native as N
    probe = r'''
#include <stdio.h>
#include <stddef.h>
#include "transit.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(tr_table_desc), sizeof(tr_atm_desc),
         sizeof(tr_batch_desc), offsetof(tr_table_desc, oor_mode),
         offsetof(tr_atm_desc, cloud_mode), offsetof(tr_batch_desc, max_layers),
         offsetof(tr_atm_desc, guillot), offsetof(tr_atm_desc, log10_p_switch),
         offsetof(tr_batch_desc, t_int));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        open(c, "w").write(probe)
        exe = os.path.join(d, "p")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    got = [ctypes.sizeof(N.TableDesc), ctypes.sizeof(N.AtmDesc), ctypes.sizeof(N.BatchDesc),
           N.TableDesc.oor_mode.offset, N.AtmDesc.cloud_mode.offset, N.BatchDesc.max_layers.offset,
           N.AtmDesc.guillot.offset, N.AtmDesc.log10_p_switch.offset, N.BatchDesc.t_int.offset]
    assert [int(x) for x in out] == got


def test_missing_library_fails_loudly(tmp_path):
    from paper_1912_07759_gb300 import _native
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _native._lib_backup = _native._lib
        try:
            _native._lib = None
            _native.load(str(tmp_path / "nope.so"))
        finally:
            _native._lib = _native._lib_backup
