"""The C ABI without a GPU: liblst.so builds and loads, exports every function include/lst.h
declares, its struct layouts match the Python binding, and its constants table equals the
oracle's."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_2207_08207_gb300 import lst

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    L = lst.lib()
    names = lst.exported_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


def test_constants_equal_oracle_constants():
    c = lst.default_config()
    mine = [float(getattr(c, f)) for f in lst._CONST_FIELDS] + [float(c.t5_overlap_hits)]
    ref = oracle.constants().tolist()
    assert mine == ref


def _c_layout():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "lst.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(lst_config), sizeof(lst_module), sizeof(lst_pls),
         sizeof(lst_event_in), sizeof(lst_counts), sizeof(lst_event_out),
         offsetof(lst_config, cycle_budget), offsetof(lst_event_out, tc_phi));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        with open(c, "w") as f:
            f.write(src)
        subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        return [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]


def test_struct_layouts_match_binding():
    from paper_2207_08207_gb300 import gen
    got = _c_layout()
    want = [ctypes.sizeof(lst.Config), gen.MODULE_DTYPE.itemsize, gen.PLS_DTYPE.itemsize,
            ctypes.sizeof(lst.EventIn), ctypes.sizeof(lst.Counts), ctypes.sizeof(lst.EventOut),
            lst.Config.cycle_budget.offset, lst.EventOut.tc_phi.offset]
    assert got == want


def test_create_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = lst.lib()
    h = ctypes.c_void_p()
    cfg = lst.default_config()
    rc = L.lst_create(ctypes.byref(h), ctypes.byref(cfg), 0)
    assert rc in (lst.LST_ECUDA, lst.LST_EINVAL)
    assert not h.value
    assert len(L.lst_last_error(None)) > 0
    # NULL contexts are rejected, not dereferenced
    assert L.lst_sync(None, None) == lst.LST_EINVAL
    assert L.lst_query(None) < 0
    L.lst_destroy(None)
