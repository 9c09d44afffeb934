"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every function include/dsmc.h declares, and the ctypes structures of the
Python binding have the C layout.  No compute call is made (no GPU here)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dsmc.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dsmc_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2602_21244_gb300 import _build
    path = _build.build()
    assert os.path.exists(path)
    L = C.CDLL(path)
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    L.dsmc_abi_version.restype = C.c_int
    assert L.dsmc_abi_version() == 3


def test_library_targets_sm_103a():
    from paper_2602_21244_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)


def test_struct_layouts_match_c():
    from paper_2602_21244_gb300 import dsmc as D
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "dsmc.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(dsmc_gas_t), sizeof(dsmc_potential_t),
         sizeof(dsmc_mlp_t), sizeof(dsmc_select_info_t), sizeof(dsmc_step_buffers_t),
         sizeof(dsmc_path_t));
  printf("%zu %zu %zu %zu\n", offsetof(dsmc_gas_t, b_max), offsetof(dsmc_potential_t, C),
         offsetof(dsmc_potential_t, p), offsetof(dsmc_step_buffers_t, ws_bytes));
  printf("%zu %zu %d\n", sizeof(dsmc_tune_entry_t), offsetof(dsmc_tune_entry_t, ms), (int)DSMC_TUNE_KERNELS);
  return 0;
}'''
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(td, "t")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(x) for x in out]
    assert sizes[:6] == [C.sizeof(D.Gas), C.sizeof(D.Potential), C.sizeof(D.Mlp),
                         C.sizeof(D.SelectInfo), C.sizeof(D.StepBuffers), C.sizeof(D.Path)]
    assert sizes[6:10] == [D.Gas.b_max.offset, D.Potential.C.offset, D.Potential.p.offset,
                           D.StepBuffers.ws_bytes.offset]
    assert sizes[10:] == [C.sizeof(D.TuneEntry), D.TuneEntry.ms.offset, len(D.TUNE_KERNELS)]


def test_context_create_fails_cleanly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2602_21244_gb300 import dsmc as D
    with pytest.raises(D.DsmcError):
        D.Context(0)
