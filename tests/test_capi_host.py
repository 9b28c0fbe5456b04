"""Host-side checks of the C-ABI library that need no GPU: it builds for sm_103a, loads, exports
every entry point include/grlb.h declares, its struct layouts match the Python binding, and
parameter validation rejects bad input."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2609_16361_b300 import capi, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "grlb.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(grlb_[a-z_0-9]+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    L = capi.lib()
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), f"{n} missing from libgrlb.so"
    assert set(capi.exported_symbols()) >= set(names)
    out = subprocess.run(["nm", "-D", "--defined-only", capi.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}$", out, re.M), n
    assert b"sm_103a" in capi.lib().grlb_version()


def test_checked_build_loads_and_exports_the_same_symbols():
    """libgrlb_checked.so (GRLB_CHECKED, relocatable device code) builds, loads beside the plain
    library and exports every declared entry point; only it reports itself as checked, and the
    plain library refuses the checker's calls with GRLB_ESTATE."""
    from paper_2609_16361_b300 import build
    path = build.build(checked=True)
    Lc = C.CDLL(path)
    for n in declared_functions():
        assert hasattr(Lc, n), f"{n} missing from libgrlb_checked.so"
    Lc.grlb_checked_build.restype = C.c_int32
    assert Lc.grlb_checked_build() == 1
    assert capi.lib().grlb_checked_build() == 0
    c = capi.grlb_check_counts()
    assert capi.lib().grlb_check_read(C.byref(c), 0) == -6
    assert b"not a bounds-checked build" in capi.lib().grlb_last_error()
    assert capi.lib().grlb_check_probe(None, 16, 0, 4, None) == -6


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "lay.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "grlb.h"
int main(void){
 printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(grlb_params), offsetof(grlb_params, T_S),
        offsetof(grlb_params, right_prim), sizeof(grlb_diag), offsetof(grlb_diag, n_floor),
        sizeof(grlb_batch_config), sizeof(grlb_check_counts), offsetof(grlb_check_counts, overflow));
 return 0;}
''')
    exe = tmp_path / "lay"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert vals == [C.sizeof(capi.grlb_params), capi.grlb_params.T_S.offset,
                    capi.grlb_params.right_prim.offset, C.sizeof(capi.grlb_diag),
                    capi.grlb_diag.n_floor.offset, C.sizeof(capi.grlb_batch_config),
                    C.sizeof(capi.grlb_check_counts), capi.grlb_check_counts.overflow.offset]


def test_parameter_validation_without_device():
    good = inputs.tgv3d(32).params
    assert capi.grlb_bytes_for(good) == pytest.approx(2 * 35 * 32 ** 3 * 4, rel=0.05)
    f16 = good.replace(storage=inputs.STORE_F16)
    assert capi.grlb_bytes_for(f16) < capi.grlb_bytes_for(good) * 0.6
    bad = [good.replace(nx=0), good.replace(omega_mom=2.5), good.replace(dt=-1.0),
           good.replace(gamma=1.0), good.replace(storage=7), good.replace(bc=3),
           good.replace(ref_p=0.0), good.replace(nx=2048, ny=2048, nz=1024)]
    for b in bad:
        assert capi.grlb_bytes_for(b) == 0
    # moment storage: FP32 and the regularized collision only, 20 values per cell and buffer
    mom = good.replace(streaming=2)
    assert capi.grlb_bytes_for(good) - capi.grlb_bytes_for(mom) == 2 * (35 - 20) * 4 * 32 ** 3
    for b in (mom.replace(collision=inputs.COLL_BGK), mom.replace(collision=inputs.COLL_RLB_GATED),
              mom.replace(storage=inputs.STORE_F16), mom.replace(storage=inputs.STORE_BF16),
              good.replace(streaming=3), good.replace(streaming=-1)):
        assert capi.grlb_bytes_for(b) == 0
    h = C.c_void_p()
    st = capi.lib().grlb_create(C.byref(capi.to_params(good.replace(nx=0))), None, C.byref(h))
    assert st == -1 and b"nx" in capi.lib().grlb_last_error()
    cells = (C.c_int64 * 1)(0)
    out = (C.c_double * 35)()
    assert capi.lib().grlb_read_cells(None, cells, 1, out) == -1


@pytest.mark.parametrize("shape", [(32, 32, 32), (10, 7, 3), (129, 1, 1), (40, 21, 7)])
def test_population_buffers_are_whole_cell_bricks(shape):
    """Populations live in bricks of 128 cells x 35 rows: a buffer holds ceil(N / 128) bricks
    whatever N is (ragged last brick included), two buffers per two-buffer domain, one for the
    one-buffer (AA) pattern; FP32 and FP16 differ only in the element size."""
    nx, ny, nz = shape
    p32 = inputs.uniform(nx, ny, nz).params
    p16 = p32.replace(storage=inputs.STORE_F16)
    bricks = -(-(nx * ny * nz) // 128)
    one_buffer_f16 = 35 * 128 * bricks * 2
    assert capi.grlb_bytes_for(p32) - capi.grlb_bytes_for(p16) == 2 * one_buffer_f16
    assert capi.grlb_bytes_for(p16) - capi.grlb_bytes_for(p16.replace(streaming=1)) == one_buffer_f16


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="a GPU is present")
def test_create_fails_cleanly_without_device():
    h = C.c_void_p()
    st = capi.lib().grlb_create(C.byref(capi.to_params(inputs.tgv3d(8).params)), None, C.byref(h))
    assert st in (-2, -3) and not h.value
    assert len(capi.lib().grlb_last_error()) > 0


def test_spectrum_shell_count_without_device():
    from oracle import spectral
    for n in (2, 16, 64, 256):
        assert capi.grlb_spectrum_shells(inputs.tgv3d(n).params) == spectral.shells(n, n, n)
    assert capi.grlb_spectrum_shells(inputs.tgv2d(64).params) == spectral.shells(64, 64, 1)
    assert capi.grlb_spectrum_shells(inputs.random_smooth(16, 8, 8).params) == -1
