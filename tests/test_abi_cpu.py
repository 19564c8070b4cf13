"""CPU-side checks of the C ABI: the library loads, exports what the header
declares, validates its arguments, and its host-only model STF matches the
oracle.  No compute call here needs a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import speckle_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "speckle.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sm_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_1701_00581_gb300 as P
    from paper_1701_00581_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return P.load()


def test_header_symbols_are_exported(lib):
    names = _header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), f"{n} declared in speckle.h but not exported"


def test_binding_covers_header():
    from paper_1701_00581_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == _header_functions()


_STRUCTS = ["sm_channel", "sm_plan_info", "sm_workspace_layout", "sm_config", "sm_burst", "sm_result",
            "sm_batch_opts", "sm_batch_io"]


def test_header_constants_match_binding():
    """Every integer #define SM_... of the header has the same value in the
    binding (a constant renumbered on one side only would pass other tests)."""
    from paper_1701_00581_gb300 import _lib
    src = open(os.path.join(ROOT, "include", "speckle.h")).read()
    defs = dict(re.findall(r"^#define\s+(SM_[A-Z0-9_]+)\s+(-?\d+)\b", src, flags=re.M))
    assert len(defs) >= 20
    for name, value in defs.items():
        assert hasattr(_lib, name), f"{name} defined in speckle.h but missing from the binding"
        assert getattr(_lib, name) == int(value), name


def test_struct_layouts_match_header(tmp_path):
    """Every ctypes mirror has the C compiler's size and field offsets for
    the header's struct (a field added on one side only shifts the rest)."""
    import shutil
    import subprocess
    from paper_1701_00581_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "speckle.h"', "int main(void) {"]
    expect = []
    for name in _STRUCTS:
        cls = getattr(_lib, name)
        lines.append(f'  printf("%zu\\n", sizeof({name}));')
        expect.append(C.sizeof(cls))
        for f in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({name}, {f[0]}));')
            expect.append(getattr(cls, f[0]).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == expect


def test_strerror(lib):
    assert lib.sm_strerror(0) == b"ok"
    assert lib.sm_strerror(-3) == b"no free slot, retry later"
    assert lib.sm_strerror(12345) == b"unknown status"


@pytest.mark.parametrize("field,value", [
    ("N", 100), ("N", 512), ("R", 0), ("R", 40), ("fc", 0.0), ("fc", 0.5), ("taper", 40),
    ("stride", 0), ("spectra_prec", 3), ("phase_weight", 3), ("max_frames", 0), ("W", 0),
    ("acc_mode", 2), ("phase_prec", 3), ("phase_iters", -1), ("phase_iters", 65)])
def test_plan_create_rejects_bad_channels(lib, field, value):
    from paper_1701_00581_gb300 import Channel
    ch = Channel(W=256, H=256, N=128, R=16).to_c()
    setattr(ch, field, value)
    h = C.c_void_p()
    assert lib.sm_plan_create(C.byref(ch), 0, C.byref(h)) == -1
    assert not h.value
    assert len(lib.sm_last_error()) > 0


def test_model_stf_matches_oracle(lib):
    from paper_1701_00581_gb300 import Channel
    rng = np.random.default_rng(5)
    for N, fc, ck in ((64, 0.2885, 0.435), (128, 0.25, 0.3), (256, 0.2885, 0.0)):
        d = rng.uniform(5, 15, 7)
        ch = Channel(W=N, H=N, N=N, R=4, fc=fc, ck=ck).to_c()
        out = np.zeros((N, N))
        assert lib.sm_model_stf(C.byref(ch), len(d), d.ctypes.data, out.ctypes.data) == 0
        ref = O.stf_model(N, fc, d, ck)
        assert np.max(np.abs(out - ref)) < 1e-12


def test_model_stf_rejects_bad_input(lib):
    from paper_1701_00581_gb300 import Channel
    ch = Channel(W=64, H=64, N=64, R=4).to_c()
    out = np.zeros((64, 64))
    d = np.array([5.0, -1.0])
    assert lib.sm_model_stf(C.byref(ch), 2, d.ctypes.data, out.ctypes.data) == -1
    assert lib.sm_model_stf(C.byref(ch), 0, d.ctypes.data, out.ctypes.data) == -1


def test_null_arguments_are_rejected(lib):
    from paper_1701_00581_gb300 import _lib
    lay = _lib.sm_workspace_layout()
    assert lib.sm_workspace_query(None, 1, 1, C.byref(lay)) == -1
    assert lib.sm_plan_get_info(None, None) == -1
    assert lib.sm_stage_bispectrum(None, 1, 1, None, None, None) == -1
    assert lib.sm_poll(None, 1, 0, None) == -1
    assert lib.sm_close(None) == 0
    assert lib.sm_plan_destroy(None) == 0


def test_open_rejects_an_unpaired_allocator(lib):
    """sm_open wants dev_alloc and dev_free together (checked before any
    device work)."""
    from paper_1701_00581_gb300 import Channel, _lib
    ch = (_lib.sm_channel * 1)(Channel(W=96, H=80, N=64, R=4, max_frames=4).to_c())
    alloc = _lib.DEV_ALLOC(lambda n, ctx: None)
    h = C.c_void_p()
    for a, f in ((alloc, _lib.DEV_FREE()), (_lib.DEV_ALLOC(), _lib.DEV_FREE(lambda p, ctx: None))):
        cfg = _lib.sm_config(1, ch, 1 << 20, 1, 0, 0, a, f, None)
        assert lib.sm_open(C.byref(cfg), C.byref(h)) == _lib.SM_EINVAL
        assert b"together" in lib.sm_last_error()
