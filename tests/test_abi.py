"""The C-ABI library loads and exports what include/*.h declares (no GPU needed)."""
import ctypes as C
import glob
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_2602_15018_gb300 import build
    try:
        build._nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    return build.build()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(neurosim_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("neurosim_evsim_create", "neurosim_evsim_step",
                     "neurosim_evsim_drain_events", "neurosim_evsim_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(built):
    lib = C.CDLL(built)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2602_15018_gb300 import _lib
    assert set(_lib.EXPORTS) == set(declared_functions())


def test_abi_version_and_defaults(built):
    from paper_2602_15018_gb300 import _lib
    L = _lib.lib()
    assert L.neurosim_abi_version() == 2
    p = _lib.Params()
    L.neurosim_evsim_default_params(C.byref(p))
    assert abs(p.c_pos - 0.2) < 1e-7 and abs(p.c_min - 0.01) < 1e-7 and p.width == 0
    assert abs(p.log_eps - 1e-3) < 1e-9 and p.input_is_log == 0


def test_struct_layout_matches_header(built):
    """Offsets of every field of the public structs, C compiler vs ctypes."""
    from paper_2602_15018_gb300 import _lib
    structs = {"neurosim_evsim_params": _lib.Params, "neurosim_evsim_stats": _lib.Stats,
               "neurosim_evsim_batch_params": _lib.BatchParams, "neurosim_texture_scene": _lib.TextureScene}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "neurosim_evsim.h"',
             "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines))
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        out = subprocess.check_output([exe], text=True).split("\n")
    got = {}
    for ln in out:
        if ln:
            s, f, v = ln.split()
            got[(s, f)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py)
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_no_gpu_fails_loudly(built):
    """Without a CUDA device the library reports an error instead of computing."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2602_15018_gb300 import _lib
    L = _lib.lib()
    p = _lib.Params()
    L.neurosim_evsim_default_params(C.byref(p))
    p.width, p.height = 8, 8
    h = C.c_void_p()
    rc = L.neurosim_evsim_create(C.byref(p), None, C.byref(h))
    assert rc != 0 and not h.value


def test_batch_defaults_and_no_gpu(built):
    """Batch defaults; without a CUDA device batch creation and the autotuner
    report an error instead of computing."""
    import torch
    from paper_2602_15018_gb300 import _lib
    L = _lib.lib()
    bp = _lib.BatchParams()
    L.neurosim_evsim_batch_default_params(C.byref(bp))
    assert bp.n_streams == 1 and bp.frames_per_step == 16 and bp.dt_us == 1000
    assert bp.t0_us == 0 and bp.event_capacity == 0 and bp.frame_slots == 0
    assert list(bp.reserved) == [0] * 4 and bp.ctas_per_sm == 0
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = _lib.Params()
    L.neurosim_evsim_default_params(C.byref(p))
    p.width, p.height = 8, 8
    h = C.c_void_p()
    assert L.neurosim_evsim_batch_create(C.byref(p), C.byref(bp), None, C.byref(h)) != 0
    assert not h.value
    # argument checks come first and need no device
    bp.n_streams = 0
    assert L.neurosim_evsim_batch_create(C.byref(p), C.byref(bp), None, C.byref(h)) == 1
    assert b"n_streams" in L.neurosim_last_error()
    ppt, pf = C.c_int32(0), C.c_int32(0)
    rc = L.neurosim_evsim_autotune(C.byref(p), C.c_void_p(16), 1, 1000, 3, None, C.byref(ppt),
                                   C.byref(pf), None)
    assert rc == 1 and b"n_frames" in L.neurosim_last_error()


def test_lowpass_gain_matches_the_oracle(built):
    """The bandwidth filter's gain from a cutoff is computed by the library on
    the host (no device needed) and must equal the oracle's own, bit for bit;
    bad arguments are rejected."""
    import numpy as np

    import oracle
    from paper_2602_15018_gb300 import _lib
    L = _lib.lib()
    a = C.c_float(0.0)
    for fc, dt in ((40.0, 1000), (400.0, 1000), (1e9, 1000), (1.0, 10), (37.0, 2000), (150.0, 250)):
        assert L.neurosim_lowpass_alpha(fc, dt, C.byref(a)) == 0
        assert np.float32(a.value) == oracle.lowpass_alpha(fc, dt), (fc, dt)
    for fc, dt in ((0.0, 1000), (-1.0, 1000), (10.0, 0), (float("inf"), 1000), (float("nan"), 1000)):
        assert L.neurosim_lowpass_alpha(fc, dt, C.byref(a)) == 1, (fc, dt)
    assert L.neurosim_lowpass_alpha(10.0, 1000, None) == 1
