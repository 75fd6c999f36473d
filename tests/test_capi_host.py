"""CPU checks of the C ABI: every declared symbol is exported, and the host-only
parts (geometry, argument checking) agree with the oracle and fail cleanly.
No kernel is launched here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth
from tests._cases import C_EXACT, regular

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            src = open(os.path.join(ROOT, "include", hdr)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(cetra_\w+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_2503_20875_gb300 import _native as N
    lib = ctypes.CDLL(N.LIB_PATH)
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding declares a signature for each of them
    assert set(names) <= set(N.SIGNATURES), set(names) - set(N.SIGNATURES)


def test_build_compiles_every_source():
    """Every translation unit under csrc/ is in the build's list (a unit left out would leave
    its symbols missing from libcetra.so on a fresh machine), and the list names no missing
    file."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "cetra_build", os.path.join(ROOT, "paper_2503_20875_gb300", "build.py"))
    build = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(build)
    units = sorted(f for f in os.listdir(build.CSRC) if f.endswith((".cu", ".cpp", ".c")))
    assert sorted(build.SOURCES) == units


def test_header_is_plain_c(tmp_path):
    """A C99 translation unit that includes the header and takes the address of every
    declared entry point compiles without a warning (the boundary needs no C++)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = _declared()
    src = ['#include "cetra.h"', "#include <stddef.h>", "typedef void (*entry)(void);",
           "static const entry table[] = {"]
    src += [f"    (entry)&{n}," for n in names]
    src += ["    NULL};", "int main(void) { return table[0] == NULL; }"]
    c = tmp_path / "consumer.c"
    c.write_text("\n".join(src) + "\n")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"), "-c", str(c),
                        "-o", str(tmp_path / "consumer.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def _geom_lib(t, f, e, durs, cadence=0.0, t0_step=0.0):
    from paper_2503_20875_gb300 import _native as N
    from paper_2503_20875_gb300.api import make_params, _ptr
    prm = make_params(cadence=cadence, t0_step=t0_step)
    info = N.cetra_plan_info()
    t = np.ascontiguousarray(t, np.float64)
    f = np.ascontiguousarray(f, np.float32)
    e = np.ascontiguousarray(e, np.float32)
    d = np.ascontiguousarray(durs, np.float64)
    rc = N.lib.cetra_plan_geometry(None, ctypes.byref(prm), _ptr(t), _ptr(f), _ptr(e), t.size,
                                   _ptr(d), d.size, ctypes.byref(info))
    return rc, info


@pytest.mark.parametrize("case", ["regular", "jitter_default_cadence", "default_step", "offset",
                                  "even_count", "q3", "p3q20"])
def test_host_geometry_matches_oracle(case):
    rng = np.random.default_rng(hash(case) % 2**32)
    t = regular(5001)
    cadence, step = C_EXACT, C_EXACT
    durs = np.array([2.5, 7.0, 31.0]) * C_EXACT
    if case == "jitter_default_cadence":
        t = t + rng.uniform(-0.2, 0.2, t.size) * C_EXACT
        cadence = 0.0
    if case == "even_count":
        t = np.sort(rng.uniform(0, 30, 1000))
        cadence = 0.0
    if case == "default_step":
        step = 0.0
    if case == "offset":
        t = t + 2.45e6
    if case == "q3":
        step = C_EXACT / 3
    if case == "p3q20":
        step = 0.15 * C_EXACT
    f = np.ones(t.size, np.float32)
    e = np.full(t.size, 1e-3, np.float32)
    rc, info = _geom_lib(t, f, e, durs, cadence, step)
    assert rc == 0
    g = oracle.geometry(t, f, e, durs, cadence, step)
    assert info.t_ref == g.t_ref and info.cadence == g.cadence and info.t0_step == g.t0_step
    assert (info.p, info.q, info.n_pad, info.n_grid, info.n_t0, info.n_kept) == \
        (g.p, g.q, g.n_pad, g.n_grid, g.n_t0, g.n_kept)


def test_host_geometry_rejects_bad_input():
    t = regular(100)
    f = np.ones(t.size, np.float32)
    e = np.full(t.size, 1e-3, np.float32)
    assert _geom_lib(t, f, e, [-1.0], C_EXACT)[0] == 1           # D <= 0
    assert _geom_lib(t, f, e, [np.nan], C_EXACT)[0] == 1         # D not finite
    assert _geom_lib(t, f, np.zeros_like(e), [0.1], C_EXACT)[0] == 1  # no usable point
    assert _geom_lib(t[:1], f[:1], e[:1], [0.1])[0] == 1          # cadence undefined
    assert _geom_lib(t, np.full_like(f, np.nan), e, [0.1], C_EXACT)[0] == 1
    assert _geom_lib(t, f, e, [0.1], C_EXACT, 100 * C_EXACT)[0] == 1  # p > 64 unsupported


def test_context_creation_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2503_20875_gb300 import _native as N
    h = ctypes.c_void_p()
    assert N.lib.cetra_create(ctypes.byref(h), 0, None) == N.CETRA_ECUDA
    assert not h.value


def test_binding_refuses_host_and_short_buffers():
    """Device arguments are checked in the binding before any call: host arrays, CPU tensors,
    wrong dtypes, non-contiguous views and short buffers never reach a kernel."""
    torch = pytest.importorskip("torch")
    from paper_2503_20875_gb300 import api
    with pytest.raises(ValueError):
        api._dptr(np.zeros(4, np.float32), "float32", 4, "x")
    with pytest.raises(ValueError):
        api._dptr(torch.zeros(4), "float32", 4, "x")
    with pytest.raises(ValueError):
        api._dptr(None, "float32", 4, "x")
    assert api._dptr(None, "float32", 4, "x", optional=True) is None


def test_static_limit_matches_header():
    """The binding's CETRA_STATIC_MAX_PERIODS is the header's."""
    from paper_2503_20875_gb300 import _native as N
    src = open(os.path.join(ROOT, "include", "cetra.h")).read()
    m = re.search(r"#define\s+CETRA_STATIC_MAX_PERIODS\s+(\d+)", src)
    assert m and int(m.group(1)) == N.CETRA_STATIC_MAX_PERIODS
