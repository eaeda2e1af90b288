"""The C-ABI library loads, exports every symbol include/*.h declares, and validates arguments on
the host (no GPU needed: every check below fails before any device call)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(pat_[A-Za-z0-9_]+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    from paper_1603_02329_gb300 import build, _lib

    build.build()
    return _lib.lib()


def test_header_declares_the_hot_path_calls():
    names = _declared_symbols()
    for n in ["pat_plan_create", "pat_plan_destroy", "pat_forward", "pat_forward_plan", "pat_adjoint", "pat_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(L):
    missing = [n for n in _declared_symbols() if not hasattr(L, n)]
    assert not missing, missing


def _grid(n=(16, 16), pml=(2, 2)):
    from paper_1603_02329_gb300.api import make_grid

    return make_grid(n, (1e-4, 1e-4), pml, 2.0)


def _call_create(L, grid, c, rho, a0, y=1.5, sens_pos=None, sens_idx=None, dt=1e-8, Nt=10, prec=0):
    from paper_1603_02329_gb300 import _lib

    dp = ctypes.POINTER(ctypes.c_double)
    s = _lib.pat_sensors()
    keep = []
    if sens_idx is not None:
        a = np.ascontiguousarray(np.asarray(sens_idx, np.int64))
        keep.append(a)
        s.count, s.index = a.size, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    if sens_pos is not None:
        a = np.ascontiguousarray(np.asarray(sens_pos, np.float64))
        keep.append(a)
        s.count, s.pos = a.shape[0], a.ctypes.data_as(dp)
    plan = ctypes.c_void_p()
    st = L.pat_plan_create(ctypes.byref(grid), c.ctypes.data_as(dp), rho.ctypes.data_as(dp), a0.ctypes.data_as(dp),
                           int(a0.size == 1), float(y), ctypes.byref(s), float(dt), int(Nt), int(prec),
                           ctypes.byref(plan))
    return st, plan


def test_host_side_argument_validation(L):
    from paper_1603_02329_gb300._lib import PAT_EINVAL, PAT_EUNSUPPORTED

    N = 256
    c = np.full(N, 1500.0)
    rho = np.full(N, 1000.0)
    a0 = np.zeros(1)
    # odd grid size
    st, _ = _call_create(L, _grid((16, 15)), np.full(240, 1500.0), np.full(240, 1000.0), a0, sens_idx=[0])
    assert st == PAT_EUNSUPPORTED
    # a prime factor of 11 (22 = 2 * 11) is not a supported FFT length
    st, _ = _call_create(L, _grid((16, 22)), np.full(352, 1500.0), np.full(352, 1000.0), a0, sens_idx=[0])
    assert st == PAT_EUNSUPPORTED
    # sensor index outside the grid
    st, _ = _call_create(L, _grid(), c, rho, a0, sens_idx=[N])
    assert st == PAT_EINVAL
    # sensor position outside the grid
    st, _ = _call_create(L, _grid(), c, rho, a0, sens_pos=[[1.0, 0.0]])
    assert st == PAT_EINVAL
    # negative sound speed
    bad = c.copy()
    bad[3] = -1.0
    st, _ = _call_create(L, _grid(), bad, rho, a0, sens_idx=[0])
    assert st == PAT_EINVAL
    # y = 1 with absorption (tan(pi y / 2) diverges)
    st, _ = _call_create(L, _grid(), c, rho, np.full(1, 0.5), y=1.0, sens_idx=[0])
    assert st == PAT_EINVAL
    # Nt = 0, dt <= 0, PML wider than half the grid
    assert _call_create(L, _grid(), c, rho, a0, sens_idx=[0], Nt=0)[0] == PAT_EINVAL
    assert _call_create(L, _grid(), c, rho, a0, sens_idx=[0], dt=0.0)[0] == PAT_EINVAL
    assert _call_create(L, _grid(pml=(9, 2)), c, rho, a0, sens_idx=[0])[0] == PAT_EINVAL
    msg = L.pat_last_error().decode()
    assert "PML" in msg
    # NULL arguments
    assert L.pat_plan_create(None, None, None, None, 0, 1.5, None, 1e-8, 10, 0, None) == PAT_EINVAL
    assert L.pat_forward_plan(None, None, None, None) == PAT_EINVAL
    assert L.pat_adjoint(None, None, None, None) == PAT_EINVAL
    assert L.pat_plan_destroy(None) == 0
    # multi-level MG-FISTA: NULL levels, nlevels outside 1 .. 8 (checked before any device work)
    from paper_1603_02329_gb300._lib import ITER_CB

    assert L.pat_mg_fista_levels(None, 2, None, None, None, None, None, None, ITER_CB(0), None, None) == PAT_EINVAL
    assert "nlevels" in L.pat_last_error().decode()
    assert L.pat_mg_fista(None, None, None, None, None, None, None, ITER_CB(0), None, None) == PAT_EINVAL
    # size limits, checked before the medium arrays are read: 1024^3 points, Nt * Ns >= 2^31
    from paper_1603_02329_gb300.api import make_grid

    g3 = make_grid((1024, 1024, 1024), (1e-4,) * 3, (4,) * 3, 2.0)
    assert _call_create(L, g3, c, rho, a0, sens_idx=[0])[0] == PAT_EUNSUPPORTED
    assert "2^27" in L.pat_last_error().decode()
    assert _call_create(L, _grid(), c, rho, a0, sens_idx=list(range(256)), Nt=1 << 24)[0] == PAT_EUNSUPPORTED
    # p0 smoothing: NULL plan / arguments (checked before any device work)
    assert L.pat_plan_set_smoothing(None, 1) == PAT_EINVAL
    assert L.pat_plan_smooth(None, None, None, None) == PAT_EINVAL


def test_header_is_plain_c_and_every_declaration_links(L, tmp_path):
    """include/*.h compile as strict C99 and C++17 on their own (no other header before them), and a C
    program that takes the address of every declared entry point links against the library: the
    boundary is plain C with unmangled names."""
    import shutil
    import subprocess

    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("gcc not found")
    names = _declared_symbols()
    src = tmp_path / "abi.c"
    body = "\n".join(f"    (fn_t)&{n}," for n in names)
    src.write_text('#include "pat.h"\n#include <stdio.h>\ntypedef void (*fn_t)(void);\n'
                   f"static const fn_t entry[] = {{\n{body}\n}};\n"
                   'int main(void) { printf("%d\\n", (int)(sizeof(entry) / sizeof(entry[0]))); return 0; }\n')
    inc = os.path.join(ROOT, "include")
    for std, lang in (("c99", "c"), ("c++17", "c++")):
        r = subprocess.run([cc if lang == "c" else (shutil.which("g++") or cc), f"-std={std}", "-Wall", "-Wextra",
                            "-pedantic", "-Werror", "-fsyntax-only", "-I", inc, "-x", lang, str(src)],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
    so = L._name   # the path the binding loaded the library from
    exe = tmp_path / "abi"
    r = subprocess.run([cc, "-std=c99", "-I", inc, str(src), so, "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def _prototypes():
    """name -> number of parameters of every pat_* function declared in include/*.h"""
    out = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"\b(pat_[A-Za-z0-9_]+)\s*\(([^;{]*?)\)\s*;", txt, flags=re.S):
            params = " ".join(m.group(2).split())
            if m.group(1).startswith("pat_iter_callback") or params in ("", "void"):
                out.setdefault(m.group(1), 0)
                continue
            depth, n = 0, 1
            for ch in params:
                depth += ch == "("
                depth -= ch == ")"
                n += ch == "," and depth == 0
            out[m.group(1)] = n
    return out


def test_binding_declares_every_entry_point_with_the_headers_arity(L):
    """The ctypes binding gives every declared entry point its argument list (ctypes would otherwise
    pass Python ints as 32-bit C ints) with as many arguments as the prototype."""
    protos = _prototypes()
    assert set(_declared_symbols()) <= set(protos)
    for name in _declared_symbols():
        f = getattr(L, name)
        assert f.argtypes is not None, name
        assert len(f.argtypes) == protos[name], (name, len(f.argtypes), protos[name])


def test_binding_structs_match_the_c_layout(L, tmp_path):
    """Size and field offsets of every struct the binding mirrors, as gcc lays them out from pat.h."""
    import shutil
    import subprocess

    from paper_1603_02329_gb300 import _lib

    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("gcc not found")
    structs = [_lib.pat_grid, _lib.pat_sensors, _lib.pat_plan_info_t, _lib.pat_fista_opts, _lib.pat_fista_report]
    lines = ['#include "pat.h"', "#include <stddef.h>", "#include <stdio.h>", "int main(void) {"]
    for S in structs:
        c = S.__name__
        lines.append(f'    printf("{c} size %zu\\n", sizeof({c}));')
        for fname, _ in S._fields_:
            cf = fname.rstrip("_")   # lambda_ in Python is lambda in C
            lines.append(f'    printf("{c} {fname} %zu\\n", offsetof({c}, {cf}));')
    lines += ["    return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    r = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        s, f, v = ln.split()
        got[(s, f)] = int(v)
    for S in structs:
        assert got[(S.__name__, "size")] == ctypes.sizeof(S), S.__name__
        for fname, _ in S._fields_:
            assert got[(S.__name__, fname)] == getattr(S, fname).offset, (S.__name__, fname)
