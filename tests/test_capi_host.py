"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every function declared in include/lp.h; argument checks that happen
before any CUDA call report LP_ERR_INVALID_ARG."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def L():
    from paper_2206_14061_gb300 import build, capi
    build.build()
    return capi.lib()


def test_exports_every_header_function(L):
    from paper_2206_14061_gb300 import capi
    names = capi.header_functions()
    assert len(names) >= 11
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(capi._SIGS)


def test_version_and_status_strings(L):
    assert b"sm_103a" in L.lp_version()
    for s in range(8):
        assert L.lp_status_string(s)
    assert L.lp_status_string(0) == b"ok"
    assert L.lp_status_string(99) == b"unknown status"


def test_invalid_arguments_fail_on_host(L):
    from paper_2206_14061_gb300 import capi
    h = ctypes.c_void_p()
    bad = [capi.LpCtxDesc(0, 1, 0, 64, 0),       # no particles
           capi.LpCtxDesc(0, 1, 1000, 0, 0),     # cap 0
           capi.LpCtxDesc(0, 1, 1000, 65, 0),    # cap above LP_MAX_CAP
           capi.LpCtxDesc(0, 0, 1000, 64, 0)]    # no columns
    for d in bad:
        assert L.lp_ctx_create(ctypes.byref(d), ctypes.byref(h)) == capi.LP_ERR_INVALID_ARG
    assert L.lp_ctx_create(None, ctypes.byref(h)) == capi.LP_ERR_INVALID_ARG
    assert L.lp_ctx_destroy(None) == capi.LP_ERR_INVALID_ARG
    assert L.lp_ctx_sync(None, None, None) == capi.LP_ERR_INVALID_ARG
    assert L.lp_step(None, None, None, None, None, 1e-5, 1, None) == capi.LP_ERR_INVALID_ARG
    assert L.lp_build_neighbors(None, None, None, 0.0, 0, 0.0, 1, 0, None,
                                None) == capi.LP_ERR_INVALID_ARG
    assert L.lp_fit_derivatives(None, None, None, None, None, 0, 1.0, 0.0, None, 0,
                                None) == capi.LP_ERR_INVALID_ARG
    assert L.lp_mui_stress(None, None, None, 0, None, None, None, None, None, None, None,
                           None) == capi.LP_ERR_INVALID_ARG
    assert L.lp_step_adjoint(None, None, None, None, None, 1e-5, 1, 1, None, None, None,
                             None) == capi.LP_ERR_INVALID_ARG
    assert L.lp_ctx_set_adjoint_memory(None, 0) == capi.LP_ERR_INVALID_ARG
    assert L.lp_ctx_set_wait_limit(None, 1, 0) == capi.LP_ERR_INVALID_ARG


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """The binding raises instead of falling back when liblp.so is absent."""
    from paper_2206_14061_gb300 import build, capi
    monkeypatch.setattr(build, "LIB", str(tmp_path / "absent.so"))
    monkeypatch.setattr(capi, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        capi.lib()


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct the binding marshals has the size and field offsets that a
    C compiler gives the declaration in include/lp.h."""
    import os
    import shutil
    import subprocess
    from paper_2206_14061_gb300 import capi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"lp_ctx_desc": capi.LpCtxDesc, "lp_particles": capi.LpParticles,
               "lp_mui": capi.LpMui, "lp_eos": capi.LpEos, "lp_params": capi.LpParams,
               "lp_neighbors": capi.LpNeighbors, "lp_diag": capi.LpDiag,
               "lp_tuning": capi.LpTuning}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lp.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", f"-I{inc}", str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True,
                               text=True).stdout.splitlines():
        a, b, v = line.split()
        got[(a, b)] = int(v)
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_binding_signatures_match_the_header():
    """Every function the binding declares takes as many arguments as its
    prototype in include/lp.h, and returns lp_status (int32) unless the
    header says otherwise."""
    import os
    import re
    from paper_2206_14061_gb300 import capi
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                       "lp.h")
    text = re.sub(r"/\*.*?\*/", " ", open(inc).read(), flags=re.S)
    protos = {}
    for m in re.finditer(r"(\w[\w\s\*]*?)\b(lp_\w+)\s*\(([^;{]*?)\)\s*;", text):
        ret, name, args = m.group(1).strip(), m.group(2), m.group(3).strip()
        n = 0 if args in ("", "void") else args.count(",") + 1
        protos[name] = (ret, n)
    assert set(capi._SIGS) <= set(protos), set(capi._SIGS) - set(protos)
    for name, (argtypes, restype) in capi._SIGS.items():
        ret, n = protos[name]
        assert len(argtypes) == n, (name, len(argtypes), n)
        if ret.endswith("lp_status"):
            assert restype is ctypes.c_int32, name
