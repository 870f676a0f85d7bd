"""The C-ABI library builds, loads and exports every entry point of include/gato.h.

No compute call is made here (this runs without a GPU).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "gato.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gato_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_07625_gb300 import build

    build.build_library()
    from paper_2510_07625_gb300 import gato

    return gato.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gato_create_batch", "gato_solve", "gato_step", "gato_sync",
                     "gato_destroy_batch", "gato_solve_plain"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    from paper_2510_07625_gb300 import gato

    assert set(declared_functions()) == set(gato.EXPORTED)


def test_defaults_and_status_strings(lib):
    from paper_2510_07625_gb300 import gato

    p = gato.gato_default_params()
    assert p.mu == 10.0 and p.beta == 2.0 and p.n_alpha == 8 and p.pcg_max_iter == 1000
    assert abs(p.pcg_eps - 1e-6) < 1e-12 and p.precond == gato.PRECOND_STAIR and p.kkt_tol == 0.0
    assert gato.gato_status_string(gato.GATO_E_INVALID) == "invalid argument"


def test_create_batch_rejects_bad_descriptors_before_touching_the_gpu(lib):
    from paper_2510_07625_gb300 import gato, inputs

    md = (gato.ModelDesc * 1)(gato.model_desc(inputs.arm7()))
    bad = gato.BatchDesc(0, 32, 1, ctypes.cast(md, ctypes.POINTER(gato.ModelDesc)),
                         gato.gato_default_params())
    with pytest.raises(gato.GatoError) as e:
        gato.gato_create_batch(bad)
    assert e.value.status == gato.GATO_E_INVALID
    bad = gato.BatchDesc(4, 1000, 1, ctypes.cast(md, ctypes.POINTER(gato.ModelDesc)),
                         gato.gato_default_params())
    with pytest.raises(gato.GatoError):
        gato.gato_create_batch(bad)
    m = gato.model_desc(inputs.arm7())
    m.mass[2] = -1.0
    md2 = (gato.ModelDesc * 1)(m)
    bad = gato.BatchDesc(4, 32, 1, ctypes.cast(md2, ctypes.POINTER(gato.ModelDesc)),
                         gato.gato_default_params())
    with pytest.raises(gato.GatoError):
        gato.gato_create_batch(bad)


def test_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    from paper_2510_07625_gb300 import gato

    monkeypatch.setattr(gato, "_lib", None)
    monkeypatch.setattr(gato, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        gato.load()


STRUCTS = {  # ctypes mirror in the binding -> C typedef in include/gato.h
    "ModelDesc": "gato_model_desc", "SolverParams": "gato_solver_params",
    "BatchDesc": "gato_batch_desc", "Problem": "gato_problem", "LaunchConfig": "gato_launch_config",
    "LaunchInfo": "gato_launch_info", "Result": "gato_result", "ServerDesc": "gato_server_desc",
    "Reply": "gato_reply", "DriveStats": "gato_drive_stats", "ServerStats": "gato_server_stats",
}


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes struct of the binding has the size and field offsets that a
    C compiler gives the header's typedef (gcc on this host)."""
    import shutil
    import subprocess

    from paper_2510_07625_gb300 import gato

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gato.h"', "int main(void) {"]
    want = {}
    for py, c in STRUCTS.items():
        cls = getattr(gato, py)
        lines.append(f'  printf("{py} size %zu\\n", sizeof({c}));')
        want[f"{py} size"] = ctypes.sizeof(cls)
        for name, _ in cls._fields_:
            cname = "lambda" if (py == "Problem" and name == "lam") else name
            lines.append(f'  printf("{py}.{name} %zu\\n", offsetof({c}, {cname}));')
            want[f"{py}.{name}"] = getattr(cls, name).offset
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        key, val = line.rsplit(" ", 1)
        got[key] = int(val)
    assert got == want
