"""CPU checks of the C ABI: the library loads, exports every declared entry
point, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_0811_1081_gb300 import buildlib as b

    b.build()
    import paper_0811_1081_gb300 as gp

    return gp.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gspca.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gspca_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "gspca_fit" in names and "gspca_create" in names and "gspca_fit_batched" in names
    for n in names:
        assert hasattr(lib, n), n


def test_python_binding_names_match_header():
    import paper_0811_1081_gb300 as gp

    for n in declared_functions():
        assert n in gp.EXPORTS, n
        assert hasattr(gp, n), n


def test_status_strings(lib):
    import paper_0811_1081_gb300 as gp

    for s in range(8):
        assert isinstance(gp.status_string(s), str) and gp.status_string(s)
    assert gp.status_string(99) == "unknown status"


def test_invalid_arguments_need_no_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.gspca_create(None, 0, 10, 10, 2, 0) == 1
    assert lib.gspca_create(ctypes.byref(h), 0, 0, 10, 2, 0) == 1
    assert lib.gspca_create(ctypes.byref(h), 0, 10, 10, 11, 0) == 1
    assert lib.gspca_create(ctypes.byref(h), 0, 10, 10, 2, 7) == 1
    assert lib.gspca_create(ctypes.byref(h), 0, 10, 10 ** 6, 2, 0) == 7  # beyond the column limit
    assert lib.gspca_fit(None, None, None, 0, 1, 1, 1, 1, 1e-6, 10, 1, None, None, None, None, None,
                         None) == 1
    assert lib.gspca_destroy(None) == 0


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import importlib

    import paper_0811_1081_gb300 as gp
    import paper_0811_1081_gb300.buildlib as b

    monkeypatch.setattr(gp, "_lib", None)
    monkeypatch.setattr(gp, "LIB", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError):
        gp.load()
    importlib.reload(b)


def header_struct_fields(name):
    """Field names, in order, of `typedef struct { ... } name;` in gspca.h."""
    src = open(os.path.join(ROOT, "include", "gspca.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    bodies = {n: b for b, n in re.findall(r"typedef struct\s*\{([^{}]*)\}\s*(\w+)\s*;", src)}
    assert name in bodies, name
    fields = []
    for decl in bodies[name].split(";"):
        decl = decl.strip()
        if not decl:
            continue
        # "int M, N, K" / "float *T, *P" / "const int *iters_lock"
        head, *rest = decl.split(",")
        names = [re.findall(r"(\w+)\s*$", head)[0]] + [re.findall(r"(\w+)\s*$", r)[0] for r in rest]
        fields += names
    return fields


@pytest.mark.parametrize("cname,pyname", [("gspca_opts", "Opts"), ("gspca_info", "Info"),
                                          ("gspca_problem", "Problem")])
def test_ctypes_structs_match_header(cname, pyname):
    """The binding's ctypes structures list the header's fields in the header's order."""
    import paper_0811_1081_gb300 as gp

    want = header_struct_fields(cname)
    got = [f.rstrip("_") for f, _ in getattr(gp, pyname)._fields_]
    assert got == want, (cname, got, want)


def _c_layout(struct, fields):
    """sizeof and offsetof of a header struct, from a C program compiled with gcc."""
    import shutil
    import subprocess
    import tempfile

    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gspca.h"', "int main(void) {",
             f'  printf("%zu\\n", sizeof({struct}));']
    lines += [f'  printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return int(out[0]), [int(v) for v in out[1:]]


@pytest.mark.parametrize("struct,pyname,rename", [("gspca_opts", "Opts", {}), ("gspca_info", "Info", {}),
                                                  ("gspca_problem", "Problem", {"lambda_": "lambda"}),
                                                  ("gspca_warm_start", "WarmStartC", {})])
def test_binding_structs_match_the_header_layout(struct, pyname, rename):
    """The ctypes mirrors of the ABI structs have the header's size, field order and offsets."""
    import paper_0811_1081_gb300 as gp

    cls = getattr(gp, pyname)
    names = [rename.get(n, n) for n, _ in cls._fields_]
    size, offs = _c_layout(struct, names)
    assert ctypes.sizeof(cls) == size
    assert [getattr(cls, n).offset for n, _ in cls._fields_] == offs


def test_every_cuda_source_is_built():
    """Every translation unit under csrc/ is in the build list (a unit left out would leave its
    kernel instantiations undefined only at load time)."""
    from paper_0811_1081_gb300 import buildlib as b

    units = sorted(f for f in os.listdir(b.CSRC) if f.endswith(".cu"))
    assert sorted(b.SOURCES) == units
