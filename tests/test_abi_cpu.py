"""The C-ABI library builds, loads without a GPU and exports every entry point that
include/gde.h declares; the ctypes structures match the C layout.  No compute calls."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gde.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gde_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2410_21634_gb300 import _build
    _build.build()
    import paper_2410_21634_gb300 as gde
    return gde.load()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "gde_solve" in names and "gde_graph_create" in names
    for name in names:
        assert hasattr(lib, name), f"{name} declared in gde.h but not exported"
    import paper_2410_21634_gb300 as gde
    assert sorted(gde.EXPORTED) == sorted(set(gde.EXPORTED) & set(names))
    assert set(gde.EXPORTED) == set(names)


def test_exported_symbols_are_c_linkage(lib):
    so = lib._name
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in declared_functions():
        assert name in syms, f"{name} missing or mangled"


def test_struct_layout_matches_header(tmp_path):
    """sizeof and every field offset of each C struct the binding mirrors"""
    import paper_2410_21634_gb300 as gde
    pairs = [("gde_solve_opts", gde.SolveOpts), ("gde_stats", gde.Stats), ("gde_profile", gde.Profile),
             ("gde_tuning", gde.Tuning), ("gde_server_opts", gde.ServerOpts),
             ("gde_server_result", gde.ServerResult), ("gde_server_info_t", gde.ServerInfo)]
    lines = []
    for cname, cls in pairs:
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        for f in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {f[0]}));')
    prog = tmp_path / "layout.c"
    prog.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"gde.h\"\nint main(void) {\n"
                    + "\n".join(lines) + "\n  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = []
    for _, cls in pairs:
        want.append(ctypes.sizeof(cls))
        want += [getattr(cls, f[0]).offset for f in cls._fields_]
    assert vals == want


def test_opts_init_and_last_error_without_gpu(lib):
    import paper_2410_21634_gb300 as gde
    o = gde.SolveOpts()
    o.precision = 7
    lib.gde_solve_opts_init(ctypes.byref(o))
    assert o.precision == gde.FP64 and o.topk == 0 and o.cuda_stream is None
    assert gde.last_error() == ""


def test_missing_library_fails_loudly(tmp_path):
    import paper_2410_21634_gb300 as gde
    with pytest.raises(ImportError):
        gde.load(str(tmp_path / "nope.so"))
