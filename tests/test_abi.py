"""The C-ABI library builds, loads without a GPU, and exports every entry point
declared in include/*.h; the Python binding knows each of them."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(mgk?_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_headers_declare_the_boundary():
    names = declared_functions()
    for must in ("mg_create", "mg_setup_transform", "mg_solve", "mg_batch_solve",
                 "mg_serve_submit", "mg_serve_poll", "mg_server_start", "mg_server_stop"):
        assert must in names


def test_library_exports_every_declared_symbol(libmg):
    import ctypes
    h = ctypes.CDLL(libmg.LIB_PATH)
    missing = [n for n in sorted(declared_functions()) if not hasattr(h, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libmg):
    assert declared_functions() <= set(libmg.exported_names())
    libmg.lib()  # loads and binds every signature without touching the GPU


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2602_01888_gb300 import mg
    monkeypatch.setattr(mg, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(mg, "_lib", None)
    import pytest
    with pytest.raises(RuntimeError):
        mg.lib()


def test_struct_layouts_match_header(libmg):
    import ctypes
    # mg_grid_desc: 2 ints, 4 doubles, 1 int (+ padding)
    assert ctypes.sizeof(libmg.mg_grid_desc) == 48
    assert ctypes.sizeof(libmg.mg_map_desc) == 4 + 4 + 32 + 16 + 16
    assert ctypes.sizeof(libmg.mg_solve_opts) == 5 * 4 + 4 + 16 + 12 + 4
    assert ctypes.sizeof(libmg.mg_solve_stats) == 8 + 3 * 8 + 256 * 8 + 8


def test_kernel_operator_struct_matches_the_c_compiler(libmg, tmp_path):
    """mgk_op_f64 / mgk_op_f32 as ctypes lays them out equal the C compiler's layout of
    mg_kernels.h (size and the offset of every field)."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f for f, _ in libmg.mgk_op_f64._fields_]
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mg_kernels.h"', "int main(void) {"]
    for t in ("mgk_op_f64", "mgk_op_f32"):
        lines.append(f'  printf("{t} size %zu\\n", sizeof({t}));')
        for f in fields:
            lines.append(f'  printf("{t} {f} %zu\\n", offsetof({t}, {f}));')
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        t, f, v = line.split()
        got[(t, f)] = int(v)
    for t, cls in (("mgk_op_f64", libmg.mgk_op_f64), ("mgk_op_f32", libmg.mgk_op_f32)):
        assert got[(t, "size")] == ctypes.sizeof(cls)
        for f in fields:
            assert got[(t, f)] == getattr(cls, f).offset, (t, f)


def test_map_classification_for_the_five_point_form(libmg):
    """mg_map_five_point (host logic, no GPU): maps whose J^T J is diagonal (Eq. 13 vanishes
    identically) are handled as 5-point operators; maps with a cross term are not."""
    from paper_2602_01888_gb300 import inputs as I
    yes = [I.MapSpec("identity"), I.MapSpec("polar"), I.MapSpec("sinh", (5.0, 0.6)),
           I.MapSpec("affine", (1.1, 0.0, 0.0, 0.9))]
    no = [I.MapSpec("sine_warp", (0.1,)), I.MapSpec("affine", (1.1, 0.2, -0.1, 0.9)),
          I.MapSpec("affine", (1.0, 0.0, 0.3, 1.0))]
    assert all(libmg.map_five_point(m) for m in yes)
    assert not any(libmg.map_five_point(m) for m in no)
    assert libmg.lib().mg_map_five_point(None) == 0
    assert libmg.lib().mg_problem_five_point(None) == -1


def test_no_oracle_on_the_product_path():
    """The package (product path) never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2602_01888_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "mg_oracle" not in txt, f


def test_kernel_entries_refuse_bad_arguments_before_any_launch(libmg):
    """Argument checks of the even-row restriction and the one-pass 5-point assembly (host
    logic, no GPU): missing arrays, even grid sizes, a 9-point operator for the 5-point pass,
    a non-positive spacing and an FP32 copy of other sizes all return 1 before anything is
    launched.  The pointers below are never dereferenced."""
    import ctypes as C
    lib = libmg.lib()
    fake = 4096

    def op(cls, nx, ny, five):
        s = cls()
        s.nx, s.ny, s.periodic, s.pitch, s.five_point = nx, ny, 0, nx + 3, five
        for f in ("cE", "cN", "cNE", "cNW", "diag", "dinv"):
            setattr(s, f, fake)
        return s

    a = op(libmg.mgk_op_f64, 65, 33, 1)
    a32 = op(libmg.mgk_op_f32, 65, 33, 1)
    for name, A in (("mgk_resid_restrict_even_f64", a), ("mgk_resid_restrict_even_f32", a32)):
        f = getattr(lib, name)
        assert f(None, fake, fake, fake, 40, None) == 1
        assert f(C.byref(A), None, fake, fake, 40, None) == 1
        assert f(C.byref(A), fake, fake, None, 40, None) == 1
        assert f(C.byref(A), fake, fake, fake, 32, None) == 1  # coarse pitch below the 33 coarse columns
    even = op(libmg.mgk_op_f64, 64, 33, 1)
    assert lib.mgk_resid_restrict_even_f64(C.byref(even), fake, fake, fake, 40, None) == 1
    nine = op(libmg.mgk_op_f64, 65, 33, 0)
    other = op(libmg.mgk_op_f32, 65, 17, 1)
    f = lib.mgk_assemble_five
    assert f(C.byref(nine), None, 0.1, 0.1, fake, fake, None) == 1
    assert f(C.byref(a), None, 0.0, 0.1, fake, fake, None) == 1
    assert f(C.byref(a), None, 0.1, 0.1, None, fake, None) == 1
    assert f(C.byref(a), C.byref(other), 0.1, 0.1, fake, fake, None) == 1
