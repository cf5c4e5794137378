"""The C-ABI library builds, loads and exports every symbol include/mg.h declares.
No compute call is made (no GPU needed)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mg.h")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1303_0008_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared()
    for required in ["mg_create_grid", "mg_set_density", "mg_solve", "mg_get_field",
                     "mg_get_force", "mg_destroy_grid", "mg_last_error", "mg_add_patches",
                     "mg_set_field", "mg_create_batch", "mg_solve_batch"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (mg_[a-z_0-9]+)\b", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing


def test_ctypes_binding_covers_the_header(libpath):
    from paper_1303_0008_gb300 import mg
    L = mg.lib()
    for name in declared():
        assert hasattr(L, name)
    assert set(mg.exported_symbols()) == set(declared())


def test_binding_rejects_bad_arguments_without_gpu(libpath):
    from paper_1303_0008_gb300 import mg
    with pytest.raises(mg.MGError) as e:
        mg.mg_create_grid(7)
    assert e.value.status == mg.MG_EINVAL
    with pytest.raises(mg.MGError) as e:
        mg.mg_create_grid(36)          # coarsest side 18 > 16
    assert e.value.status == mg.MG_EINVAL
    with pytest.raises(mg.MGError):
        mg.options(nu_pre=0, nu_post=0) and mg.mg_create_grid(8, mg.options(nu_pre=0, nu_post=0))
    for bad in (dict(time_kernels=3), dict(time_kernels=-1), dict(omega=1.5), dict(coarse_sweeps=0)):
        with pytest.raises(mg.MGError) as e:
            mg.mg_create_grid(8, mg.options(**bad))
        assert e.value.status == mg.MG_EINVAL, bad


def _c_layout(struct, fields, tmp_path):
    """sizeof and offsetof of a header struct, from a C program built with the
    host compiler against include/mg.h."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mg.h"', 'int main(void) {',
             f'  printf("%zu\\n", sizeof({struct}));']
    lines += [f'  printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    lines += ['  return 0;', '}']
    src = tmp_path / f"{struct}.c"
    exe = tmp_path / f"{struct}.out"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    return int(out[0]), [int(x) for x in out[1:]]


@pytest.mark.parametrize("name", ["mg_options", "mg_solve_stats"])
def test_binding_structs_match_the_header_layout(name, tmp_path):
    """The ctypes mirrors of the header's option and statistics structs have the
    header's size and every field at the header's offset."""
    from paper_1303_0008_gb300 import mg
    cls = getattr(mg, name)
    fields = [f for f, _ in cls._fields_]
    # Python keywords carry a trailing underscore in the binding (lambda_)
    size, offsets = _c_layout(name, [f.rstrip("_") for f in fields], tmp_path)
    assert ctypes_sizeof(cls) == size
    assert [getattr(cls, f).offset for f in fields] == offsets


def ctypes_sizeof(cls):
    import ctypes
    return ctypes.sizeof(cls)


def test_default_options_are_the_documented_ones(libpath):
    """mg_default_options (a host call) fills the documented defaults."""
    from paper_1303_0008_gb300 import mg
    o = mg.options()
    assert (o.prec, o.nu_pre, o.nu_post) == (mg.MG_FP64, 2, 2)
    assert (o.coarse_sweeps, o.coarse_drop, o.time_kernels) == (4, 1e-2, 0)
    assert o.omega == 1.0 and abs(o.w - 1.0 / 3.0) < 1e-15


def test_product_package_never_reaches_the_oracle():
    """The product path (the package's modules and its CUDA sources) imports, loads
    or builds nothing from oracle/: the oracle is test infrastructure only, and the
    binding fails loudly instead of falling back to it."""
    import ast
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_1303_0008_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for fn in files:
            path = os.path.join(dirpath, fn)
            if fn.endswith(".py"):
                tree = ast.parse(open(path).read())
                for node in ast.walk(tree):
                    if isinstance(node, ast.Import):
                        assert not any(a.name.split(".")[0] == "oracle" for a in node.names), path
                    if isinstance(node, ast.ImportFrom):
                        assert (node.module or "").split(".")[0] != "oracle", path
                    if isinstance(node, ast.Constant) and isinstance(node.value, str):
                        assert "liborc" not in node.value and "mg_oracle" not in node.value, path
            elif fn.endswith((".cu", ".cuh", ".h")):
                text = open(path).read()
                assert "oracle/" not in text and "mg_oracle" not in text, path
