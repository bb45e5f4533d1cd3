"""The C-ABI library builds, loads without a GPU and exports every function
include/sg.h declares.  No compute call is made here."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(?:sg_status|void|int|long long|const char\s*\*)\s+(sg_\w+)\s*\(", txt):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2209_14740_gb300 import binding
    if not os.path.exists(binding.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return binding.load()


def test_header_declares_entry_points():
    names = header_functions()
    for must in ("sg_assemble", "sg_matvec", "sg_precond", "sg_gmres"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2209_14740_gb300 import binding
    names = header_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) <= set(binding.EXPORTED) | set(names)
    assert lib.sg_version() == 100


def test_invalid_arguments_rejected_without_gpu(lib):
    """Host-side validation runs before any device call."""
    import ctypes as C
    from paper_2209_14740_gb300 import binding
    h = C.c_void_p()
    assert lib.sg_assemble(None, None, C.byref(h)) == binding.SG_EINVAL
    d = binding.SgDesc()
    d.dim = 3
    assert lib.sg_assemble(C.byref(d), None, C.byref(h)) == binding.SG_EINVAL
    assert b"dim" in lib.sg_last_error()
    # a grid whose node count overflows the device's 32-bit unknown index
    d = binding.SgDesc()
    d.dim, d.nx, d.ny, d.h, d.s, d.r = 2, 50000, 50000, 1e-5, 0, 0
    assert lib.sg_assemble(C.byref(d), None, C.byref(h)) == binding.SG_EINVAL
    assert b"too large" in lib.sg_last_error()
    assert lib.sg_matvec(None, 0, None, None, None) == binding.SG_EINVAL
    assert lib.sg_gmres(None, None, None, None, None, None) == binding.SG_EINVAL


def test_header_compiles_as_plain_c(tmp_path):
    """include/sg.h is a C header: a C99 translation unit that uses its
    structs compiles with gcc -Wall -Werror."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    src = tmp_path / "use.c"
    src.write_text('#include "sg.h"\n'
                   'int main(void) { sg_desc d; sg_gmres_opts o; sg_gmres_info i; sg_tune t;\n'
                   '  (void)d; (void)o; (void)i; (void)t; return (int)sizeof(sg_tune); }\n')
    subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-c", str(src), "-o",
                    str(tmp_path / "use.o")], check=True)
