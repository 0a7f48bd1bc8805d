"""The C ABI without a GPU: the header compiles as C and C++, the library
exports every function the header declares, the binding's structs match the
C layouts, and calls fail loudly (no CPU fallback) when no device exists."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2112_06300_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ccd.h")


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ccd_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_compiles_as_c_and_cpp():
    d = tempfile.mkdtemp()
    src = os.path.join(d, "t.c")
    open(src, "w").write('#include "ccd.h"\nint main(void){ccd_opts o; ccd_default_opts(&o); return 0;}\n')
    for cc, ext in (("gcc", "c"), ("g++", "cpp")):
        s = os.path.join(d, "t." + ext)
        os.replace(src, s) if ext == "c" else open(s, "w").write(open(os.path.join(d, "t.c")).read())
        r = subprocess.run([cc, "-fsyntax-only", "-Wall", "-Werror", "-I", os.path.dirname(HEADER), s],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_every_declared_function_is_exported(libpath):
    names = declared_functions()
    assert {"ccd_create", "ccd_destroy", "ccd_broad", "ccd_narrow", "ccd_step",
            "ccd_get_status", "ccd_status_str", "ccd_measure_fp64_peak"} <= set(names)
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for n in names:
        getattr(lib, n)


def test_struct_layouts_match_binding():
    """Size and every field offset of each struct the binding mirrors."""
    from paper_2112_06300_gb300 import ccd
    d = tempfile.mkdtemp()
    src = os.path.join(d, "s.c")
    structs = (ccd.ccd_opts, ccd.ccd_stats, ccd.ccd_tuning, ccd.ccd_memory_model, ccd.ccd_server_opts,
               ccd.ccd_server_stats)
    lines = []
    for st in structs:
        lines.append(f'printf("%zu\\n", sizeof({st.__name__}));')
        for name, _ in st._fields_:
            lines.append(f'printf("%zu\\n", offsetof({st.__name__}, {name}));')
    open(src, "w").write('#include <stdio.h>\n#include <stddef.h>\n#include "ccd.h"\nint main(void){'
                         + "".join(lines) + "return 0;}\n")
    exe = os.path.join(d, "s")
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), src, "-o", exe], check=True)
    vals = iter(map(int, subprocess.run([exe], capture_output=True, text=True).stdout.split()))
    for st in structs:
        assert next(vals) == ctypes.sizeof(st), st.__name__
        for name, _ in st._fields_:
            assert next(vals) == getattr(st, name).offset, (st.__name__, name)


def test_status_strings_and_defaults():
    from paper_2112_06300_gb300 import ccd
    assert ccd.ccd_status_str(ccd.CCD_OK) == "ok"
    assert "too small" in ccd.ccd_status_str(ccd.CCD_ETRUNC)
    o = ccd.ccd_default_opts()
    assert o.delta == 1e-6 and o.max_iter == 10 ** 6 and o.min_sep == 0.0


def test_calls_fail_loudly_without_a_device():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2112_06300_gb300 import ccd
    with pytest.raises(ccd.CCDError):
        ccd.ccd_create(None, 0)
    with pytest.raises(ccd.CCDError):
        ccd.ccd_measure_fp64_peak(0)
