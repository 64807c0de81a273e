"""CPU checks of the C-ABI boundary: libshe.so builds for sm_103a, loads
without a GPU, exports every symbol include/she.h declares, and the ctypes
structures have the C layout (offsets measured by compiling she.h with gcc).
No compute call is made here."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2406_12157_gb300 import _abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "she.h")


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_library_loads_and_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    declared = set(re.findall(r"\b(she_[a-z_0-9]+)\s*\(", open(HEADER).read()))
    assert declared, "no declarations parsed"
    assert declared == set(_abi.EXPORTS)
    for name in declared:
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    syms = set(re.findall(r" T (she_[a-z_0-9]+)$", out, re.M))
    assert declared <= syms


def test_build_targets_sm103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _c_offsets(struct, fields):
    src = "#include <stddef.h>\n#include <stdio.h>\n#include \"she.h\"\nint main(void){\n"
    src += 'printf("%%zu\\n", sizeof(%s));\n' % struct
    for f in fields:
        src += 'printf("%%zu\\n", offsetof(%s, %s));\n' % (struct, f)
    src += "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "o.c")
        exe = os.path.join(d, "o")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    return vals[0], vals[1:]


@pytest.mark.parametrize("cls,cname", [(_abi.she_params, "struct she_params"),
                                       (_abi.she_stats_out, "struct she_stats_out"),
                                       (_abi.she_sizes, "struct she_sizes")])
def test_struct_layout_matches_header(cls, cname):
    fields = [f for f, _ in cls._fields_]
    size, offs = _c_offsets(cname, fields)
    assert ctypes.sizeof(cls) == size
    for f, o in zip(fields, offs):
        assert getattr(cls, f).offset == o, f


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(_abi.LibraryMissing):
        _abi.load(str(tmp_path / "nope.so"))


def test_scheme_constants_and_marshalling():
    # the enum values the header declares, and the binding's mapping of the
    # problem's scheme (an unknown name is an error, not forward Euler)
    text = open(HEADER).read()
    assert re.search(r"SHE_FE\s*=\s*0\s*,\s*SHE_PC\s*=\s*1", text)
    assert (_abi.SHE_FE, _abi.SHE_PC) == (0, 1)
    import paper_2406_12157_gb300 as S
    import she_workloads as W
    assert S.params_from_problem(W.oracle_rod()).scheme == _abi.SHE_FE
    assert S.params_from_problem(W.oracle_rod(scheme="pc")).scheme == _abi.SHE_PC
    with pytest.raises(KeyError):
        S.params_from_problem(W.oracle_rod(scheme="rk4"))


def test_noalloc_limit_matches_header():
    # the binding's copy of the fixed scratch size of she_step_plain_noalloc
    m = re.search(r"#define\s+SHE_NOALLOC_MAX_FACES\s+\(1\s*<<\s*(\d+)\)", open(HEADER).read())
    assert m, "SHE_NOALLOC_MAX_FACES not found"
    assert _abi.SHE_NOALLOC_MAX_FACES == 1 << int(m.group(1))
