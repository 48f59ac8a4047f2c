"""The C-ABI library builds, loads without a GPU and exports every declared
symbol; the binding's structs and constants match the header as the C compiler
lays it out."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(sbci_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_2603_06101_gb300 import build, sbci

    if not os.path.exists(sbci.LIB_PATH):
        build.build()
    return sbci.LIB_PATH


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert len(names) >= 13
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(lib_path):
    from paper_2603_06101_gb300 import sbci

    assert set(sbci.EXPORTS) <= _declared()


def test_host_only_calls_without_gpu(lib_path):
    """Entry points that need no device work behave on a CPU-only host."""
    from paper_2603_06101_gb300 import sbci

    lib = sbci.load()
    p = sbci.params()
    assert p.eps0 == 1e-10 and p.r0 == 1e-5 and p.max_cycle == 20
    assert lib.sbci_params_init(None) == sbci.SBCI_ERR_INVALID
    assert b"NULL" in lib.sbci_last_error()
    # argument validation happens before any CUDA call
    h = ctypes.c_void_p()
    assert lib.sbci_init_integrals(ctypes.byref(h), 17, 1, 1, None, None, 0.0, None) == sbci.SBCI_ERR_INVALID
    import numpy as np

    h1 = np.zeros((2, 2))
    eri = np.zeros((2, 2, 2, 2))
    h1[0, 0] = float("nan")
    st = lib.sbci_init_integrals(ctypes.byref(h), 2, 1, 1, h1.ctypes.data_as(ctypes.c_void_p),
                                 eri.ctypes.data_as(ctypes.c_void_p), 0.0, None)
    assert st == sbci.SBCI_ERR_NUMERIC
    h1[0, 0] = 0.0
    h1[0, 1] = 1.0  # not symmetric
    st = lib.sbci_init_integrals(ctypes.byref(h), 2, 1, 1, h1.ctypes.data_as(ctypes.c_void_p),
                                 eri.ctypes.data_as(ctypes.c_void_p), 0.0, None)
    assert st == sbci.SBCI_ERR_INVALID


_STRUCTS = ["sbci_params", "sbci_report", "sbci_trace_record", "sbci_kernel_stat", "sbci_batch_class"]
_CONSTS = ["SBCI_OK", "SBCI_ERR_INVALID", "SBCI_ERR_NOMEM", "SBCI_ERR_CUDA", "SBCI_ERR_NUMERIC",
           "SBCI_ERR_NOT_CONVERGED", "SBCI_ERR_TIMEOUT", "SBCI_ERR_CANCELLED", "SBCI_FP64", "SBCI_TF32X3",
           "SBCI_BF16X3", "SBCI_FP32"]


def test_binding_layouts_match_the_c_compiler(tmp_path):
    """Every struct of the binding has the C compiler's size and field offsets,
    and every constant its value (a layout mismatch would corrupt arguments
    silently)."""
    import shutil
    import subprocess

    from paper_2603_06101_gb300 import sbci

    if shutil.which("gcc") is None:
        pytest.skip("gcc missing")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "sbci.h"', "int main(void) {"]
    for s in _STRUCTS:
        lines.append(f'  printf("{s} size %zu\\n", sizeof({s}));')
        for name, _ in getattr(sbci, s)._fields_:
            lines.append(f'  printf("{s} {name} %zu\\n", offsetof({s}, {name}));')
    for k in _CONSTS:
        lines.append(f'  printf("const {k} %d\\n", (int){k});')
    lines.append('  printf("const NOALLOC %u\\n", (unsigned)SBCI_NOALLOC_SCRATCH_BYTES);')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in filter(None, out):
        a, b, v = line.split()
        if a == "const":
            want = sbci.NOALLOC_SCRATCH_BYTES if b == "NOALLOC" else getattr(sbci, b)
            assert int(v) == want, line
        elif b == "size":
            assert ctypes.sizeof(getattr(sbci, a)) == int(v), line
        else:
            assert getattr(getattr(sbci, a), b).offset == int(v), line
        seen += 1
    assert seen == len(_CONSTS) + 1 + sum(1 + len(getattr(sbci, s)._fields_) for s in _STRUCTS)



def _prototypes():
    src = open(os.path.join(ROOT, "include", "sbci.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"#[^\n]*", "", src)
    out = {}
    for ret, name, args in re.findall(r"([A-Za-z_][\w \*]*?)\s*\b(sbci_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", src):
        args = [a.strip() for a in args.split(",") if a.strip() and a.strip() != "void"]
        out[name] = (" ".join(ret.split()), args)
    return out


def _kind_c(decl):
    if "*" in decl:
        return "ptr"
    words = decl.replace("const ", "").split()
    base = " ".join(words[:-1])
    return {"int": "int", "double": "double", "long long": "longlong", "size_t": "size_t"}[base]


def _kind_ctypes(t):
    if t is ctypes.c_void_p or t is ctypes.c_char_p or (isinstance(t, type) and issubclass(t, ctypes._Pointer)):
        return "ptr"
    if t is ctypes.c_size_t:
        return "size_t"
    return {ctypes.c_int: "int", ctypes.c_double: "double", ctypes.c_longlong: "longlong"}[t]


def test_binding_prototypes_match_the_header(lib_path):
    """Argument count and kind (pointer, int, double, long long, size_t) and the
    return type of every bound entry point against its header prototype."""
    from paper_2603_06101_gb300 import sbci

    lib = sbci.load()
    protos = _prototypes()
    for name in sbci.EXPORTS:
        ret, args = protos[name]
        fn = getattr(lib, name)
        assert [_kind_ctypes(t) for t in fn.argtypes] == [_kind_c(a) for a in args], name
        want_ret = {"sbci_status": ctypes.c_int, "void": None, "const char *": ctypes.c_char_p}[ret]
        assert fn.restype is want_ret, (name, ret)


def test_sigma_noalloc_wrapper_rejects_bad_tensors_before_the_library():
    """The binding checks dtype, size, contiguity and device of c and out
    before any call into the library (a wrong tensor would let the kernels read
    or write past the caller's buffer)."""
    torch = pytest.importorskip("torch")
    from paper_2603_06101_gb300 import sbci

    class FakeLib:
        calls = 0

        def sbci_sigma_noalloc(self, *a):
            FakeLib.calls += 1
            return 0

    ctx = object.__new__(sbci.Context)
    ctx._lib = FakeLib()
    ctx._h = None
    ctx.ndet = 16
    good = torch.zeros(16, dtype=torch.float64)
    cases = [
        (torch.zeros(16, dtype=torch.float32), good, TypeError),   # wrong dtype of c
        (good, torch.zeros(16, dtype=torch.float32), TypeError),   # wrong dtype of out
        (torch.zeros(15, dtype=torch.float64), good, ValueError),  # short c
        (good, torch.zeros(17, dtype=torch.float64), ValueError),  # long out
        (torch.zeros(32, dtype=torch.float64)[::2], good, ValueError),  # not contiguous
        (good, good.clone(), ValueError),                          # host tensors
        (good.numpy(), good, TypeError),                           # not a tensor
    ]
    for c, out, exc in cases:
        with pytest.raises(exc):
            ctx.sigma_noalloc(c, out)
    assert FakeLib.calls == 0
    ctx._h = None
