"""The C ABI library builds, loads and exports every symbol of include/sbv.h (no GPU needed)."""
import ctypes as C
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def declared_symbols():
    text = (ROOT / "include" / "sbv.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sbv_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_12004_gb300 import build
    build.build()
    from paper_2504_12004_gb300 import _lib
    return _lib.load()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("sbv_blocking", "sbv_knn", "sbv_loglik", "sbv_predict", "sbv_create",
              "sbv_destroy", "sbv_last_error", "sbv_sync_status"):
        assert s in syms


def test_every_declared_symbol_is_exported(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_binding_signatures_cover_header(lib):
    from paper_2504_12004_gb300 import _lib
    assert set(declared_symbols()) <= set(_lib.SIGNATURES)


def test_null_context_is_rejected_without_device(lib):
    assert lib.sbv_version() >= 100
    assert lib.sbv_last_error(None) == b"null context"
    rc = lib.sbv_loglik(None, None, 0, None, 0, 0, None, None, None, None, 0, 0, 0, None, 0, 0,
                        0, None, None, None, None)
    assert rc == 1  # SBV_EINVAL
    rc = lib.sbv_blocking(None, None, 0, 0, 0, None, 0, 0, 0, None, None, None, None, None, None,
                          None)
    assert rc == 1
    v = C.c_double(0.0)
    assert lib.sbv_peak_probe(None, 0, C.byref(v)) == 1
    rc = lib.sbv_loglik_grad(None, None, 0, None, 0, 0, None, None, None, None, 0, 0, 0, None, 0,
                             0, None, None, None, None, None, None)
    assert rc == 1


def test_mle_structs_match_the_c_layout():
    """ctypes mirrors of sbv_mle_opts / sbv_mle_result: natural alignment gives
    the C layout (int32, 4 bytes padding, 3 doubles, 4 int32) and (double, 5 int32)."""
    import ctypes
    from paper_2504_12004_gb300 import _lib
    assert ctypes.sizeof(_lib.MleOpts) == 48 and _lib.MleOpts.gradient.offset == 44
    assert ctypes.sizeof(_lib.MleResult) == 32 and _lib.MleResult.grad_evals.offset == 24
    o = _lib.mle_opts(gradient="analytic", precision="fp64")
    assert o.gradient == 1 and o.precision == 0


def test_option_structs_match_a_c_compilers_layout(tmp_path):
    """sizeof and offsetof of the option and result structs, printed by a C
    program compiled against include/sbv.h, equal the ctypes mirrors'."""
    import ctypes
    import subprocess
    from paper_2504_12004_gb300 import _lib
    mirrors = {"sbv_mle_opts": _lib.MleOpts, "sbv_mle_result": _lib.MleResult,
               "sbv_surrogate_opts": _lib.SurrogateOpts}
    lines = []
    for cname, py in mirrors.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"sbv.h\"\n"
                   "int main(void) {\n" + "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", str(ROOT / "include"), str(src), "-o", str(exe)],
                   check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n"):
        if line:
            c, f, v = line.split()
            got[(c, f)] = int(v)
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_product_path_does_not_import_oracle():
    pkg = ROOT / "paper_2504_12004_gb300"
    for f in list(pkg.rglob("*.py")) + list(pkg.rglob("*.cu")) + list(pkg.rglob("*.cuh")):
        src = f.read_text()
        assert "import oracle" not in src and "from oracle" not in src, f
        assert "_work/" not in src, f
