"""Host-side checks of the C ABI that need no GPU: the library builds, loads and
exports every entry point declared in include/perm.h; argument errors are
reported synchronously."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_03421_gb300 import _build, capi
    _build.build()
    return capi.lib()


def declared_functions():
    import glob
    text = "".join(open(p).read() for p in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(perm_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("perm_glynn", "perm_ryser", "perm_combinatoric", "perm_auto", "perm_batched",
                     "perm_glynn_partial", "perm_create", "perm_destroy", "perm_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings_and_version(lib):
    from paper_2510_03421_gb300 import capi
    seen = set()
    for code in range(7):
        s = capi.status_string(code)
        assert s and s not in seen
        seen.add(s)
    assert capi.status_string(99) == "unknown status"
    assert lib.perm_version() >= 100


def test_null_handle_is_rejected(lib):
    from paper_2510_03421_gb300 import capi
    out = (ctypes.c_double * 2)()
    a = (ctypes.c_double * 4)()
    for name in ("perm_glynn", "perm_ryser", "perm_combinatoric", "perm_auto"):
        rc = getattr(lib, name)(None, ctypes.addressof(a), 2, 2, 2, capi.PERM_F64, ctypes.addressof(out), None, None)
        assert rc == capi.PERM_EINVAL, name
    rc = lib.perm_glynn_partial(None, ctypes.addressof(a), 2, 2, 2, capi.PERM_F64, 0, 2, ctypes.addressof(out), None,
                                None)
    assert rc == capi.PERM_EINVAL
    occ = (ctypes.c_uint64 * 1)(3)
    rc = lib.perm_sbp(None, ctypes.addressof(a), 2, 2, 2, capi.PERM_F64, ctypes.addressof(occ), 1,
                      ctypes.addressof(out), None, None)
    assert rc == capi.PERM_EINVAL
    rc = lib.perm_cauchy(None, ctypes.addressof(a), ctypes.addressof(a), 2, 1, ctypes.addressof(out), None, None)
    assert rc == capi.PERM_EINVAL
    assert lib.perm_destroy(None) == capi.PERM_EINVAL
    assert lib.perm_create(None, 0) == capi.PERM_EINVAL


def test_create_without_gpu_reports_cuda_error(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2510_03421_gb300 import capi
    h = ctypes.c_void_p()
    assert lib.perm_create(ctypes.byref(h), 0) == capi.PERM_ECUDA
    assert not h.value


def test_opts_struct_layout_matches_header():
    from paper_2510_03421_gb300 import capi
    # six int32, one uint64, one pointer
    assert ctypes.sizeof(capi.perm_opts) == 6 * 4 + 8 + 8
    assert capi.perm_opts.max_terms.offset == 24 and capi.perm_opts.err.offset == 32


def test_damaged_cost_model_file_is_refused(tmp_path):
    # a damaged or mismatched model file raises instead of installing garbage; perm_auto
    # then keeps its current model (or the built-in rule)
    import numpy as np

    from paper_2510_03421_gb300 import costmodel
    w, dims, meta = costmodel.load()  # the shipped model loads
    assert dims[0] == 12 and dims[2] == 8 and np.all(np.isfinite(w))
    bad = tmp_path / "bad.npz"
    bad.write_bytes(b"not an npz archive")
    with pytest.raises(ValueError):
        costmodel.load(str(bad))
    nan = tmp_path / "nan.npz"
    w2 = w.copy()
    w2[5] = np.nan
    np.savez(nan, weights=w2, dims=np.array(dims), meta=np.array("{}"))
    with pytest.raises(ValueError):
        costmodel.load(str(nan))
    short = tmp_path / "short.npz"
    np.savez(short, weights=w[:-3], dims=np.array(dims), meta=np.array("{}"))
    with pytest.raises(ValueError):
        costmodel.load(str(short))


def test_paper_function_names_resolve_without_a_gpu():
    import paper_2510_03421_gb300 as p
    for base in ("combinatoric", "glynn", "ryser", "opt"):
        for suffix in ("", "_square", "_rectangular"):
            f = getattr(p, base + suffix)
            assert callable(f) and f.__name__ == base + suffix
    with pytest.raises(AttributeError):
        getattr(p, "glynn_triangular")


def test_cpp_interface_compiles_and_links(tmp_path):
    # include/permanent.hpp (the paper's C++ function shapes over the C ABI) with every
    # element type the check program uses; linked against the built library
    import shutil
    import subprocess
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    from paper_2510_03421_gb300 import _build
    lib = _build.build()
    exe = tmp_path / "paper_api_check"
    subprocess.check_call([gxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "paper_api_check.cpp"), lib, "-o", str(exe)])
    assert exe.exists()


def test_public_headers_compile_cleanly():
    # the C headers as C11 and the C++ interface as C++17, warnings as errors
    import glob
    import shutil
    import subprocess
    gcc, gxx = shutil.which("gcc"), shutil.which("g++")
    if gcc is None or gxx is None:
        pytest.skip("no gcc / g++")
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        subprocess.check_call([gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-x", "c", h])
    subprocess.check_call([gxx, "-std=c++17", "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-I",
                           os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "paper_api_check.cpp")])


def test_null_handle_cauchy_sbp(lib):
    from paper_2510_03421_gb300 import capi
    a = (ctypes.c_double * 4)()
    occ = (ctypes.c_uint64 * 1)(3)
    rc = lib.perm_cauchy_sbp(None, ctypes.addressof(a), 2, ctypes.addressof(a), 2, ctypes.addressof(occ), 1,
                             ctypes.addressof(a), None, None)
    assert rc == capi.PERM_EINVAL
