"""The functions of the paper's Python module (usage section) under the same names:
combinatoric, glynn, ryser and opt, with the _square / _rectangular variants, each
taking one 2-D array and returning a Python number."""
import numpy as np
import pytest

from gpu_util import device

pytestmark = pytest.mark.gpu

WORKED = [[1, 2, 3], [4, 5, 6], [7, 8, 9]]  # the usage section's example, per = 450


@pytest.fixture(scope="module")
def pkg():
    device()
    import paper_2510_03421_gb300 as p
    return p


def test_worked_example_integer_float_complex(pkg):
    for name in ("combinatoric", "glynn", "ryser", "opt", "glynn_square", "opt_square"):
        f = getattr(pkg, name)
        v = f(np.array(WORKED))
        assert v == 450 and isinstance(v, int), name
        assert f(np.array(WORKED, dtype=np.float64)) == 450.0, name
        c = f(np.array(WORKED, dtype=np.complex128) * (1 + 1j))
        assert isinstance(c, complex) and abs(c - 450 * (1 + 1j) ** 3) <= 1e-12 * abs(c), name


def test_rectangular_variants_and_shape_checks(pkg):
    ones = np.ones((2, 4))
    for name in ("combinatoric", "glynn", "ryser", "opt"):
        assert getattr(pkg, name + "_rectangular")(ones) == 12.0  # 4! / 2!
        with pytest.raises(ValueError):
            getattr(pkg, name + "_square")(ones)
        with pytest.raises(ValueError):
            getattr(pkg, name + "_rectangular")(np.ones((3, 3)))


def test_device_tensor_input(pkg):
    import torch
    A = torch.tensor(WORKED, dtype=torch.float64, device="cuda:0")
    assert pkg.opt(A) == 450.0
    assert pkg.glynn(A.T.contiguous()) == 450.0  # per(A^T) = per(A)


def test_cpp_interface_runs(tmp_path):
    # include/permanent.hpp: the paper's C++ shapes permanent::fn<Type, IntType>(m, n, ptr)
    import os
    import shutil
    import subprocess
    device()
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    from paper_2510_03421_gb300 import _build
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    exe = tmp_path / "paper_api_check"
    subprocess.check_call([gxx, "-std=c++17", "-O1", "-I", os.path.join(root, "include"),
                           os.path.join(root, "tests", "paper_api_check.cpp"), _build.build(), "-o", str(exe)])
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0, run.stdout + run.stderr
    lines = run.stdout.strip().splitlines()
    assert len(lines) == 13 and all(l.startswith("ok ") for l in lines), run.stdout
