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
