"""The double-float arithmetic of the HHO_F32X2 kernels, on the GPU, against
exact rational arithmetic.

hho_f2x_check runs the kernels' pair operations (f2x.cuh) on exact input
pairs.  The double-word algorithms (TwoSum, Fast2Sum, TwoProd by FMA and the
DWPlusDW / DWTimesDW forms of Joldes, Muller and Popescu, ACM TOMS 2017)
keep errors of order u^2 (u = 2^-24) times the magnitudes involved; an
FP32-level error (order u) means an error-free transform was broken, for
instance by the compiler contracting a product into the sum after it."""
from fractions import Fraction

import numpy as np
import pytest

from tests.libutil import ensure_built

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U2 = Fraction(1, 2 ** 48)


@pytest.fixture(scope="module")
def hho():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_2505_15771_gb300 import hho
    return hho


def normalised_pairs(rng, n):
    """n pairs (hi, lo) with |lo| < ulp(hi)/2, |hi| in [1e-2, 1e2], random signs."""
    hi = (rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-2, 2, n)).astype(np.float32)
    lo = (np.spacing(np.abs(hi)) * rng.uniform(-0.49, 0.49, n)).astype(np.float32)
    return np.stack([hi, lo], axis=-1)


def exact(p):
    return Fraction(float(p[0])) + Fraction(float(p[1]))


def test_double_float_operations_meet_their_error_bounds(hho):
    rng = np.random.default_rng(20260)
    n = 3000
    x, y, z = (normalised_pairs(rng, n) for _ in range(3))
    # a third of the items nearly cancel in x + y and x - y (the bound is
    # relative to |x| + |y|, so cancellation is allowed to lose relative accuracy)
    m = n // 3
    y[:m] = -x[:m]
    y[:m, 1] = (np.spacing(np.abs(x[:m, 0])) * rng.uniform(-0.49, 0.49, m)).astype(np.float32)
    out = hho.hho_f2x_check(np.stack([x, y, z], axis=1))
    worst = [Fraction(0)] * 6
    for i in range(n):
        X, Y, Z = exact(x[i]), exact(y[i]), exact(z[i])
        refs = [X + Y, X - Y, X * Y, X * Y + Z, X / Y, ((X * Z + Y) * Z + X) * Z + Y]
        scale = [abs(X) + abs(Y), abs(X) + abs(Y), abs(X * Y), abs(X * Y) + abs(Z), abs(X / Y),
                 abs(X * Z ** 3) + abs(Y * Z ** 2) + abs(X * Z) + abs(Y)]
        for k in range(6):
            err = abs(exact(out[i, k]) - refs[k]) / scale[k] / U2
            worst[k] = max(worst[k], err)
    names = ["add", "sub", "mul", "fma", "div", "horner"]
    print({nm: float(w) for nm, w in zip(names, worst)})
    # bounds in units of u^2: a few for one operation, more for the chain of three
    bounds = [4, 4, 8, 8, 16, 32]
    for nm, w, b in zip(names, worst, bounds):
        assert w <= b, (nm, float(w))


def test_double_float_check_rejects_bad_arguments(hho):
    with pytest.raises(Exception):
        hho.hho_f2x_check(np.zeros((0, 3, 2), np.float32))
