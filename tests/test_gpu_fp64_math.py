"""The integrator's FP64 reciprocal, reciprocal square root and square root
(Newton-refined hardware approximations) against references in extended
precision: a few units in the last place at most, over the range the
right-hand side meets (radii 1e-3 .. 1e8, their squares and products)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1706_07062_gb300 import kerr as K  # noqa: E402

pytestmark = pytest.mark.gpu


def ulp_err(got, want_ld):
    """|got - want| in units of the last place of the double nearest want."""
    w = want_ld.astype(np.float64)
    return np.abs((got.astype(np.longdouble) - want_ld) / np.spacing(np.abs(w)).astype(np.longdouble))


def test_fp64_primitives_within_a_few_ulp():
    rng = np.random.default_rng(7)
    x = np.concatenate([10.0 ** rng.uniform(-6, 30, 400_000),
                        rng.uniform(0.5, 2.0, 100_000),            # one binade, densely
                        np.array([1.0, 2.0, 4.0, 0.25, 3.0, 1e-300, 1e300])])
    got = K.kerr_check_fp64_math(torch.tensor(x, device="cuda:0")).cpu().numpy()
    xl = x.astype(np.longdouble)
    # np.longdouble is at least the 80-bit format: its 1/x and sqrt are exact
    # to well below a double ulp
    assert np.finfo(np.longdouble).eps < 1e-18
    e_rcp = ulp_err(got[0], 1 / xl)
    e_rsq = ulp_err(got[1], 1 / np.sqrt(xl))
    e_sqrt = ulp_err(got[2], np.sqrt(xl))
    assert e_rcp.max() <= 2.0, e_rcp.max()
    assert e_rsq.max() <= 2.0, e_rsq.max()
    assert e_sqrt.max() <= 2.0, e_sqrt.max()
    # most results are correctly rounded
    assert np.mean(e_rcp <= 0.5) > 0.9 and np.mean(e_sqrt <= 0.5) > 0.9


def test_fp64_primitives_special_values():
    x = np.array([0.0, np.inf, np.nan, -1.0])
    got = K.kerr_check_fp64_math(torch.tensor(x, device="cuda:0")).cpu().numpy()
    assert got[2][0] == 0.0                        # sqrt(0) = 0
    assert np.isnan(got[:, 2]).all()               # NaN propagates
    assert np.isnan(got[1][3]) and np.isnan(got[2][3])   # negative: no root
    assert got[0][3] == -1.0
