"""The FLOP-counting transcription of eqs. opt0/opti computes the same
acceleration as the oracle's Christoffel-form right-hand side (eq. geo)."""
import numpy as np
import pytest

from oracle import flops as F
from oracle import oracle as O


@pytest.mark.parametrize("a", [0.0, 0.4, 0.9, 0.999])
def test_optimised_form_matches_christoffel_form(a):
    rng = np.random.default_rng(11)
    for _ in range(40):
        r = rng.uniform(1.05 * (1 + np.sqrt(1 - a * a)), 200.0)
        th, ph = rng.uniform(0.01, np.pi - 0.01), rng.uniform(0, 2 * np.pi)
        X = [(r * np.cos(ph) - a * np.sin(ph)) * np.sin(th),
             (r * np.sin(ph) + a * np.cos(ph)) * np.sin(th), r * np.cos(th)]
        y = np.array([rng.normal(), *X, *rng.normal(size=4)])
        ref = O.rhs(a, y)[4:]
        got = np.array(F.rhs_opt(a, a * a, list(y), sqrt=np.sqrt))
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_counts_are_stable():
    t = F.count_rhs()
    assert (t.add, t.mul, t.div, t.sqrt) == (51, 104, 3, 2)
    assert F.count_attempt().flops == 366
