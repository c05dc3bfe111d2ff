"""Host-side pieces of the experiments (no GPU): the closed-form Student-t CDF
used by the GPU stream generator, pinned against scipy's implementation, and
the Bell numbers of the complexity model (Eq. complxn)."""
import numpy as np
from scipy import special

from paper_1701_06446_gb300.experiments import bell
from paper_1701_06446_gb300.streams import student_t_cdf_even


def test_student_t_cdf_even_matches_scipy():
    x = np.concatenate([np.linspace(-40, 40, 4001), [0.0, 1e-8, -1e-8, 1e3, -1e3]])
    for nu in (2, 4, 6, 10, 30):
        np.testing.assert_allclose(student_t_cdf_even(x, nu), special.stdtr(nu, x), rtol=0, atol=1e-15)


def test_student_t_cdf_rejects_odd_nu():
    import pytest
    with pytest.raises(ValueError):
        student_t_cdf_even(np.zeros(3), 5)


def test_bell_numbers():
    assert [bell(d) for d in range(9)] == [1, 1, 2, 5, 15, 52, 203, 877, 4140]
