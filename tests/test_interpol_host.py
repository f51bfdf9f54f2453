"""Interpol's host computation (Sec. 4.4, Eq. (polinterpcoef)) against the oracle's, without a GPU:
the library's Chebyshev coefficients of each f_i on the region's real axis."""
import numpy as np
import pytest

from oracle import interpol
from synth.problems import _exp, _rational, _sqrt


@pytest.mark.parametrize("d", [2, 9, 40])
def test_coefficients_match_the_oracle(d):
    from paper_1910_11712_gb300 import binding
    binding.load(build_if_missing=True)
    region = {"center": 1.5 + 0j, "a": 1.2, "b": 0.05}
    fns = [_exp(alpha=-1.0), _rational([-1.0, 0.0]), _rational([1.0, 0.5], [1.0, 5.0]),
           _sqrt(shift=-0.5, alpha=1.0, beta=1j)]
    c_lib = binding.interpol_coefficients(fns, region, d)
    c_ora = interpol.coefficients(fns, region, d)
    assert np.abs(c_lib - c_ora).max() <= 1e-14 * max(1.0, np.abs(c_ora).max())


def test_coefficient_refusals():
    from paper_1910_11712_gb300 import binding
    binding.load(build_if_missing=True)
    with pytest.raises(binding.NepError):
        binding.interpol_coefficients([_exp()], {"center": 1 + 1j, "a": 1.0, "b": 0.1}, 8)  # complex centre
    with pytest.raises(binding.NepError):
        binding.interpol_coefficients([_exp()], {"center": 1.0, "a": 1.0, "b": 0.1}, 1)     # degree < 2
