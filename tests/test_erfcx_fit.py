"""The float32 short-range kernel takes erfc(x) as exp(-x^2) times a fitted
erfc(x) exp(x^2) (Eq. velocity_shortrange needs erfc and the Gaussian of
the Ewald split).  These checks pin the coefficients compiled into
k_short.cu to the committed fit and bound its error against scipy's erfcx."""
import importlib.util
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2406_07366_gb300", "csrc")


def _gen():
    pytest.importorskip("scipy")
    spec = importlib.util.spec_from_file_location("gen_erfcx_fit", os.path.join(CSRC, "gen_erfcx_fit.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _compiled_coefficients():
    src = open(os.path.join(CSRC, "k_short.cu")).read()
    body = re.search(r"constexpr float c\[11\] = \{([^}]*)\}", src).group(1)
    return np.array([float(v.strip().rstrip("f")) for v in body.split(",")])


def test_compiled_coefficients_are_the_fit():
    g = _gen()
    _, _, c = g.fit()
    assert np.allclose(_compiled_coefficients(), c, rtol=1e-8, atol=1e-12)


def test_fit_error_in_float32():
    g = _gen()
    xs, h, c = g.fit()
    assert g.float32_rel_error(xs, h, _compiled_coefficients()) < 4e-7


def test_fit_special_values():
    from scipy.special import erfc
    g = _gen()
    c = _compiled_coefficients()
    for x in (0.0, 0.5, 1.0, 2.0, 3.5, 6.0):
        t = 1.0 / (1.0 + g.P * x)
        h = np.polyval(c[::-1], t)
        assert abs(h * np.exp(-x * x) - erfc(x)) <= 4e-7 * erfc(x)
