"""The oracle's prior constants against the paper's printed configuration
(tests/golden/prior_configuration.json, Appendix B.2 and Sec. 2.2)."""
import json
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(__file__)


def test_prior_constants_match_the_paper():
    g = json.load(open(os.path.join(HERE, "golden", "prior_configuration.json")))
    assert oracle.PRIOR_MU_SD == g["profile_shift_mu"]["sd"]
    assert g["profile_shift_mu"]["mean"] == 0.0
    assert oracle.PRIOR_ALPHA_MEAN == g["peak_asymmetry_alpha"]["mean"]
    assert oracle.PRIOR_ALPHA_SD == g["peak_asymmetry_alpha"]["sd"]
    assert oracle.PRIOR_W_SHAPE == g["peak_width_w"]["shape"]
    assert oracle.PRIOR_W_RATE == g["peak_width_w"]["second_parameter"]
    assert g["intensity_h"]["shape"] == 1


def test_intensity_rate_is_inverse_max_signal():
    """Sec. 2.2: lambda = 1/eta with eta = max(Y - B)."""
    x = np.linspace(10, 20, 6)
    y = np.array([10, 80, 400, 90, 30, 12.0])
    bg = np.array([5, 6, 7, 8, 9, 10.0])
    P = oracle.Problem([0, 1], [15.0], [1.0], x, y, bg)
    assert P.prior.lambda_ == pytest.approx(1.0 / 393.0)
