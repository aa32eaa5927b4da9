"""The oracle's default parameters are the ones the paper prints
(Sec. IV-F), read from tests/golden/paper_parameters.txt."""
import pytest

import oracle
from tests.golden.load import paper_parameters


def test_kernel_defaults_match_paper():
    p = paper_parameters()
    kp = oracle.KernelParams()
    for name in ("lambda_omega", "alpha1", "alpha2", "mu1", "mu2", "mu3",
                 "rho", "t_max", "th"):
        assert getattr(kp, name) == pytest.approx(p[name]), name


def test_hrms_defaults_match_paper():
    p = paper_parameters()
    hp = oracle.HrmsParams()
    assert hp.lam == pytest.approx(p["lambda"])
    assert hp.r == p["r"]
