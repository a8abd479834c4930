"""Singular values only (bdc_svd_values): the same tree, deflation and
secular roots with two rows of V per node instead of the panels.  Same
bar as the full path: relative singular-value error <= 1e-13 n against the
FP64 oracle, and agreement with the full path's values."""
import numpy as np
import pytest
import torch

import oracle
from oracle import check
from paper_2508_11467_gb300 import inputs

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def bdc():
    from paper_2508_11467_gb300 import bdc as b
    from paper_2508_11467_gb300 import build
    build.build()
    b.lib()
    return b


def _vals(bdc, d, e, **kw):
    S, info = bdc.svd_values(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda(), **kw)
    assert info == 0
    s = S.cpu().numpy()
    assert np.all(np.diff(s) <= 0) and np.all(s >= 0)
    return s


@pytest.mark.parametrize("n,leaf", [(1, 16), (2, 16), (7, 4), (32, 32), (33, 16), (100, 8), (257, 4), (1000, 16)])
def test_values_small(bdc, n, leaf):
    d, e = inputs.uniform(n, 300 + n)
    s = _vals(bdc, d, e, leaf=leaf)
    assert check.sigma_rel_err(s, oracle.sigma_only(d, e)) <= 1e-13 * n


@pytest.mark.parametrize("kind,seed", [("uniform", 0), ("graded", 1), ("clustered", 2)])
def test_values_config2(bdc, kind, seed):
    d, e = inputs.make(kind, 4096, seed)
    s = _vals(bdc, d, e)
    assert check.sigma_rel_err(s, oracle.sigma_only(d, e)) <= 1e-13 * 4096
    S, U, VT, info = bdc.svd(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda())
    assert np.max(np.abs(s - S.cpu().numpy())) <= 1e-13 * 4096 * s[0]


def test_values_closed_form(bdc):
    n = 4096
    d, e = inputs.ones(n)
    k = np.arange(1, n + 1)
    s = _vals(bdc, d, e)
    assert check.sigma_rel_err(s, 2.0 * np.cos(k * np.pi / (2 * n + 1))) <= 1e-13 * n


def test_values_edge_cases(bdc):
    d, e = inputs.uniform(200, 7)
    d = d.copy()
    d[[0, 57, 99, 199]] = 0.0
    s = _vals(bdc, d, e)
    assert check.sigma_rel_err(s, oracle.sigma_only(d, e)) <= 1e-13 * 200
    s = _vals(bdc, np.zeros(100), np.zeros(99))
    assert np.all(s == 0.0)
    d, e = inputs.uniform(300, 10)
    sgn = np.where(np.arange(300) % 3 == 0, -1.0, 1.0)
    s = _vals(bdc, d * sgn * 1e150, e * sgn[:299] * 1e150)
    assert check.sigma_rel_err(s, oracle.sigma_only(d, e) * 1e150) <= 1e-13 * 300
    d[5] = np.inf
    S, info = bdc.svd_values(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda(), check=False)
    assert info == bdc.BDC_ERR_NONFINITE


def test_values_across_the_exponent_range(bdc):
    """Entries of 1e150 beside entries of 1e-170, in rows whose d and e are
    both below the normal range once scaled: the merge's coupling entries
    are then subnormal, and the rotation folding them must still be
    orthogonal (the two tracked rows of V carry it to the parent's z)."""
    d, e = inputs.uniform(300, 12)
    d, e = d * 1e150, e * 1e150
    d[::7] = 1e-170
    e[3::11] = -1e-170
    s = _vals(bdc, d, e, leaf=16)
    assert check.sigma_rel_err(s, oracle.sigma_only(d, e)) <= 1e-13 * 300


def test_values_seeded_start(bdc):
    d, e = inputs.graded(2048, 3)
    s0 = _vals(bdc, d, e)
    s1 = _vals(bdc, d, e, seed="analytic")
    assert np.max(np.abs(s0 - s1)) <= 64 * EPS * s0[0]
