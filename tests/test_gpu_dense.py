"""The dense front and back end on the GPU against the FP64 oracle and LAPACK.

* bdc_gebrd (Sec. 4.1, Algorithm 1, blocked with the merged rank-(2b)
  update) against the unblocked oracle: d, e, tauq, taup and the stored
  reflectors element by element (the Householder reduction is unique for a
  fixed sign convention), within 1e-13 n of ||A||; and A = Q1 B P1^T with
  Q1, P1 formed by bdc_ormbr.
* bdc_geqrf / bdc_orgqr (Sec. 4.3) against the oracle's R and LAPACK's R,
  Q R = A and Q^T Q = I.
* bdc_gesvd: singular values against LAPACK (numpy) and the oracle's own
  pipeline, reconstruction and orthogonality, square and tall-and-skinny.
Test matrices: A = Qm diag(sigma) Qn^T with the SVD_arith/geo/logrand
singular values of the paper's test set (inputs.dense) and Gaussian ones.
"""
import numpy as np
import pytest
import torch

from oracle import dense_svd as od
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


def _matrix(kind, m, n, seed):
    if kind == "gauss":
        return np.random.default_rng(seed).standard_normal((m, n))
    Q, s, V = inputs.dense(kind, m, n, 1e4, seed)
    return (Q * s[None, :]) @ V.T


def _orth(X):
    G = X.t() @ X
    G.diagonal().sub_(1.0)
    return float(torch.linalg.norm(G))


@pytest.mark.parametrize("m,n,kind", [(1, 1, "gauss"), (2, 2, "gauss"), (5, 3, "gauss"), (33, 33, "gauss"),
                                      (64, 64, "geo"), (100, 37, "gauss"), (97, 96, "arith"),
                                      (300, 300, "logrand"), (700, 500, "gauss"), (1000, 1000, "geo")])
def test_gebrd_matches_oracle(bdc, m, n, kind):
    A = _matrix(kind, m, n, m + n)
    Ar_ref, d_ref, e_ref, tq_ref, tp_ref = od.gebrd(A)
    Ar, d, e, tq, tp, info = bdc.gebrd(torch.from_numpy(A).cuda())
    torch.cuda.synchronize()
    assert info == 0
    nA = np.linalg.norm(A)
    tol = 1e-13 * max(n, 1) * nA
    # B is unique up to the signs of its entries: a pivot that rounding puts
    # on the other side of zero (|alpha| << ||x||) flips beta and the rest
    # of that reflector; |d|, |e| are unique
    dg, eg = d.cpu().numpy(), e.cpu().numpy()
    # Element-wise parity is only defined where the reduction itself is
    # well conditioned: the oracle is run again on A perturbed by 1e-16
    # relative, and if its own |d|, |e| move by more than the tolerance (a
    # near-breakdown of the Golub-Kahan recurrence: some e_i ~ 1e-7 ||A||),
    # the GPU result is judged by reconstruction and singular values only.
    _, d_p, e_p, _, _ = od.gebrd(A * (1.0 + 1e-16 * np.random.default_rng(0).standard_normal(A.shape)))
    stable = (np.max(np.abs(np.abs(d_p) - np.abs(d_ref)), initial=0.0) <= tol and
              np.max(np.abs(np.abs(e_p) - np.abs(e_ref)), initial=0.0) <= tol)
    if stable:
        assert np.max(np.abs(np.abs(dg) - np.abs(d_ref)), initial=0.0) <= tol
        assert np.max(np.abs(np.abs(eg) - np.abs(e_ref)), initial=0.0) <= tol
    else:
        print(f"{m}x{n} {kind}: the reduction is ill-conditioned (the oracle moves under a 1e-16 perturbation)")
        import oracle
        s_ref = np.linalg.svd(A, compute_uv=False)
        assert np.max(np.abs(oracle.sigma_only(dg, eg) - s_ref)) <= tol
    same = stable and np.array_equal(np.sign(dg), np.sign(d_ref)) and np.array_equal(np.sign(eg), np.sign(e_ref))
    if same:
        # no flip: reflector scalars and vectors element by element (entries of
        # unit-scale vectors, relative)
        assert np.max(np.abs(tq.cpu().numpy() - tq_ref), initial=0.0) <= 1e-12 * n
        assert np.max(np.abs(tp.cpu().numpy()[:max(n - 1, 0)] - tp_ref[:max(n - 1, 0)]), initial=0.0) <= 1e-12 * n
        low = np.tril(np.ones((m, n), dtype=bool), -1)
        up = np.triu(np.ones((m, n), dtype=bool), 2)
        Arn = Ar.cpu().numpy()
        assert np.max(np.abs(Arn[low] - Ar_ref[low]), initial=0.0) <= 1e-11 * n
        assert np.max(np.abs(Arn[up] - Ar_ref[up]), initial=0.0) <= 1e-11 * n
    else:
        print(f"{m}x{n} {kind}: a pivot changed sign under rounding; reflectors compared through A = Q1 B P1^T")
    # A = Q1 B P1^T with Q1 = bdc_ormbr(0, I), P1^T = bdc_ormbr(1, I)
    Q = torch.eye(m, n, dtype=torch.float64, device="cuda").t().contiguous().t()
    bdc.ormbr(0, Ar, tq, Q)
    PT = torch.eye(n, dtype=torch.float64, device="cuda").t().contiguous().t()
    bdc.ormbr(1, Ar, tp, PT)
    B = torch.diag(d)
    if n > 1:
        B += torch.diag(e, 1)
    Ac = torch.from_numpy(A).cuda()
    assert float(torch.linalg.norm(Q @ B @ PT - Ac)) <= tol
    assert _orth(Q) <= 1e-13 * n and _orth(PT.t()) <= 1e-13 * n


@pytest.mark.parametrize("m,n", [(1, 1), (7, 3), (64, 64), (300, 31), (1000, 200), (2500, 100)])
def test_geqrf_orgqr(bdc, m, n):
    A = _matrix("gauss", m, n, 7 * m + n)
    Ar, tau, info = bdc.geqrf(torch.from_numpy(A).cuda())
    torch.cuda.synchronize()
    assert info == 0
    R = torch.triu(Ar[:n, :n]).cpu().numpy()
    Ar_ref, tau_ref = od.geqrf(A)
    nA = np.linalg.norm(A)
    assert np.max(np.abs(R - np.triu(Ar_ref[:n, :n]))) <= 1e-13 * n * nA
    assert np.max(np.abs(R - np.linalg.qr(A, mode="r"))) <= 1e-13 * n * nA
    assert np.max(np.abs(tau.cpu().numpy() - tau_ref)) <= 1e-12 * n
    Q = bdc.orgqr(Ar, tau)
    torch.cuda.synchronize()
    Rc = torch.from_numpy(R).cuda()
    assert float(torch.linalg.norm(Q @ Rc - torch.from_numpy(A).cuda())) <= 1e-13 * n * nA
    assert _orth(Q) <= 1e-13 * n


@pytest.mark.parametrize("m,n,kind,prec", [(200, 200, "gauss", "fp64"), (513, 300, "geo", "fp64"),
                                           (1000, 1000, "logrand", "exact"), (777, 333, "arith", "exact"),
                                           (2000, 300, "gauss", "fp64"), (20000, 1000, "geo", "exact"),
                                           (2048, 2048, "gauss", "exact")])
def test_gesvd(bdc, m, n, kind, prec):
    A = _matrix(kind, m, n, m * 3 + n)
    S, U, VT, info = bdc.gesvd(torch.from_numpy(A).cuda(), prec=prec)
    torch.cuda.synchronize()
    assert info == 0
    s = S.cpu().numpy()
    s_ref = np.linalg.svd(A, compute_uv=False)
    tol = 1e-13 * n
    assert np.all(np.diff(s) <= 0)
    assert np.max(np.abs(s - s_ref)) <= tol * s_ref[0]
    Ac = torch.from_numpy(A).cuda()
    res = float(torch.linalg.norm(U * S[None, :] @ VT - Ac) / torch.linalg.norm(Ac))
    assert res <= tol, res
    assert _orth(U) <= tol and _orth(VT.t()) <= tol


def test_gesvd_matches_oracle_pipeline(bdc):
    """The oracle's own unblocked pipeline (gebrd, QR iteration, back
    transformation) gives the same singular values."""
    A = _matrix("logrand", 150, 90, 5)
    s_ref, U_ref, VT_ref = od.gesvd(A)
    S, U, VT, info = bdc.gesvd(torch.from_numpy(A).cuda())
    assert info == 0
    assert np.max(np.abs(S.cpu().numpy() - s_ref)) <= 1e-13 * 90 * s_ref[0]
