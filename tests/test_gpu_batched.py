"""Batched SVD (bdc_svd_batched, plans replayed as CUDA graphs, autotuner)
against the FP64 oracle.

Every checked matrix meets the FP64 bar of the single-matrix path
(relative singular-value error, residual and orthogonality <= 1e-13 n).
The 2048-matrix batch has orders floor(exp(U(ln 32, ln 1024))) (seed 3),
d, e ~ U(0.5, 1.5); a spread of its matrices is checked one by one.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import check
from paper_2508_11467_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bdc():
    from paper_2508_11467_gb300 import bdc as b
    from paper_2508_11467_gb300 import build
    build.build()
    b.lib()
    return b


def _flat(mats):
    ns = np.array([len(d) for d, _ in mats], dtype=np.int32)
    off = np.concatenate([[0], np.cumsum(ns)])
    D = np.zeros(int(off[-1]))
    E = np.zeros(int(off[-1]))
    for b, (d, e) in enumerate(mats):
        D[off[b]:off[b] + len(d)] = d
        E[off[b]:off[b] + len(e)] = e
    return ns, torch.from_numpy(D).cuda(), torch.from_numpy(E).cuda()


def _orth(X):
    G = X.t() @ X
    G.diagonal().sub_(1.0)
    return float(torch.linalg.norm(G))


def _check(d, e, S, U, VT, tol_scale=1e-13, res_tol=None):
    n = len(d)
    s = S.cpu().numpy()
    tol = tol_scale * n
    assert np.all(np.diff(s) <= 0) and np.all(s >= 0)
    assert check.sigma_rel_err(s, oracle.sigma_only(d, e)) <= tol
    res = oracle.residual(d, e, s, U.cpu().numpy(), VT.cpu().numpy())
    assert res <= (res_tol if res_tol is not None else tol), res
    assert _orth(U) <= tol and _orth(VT.t()) <= tol


def test_batched_list_api_matches_oracle(bdc):
    mats = inputs.batch(64, seed=3, lo=32, hi=300)
    ds = [torch.from_numpy(d).cuda() for d, _ in mats]
    es = [torch.from_numpy(e).cuda() for _, e in mats]
    Ss, Us, VTs, info = bdc.svd_batched(ds, es)
    torch.cuda.synchronize()
    assert int(info.abs().max()) == 0
    for b, (d, e) in enumerate(mats):
        _check(d, e, Ss[b], Us[b], VTs[b])


def test_batched_matches_single_matrix_bitwise(bdc):
    mats = inputs.batch(20, seed=7, lo=32, hi=400)
    ds = [torch.from_numpy(d).cuda() for d, _ in mats]
    es = [torch.from_numpy(e).cuda() for _, e in mats]
    Ss, Us, VTs, info = bdc.svd_batched(ds, es)
    for b in (0, 7, 19):
        S1, U1, VT1, _ = bdc.svd(ds[b], es[b])
        assert torch.equal(Ss[b], S1) and torch.equal(Us[b], U1) and torch.equal(VTs[b], VT1)


def test_plan_graph_equals_direct_call_and_replays(bdc):
    mats = inputs.batch(48, seed=5, lo=32, hi=512)
    ns, D, E = _flat(mats)
    plan = bdc.BatchPlan(D, E, ns)
    plan.launch()
    torch.cuda.synchronize()
    assert int(plan.info.abs().max()) == 0
    ds = [torch.from_numpy(d).cuda() for d, _ in mats]
    es = [torch.from_numpy(e).cuda() for _, e in mats]
    Ss, Us, VTs, _ = bdc.svd_batched(ds, es)
    for b in range(len(mats)):
        S, U, VT = plan.result(b)
        assert torch.equal(S, Ss[b]) and torch.equal(U, Us[b]) and torch.equal(VT, VTs[b])
    # the graph reads the inputs at launch time: new values, same plan
    mats2 = [inputs.uniform(int(n), 1000 + b) for b, n in enumerate(ns)]
    _, D2, E2 = _flat(mats2)
    plan.d.copy_(D2)
    plan.e.copy_(E2)
    plan.launch()
    plan.launch()
    torch.cuda.synchronize()
    for b in (0, 11, 47):
        S, U, VT = plan.result(b)
        _check(*mats2[b], S, U, VT)
    plan.close()


def _residual_gpu(d, e, S, U, VT):
    d = torch.as_tensor(d, device="cuda", dtype=torch.float64)
    e = torch.as_tensor(e, device="cuda", dtype=torch.float64)
    U, VT, S = U.double(), VT.double(), S.double()
    V = VT.t()
    BV = d[:, None] * V
    BV[:-1] += e[:, None] * V[1:]
    return float(torch.linalg.norm(BV - U * S[None, :]) / torch.sqrt((d * d).sum() + (e * e).sum()))


def _check_batch(mats, plan, tol_scale, rounded=False):
    """Every matrix's singular values against the oracle (sigma-only QR of
    each matrix); residual and orthogonality of 256 matrices spread over the
    sizes (cuBLAS checkers on the device)."""
    if rounded:   # FP32: the oracle of the FP32-rounded input
        mats = [(d.astype(np.float32).astype(np.float64), e.astype(np.float32).astype(np.float64)) for d, e in mats]
    refs = oracle.sigma_only_many(mats)
    ns = np.array([len(d) for d, _ in mats])
    worst = 0.0
    for b, (d, e) in enumerate(mats):
        s = plan.result(b)[0].double().cpu().numpy()
        assert np.all(np.diff(s) <= 0) and np.all(s >= 0), b
        err = check.sigma_rel_err(s, refs[b])
        assert err <= tol_scale * ns[b], (b, ns[b], err)
        worst = max(worst, err / ns[b])
    order = np.argsort(ns)
    for b in order[np.linspace(0, len(ns) - 1, 256).astype(int)]:
        S, U, VT = plan.result(int(b))
        tol = tol_scale * ns[b]
        assert _residual_gpu(*mats[b], S, U, VT) <= tol, b
        assert _orth(U.double()) <= tol and _orth(VT.double().t()) <= tol, b
    print(f"worst sigma error / n over {len(mats)} matrices: {worst:.2e}")


def test_config4_2048_matrices(bdc):
    """2048 bidiagonals, n log-uniform in [32, 1024], one graph launch: every
    matrix's singular values against the oracle."""
    mats = inputs.batch(2048, seed=3)
    ns, D, E = _flat(mats)
    assert ns.min() >= 32 and ns.max() <= 1024
    plan = bdc.BatchPlan(D, E, ns)
    plan.launch()
    torch.cuda.synchronize()
    assert int(plan.info.abs().max()) == 0
    _check_batch(mats, plan, 1e-13)
    plan.close()


def test_config4_2048_matrices_split_products(bdc):
    """The same batch with the split-BF16 products (the benchmark's FP64 batch)."""
    mats = inputs.batch(2048, seed=3)
    ns, D, E = _flat(mats)
    plan = bdc.BatchPlan(D, E, ns, prec="exact", mixed_min=64)
    plan.launch()
    torch.cuda.synchronize()
    assert int(plan.info.abs().max()) == 0
    _check_batch(mats, plan, 1e-13)
    plan.close()


def test_batched_mixed_products(bdc):
    mats = inputs.batch(32, seed=9, lo=300, hi=1024)
    ns, D, E = _flat(mats)
    plan = bdc.BatchPlan(D, E, ns, prec="exact")
    plan.launch()
    torch.cuda.synchronize()
    assert int(plan.info.abs().max()) == 0
    for b in (0, 13, 31):
        S, U, VT = plan.result(b)
        _check(*mats[b], S, U, VT, res_tol=1e-12)
    plan.close()


def test_autotune_picks_a_candidate_and_caches(bdc):
    import time
    ns = inputs.batch_sizes(256, seed=3)
    leaf, mm, ms = bdc.autotune(ns, "fp64", reps=2)
    assert leaf in (8, 12, 16, 24, 32) and ms > 0
    t0 = time.perf_counter()
    leaf2, mm2, ms2 = bdc.autotune(ns, "fp64", reps=2)
    assert (leaf2, mm2, ms2) == (leaf, mm, ms)
    assert time.perf_counter() - t0 < 0.5
    leaf3, mm3, _ = bdc.autotune(ns, "exact", reps=1)
    assert leaf3 in (8, 12, 16, 24, 32) and mm3 in (32, 64, 128, 256, 512, 4096)
    # the chosen configuration solves the batch correctly
    mats = inputs.batch(256, seed=3)
    _, D, E = _flat(mats)
    plan = bdc.BatchPlan(D, E, ns, leaf=leaf)
    plan.launch()
    torch.cuda.synchronize()
    assert int(plan.info.abs().max()) == 0
    S, U, VT = plan.result(5)
    _check(*mats[5], S, U, VT)
    plan.close()


# ---------------------------------------------------------------- FP32
def _check32(d, e, S, U, VT, tol_scale=1e-5):
    """FP32 bar: 1e-5 n on sigma, residual and orthogonality, measured in FP64
    against the oracle of the FP32-rounded input."""
    d = d.astype(np.float32).astype(np.float64)
    e = e.astype(np.float32).astype(np.float64)
    n = len(d)
    tol = tol_scale * n
    s = S.double().cpu().numpy()
    assert np.all(np.diff(s) <= 0) and np.all(s >= 0)
    assert check.sigma_rel_err(s, oracle.sigma_only(d, e)) <= tol
    assert oracle.residual(d, e, s, U.double().cpu().numpy(), VT.double().cpu().numpy()) <= tol
    assert _orth(U.double()) <= tol and _orth(VT.double().t()) <= tol


def test_fp32_batch_matches_oracle(bdc):
    mats = inputs.batch(64, seed=3, lo=32, hi=300)
    ns, D, E = _flat(mats)
    plan = bdc.BatchPlan(D.float(), E.float(), ns, dtype=torch.float32)
    plan.launch()
    torch.cuda.synchronize()
    assert int(plan.info.abs().max()) == 0
    for b, (d, e) in enumerate(mats):
        S, U, VT = plan.result(b)
        assert S.dtype == torch.float32
        _check32(d, e, S, U, VT)
    plan.close()


@pytest.mark.parametrize("kind", ["graded", "clustered", "ones"])
def test_fp32_other_inputs(bdc, kind):
    mats = [inputs.make(kind, n, 11 + n) for n in (33, 200, 513)]
    ns, D, E = _flat(mats)
    plan = bdc.BatchPlan(D.float(), E.float(), ns, dtype=torch.float32)
    plan.launch()
    torch.cuda.synchronize()
    assert int(plan.info.abs().max()) == 0
    for b, (d, e) in enumerate(mats):
        _check32(d, e, *plan.result(b))
    plan.close()


def test_fp32_config4_2048_matrices(bdc):
    mats = inputs.batch(2048, seed=3)
    ns, D, E = _flat(mats)
    plan = bdc.BatchPlan(D.float(), E.float(), ns, dtype=torch.float32)
    plan.launch()
    plan.launch()
    torch.cuda.synchronize()
    assert int(plan.info.abs().max()) == 0
    _check_batch(mats, plan, 1e-5, rounded=True)
    plan.close()


def test_fp32_rejects_fp64_only_options(bdc):
    ns = np.array([40, 50], dtype=np.int32)
    D = torch.ones(90, device="cuda")
    with pytest.raises(bdc.BDCError):
        bdc.BatchPlan(D, D, ns, prec="exact", dtype=torch.float32)


def test_fp32_autotune(bdc):
    ns = inputs.batch_sizes(256, seed=4)
    leaf, mm, ms = bdc.autotune(ns, reps=2, dtype=torch.float32)
    assert leaf in (8, 12, 16, 24, 32) and ms > 0
    assert bdc.autotune(ns, reps=2, dtype=torch.float32) == (leaf, mm, ms)
