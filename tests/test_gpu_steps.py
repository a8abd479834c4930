"""Per-stage parity of the CUDA merge kernels against the oracle (Sec. 4.2.1).

Each stage runs through its C-ABI step entry point on the same seeded input
as the oracle, compared element by element.
"""
import numpy as np
import pytest
import torch

from oracle import merge

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def bdc():
    from paper_2508_11467_gb300 import bdc as b
    from paper_2508_11467_gb300 import build
    build.build()
    b.lib()
    return b


def _M(N, seed, gap=1e-3):
    rng = np.random.default_rng(seed)
    d = np.concatenate(([0.0], np.sort(rng.uniform(gap, 1.0, N - 1))))
    for i in range(1, N):
        d[i] = max(d[i], d[i - 1] + gap)
    z = rng.uniform(0.05, 0.5, N) * rng.choice([-1.0, 1.0], N)
    return d, z


def _cu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("N,seed,gap", [(1, 0, 1e-3), (2, 1, 1e-3), (5, 2, 1e-3), (97, 3, 1e-3),
                                        (700, 4, 1e-4), (1500, 5, 1e-6)])
def test_secular_roots_match_oracle(bdc, N, seed, gap):
    d, z = _M(N, seed, gap)
    org, tau, om, info = bdc.secular_solve(_cu(d), _cu(z))
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    o_org, o_tau, o_om = merge.secular_roots(d, z)
    om_g = om.cpu().numpy()
    # omega to a few ulps of its own size (both solve f = 0 to rounding)
    assert np.max(np.abs(om_g - o_om) / o_om) <= 64 * EPS
    # interlacing, and the GPU's (org, tau) satisfy the secular equation
    assert np.all(om_g > d) and np.all(om_g[:-1] < d[1:])
    f, scale = merge.secular_f(d, z, org.cpu().numpy(), tau.cpu().numpy())
    assert np.all(np.abs(f) <= 64 * EPS * scale)


def _M_near_poles(N=200, seed=11):
    # roots within ~1e-27 (relative) of their poles: poles clustered at the
    # origin (0, 2.3e-11, 3.1e-10, 6.2e-9) with weights down to 1e-14, a pair
    # of tiny weights in the interior and a weak last pole (the shapes that
    # the top merges of an n = 16384 uniform matrix produce)
    rng = np.random.default_rng(seed)
    d = np.concatenate(([0.0, 2.2654e-11, 3.1e-10, 6.2e-9], np.sort(rng.uniform(1e-3, 1.0, N - 4))))
    for i in range(5, N):
        d[i] = max(d[i], d[i - 1] + 1e-4)
    z = rng.uniform(0.05, 0.5, N) * rng.choice([-1.0, 1.0], N)
    z[0], z[1], z[2], z[3] = 0.104, -8.82e-15, 6.6e-12, 3.3e-13
    z[50], z[51] = 3e-13, -2e-14
    z[N - 1] = 3.9e-6
    return d, z


def test_secular_near_pole_roots(bdc):
    # The rational model's quadratic is solved for the new iterate, measured
    # from the origin pole, not for a step added to the old one: a root within
    # eps |x| of its pole is reached by the model, not by bisection (a numpy
    # model of the step form needs up to 15 steps here, of the iterate form 7)
    d, z = _M_near_poles()
    org, tau, om, it, info = bdc.secular_solve_ex(_cu(d), _cu(z))
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    o_org, o_tau, o_om = merge.secular_roots(d, z)
    om_g = om.cpu().numpy()
    assert np.max(np.abs(om_g - o_om) / o_om) <= 64 * EPS
    # w = d_o + tau rounds onto the pole for these roots: interlacing holds
    # for (org, tau), the representation the vectors use
    og, tg = org.cpu().numpy(), tau.cpu().numpy()
    i = np.arange(len(d))
    assert np.all((og == i) | (og == i + 1))
    assert np.all(np.where(og == i, tg > 0, tg < 0))
    assert np.all(om_g >= d) and np.all(om_g[:-1] <= d[1:])
    f, scale = merge.secular_f(d, z, og, tg)
    assert np.all(np.abs(f) <= 64 * EPS * scale)
    # the offsets from the origin pole agree with the oracle's (to a few
    # hundred ulps of the offset itself: the roots near an interval's middle,
    # offset ~1e-3 from a pole ~0.5, carry ~eps |w| of rounding in either
    # solver; the near-pole offsets, 1e-38 to 1e-31, agree to a few ulps)
    same = og == o_org
    assert np.all(np.abs(tg[same] - o_tau[same]) <= 256 * EPS * np.abs(o_tau[same]))
    assert int(it.max().item()) <= 10


@pytest.mark.parametrize("N,seed", [(1, 7), (3, 8), (64, 9), (513, 10)])
def test_lowner_matches_oracle(bdc, N, seed):
    d, z = _M(N, seed, 1e-4)
    o_org, o_tau, _ = merge.secular_roots(d, z)
    zt_ref = merge.lowner_ztilde(d, z, o_org, o_tau)
    zt = bdc.lowner_z(_cu(d), _cu(z), _cu(o_org.astype(np.int32)), _cu(o_tau)).cpu().numpy()
    assert np.all(np.sign(zt) == np.sign(zt_ref))
    assert np.max(np.abs(zt - zt_ref) / np.abs(zt_ref)) <= 8 * N * EPS


@pytest.mark.parametrize("N,seed", [(1, 11), (4, 12), (100, 13), (600, 14)])
def test_m_vectors_match_oracle(bdc, N, seed):
    d, z = _M(N, seed, 1e-4)
    o_org, o_tau, _ = merge.secular_roots(d, z)
    zt = merge.lowner_ztilde(d, z, o_org, o_tau)
    UM_ref, VM_ref = merge.m_vectors(d, zt, o_org, o_tau)
    UM, VM = bdc.m_vectors(_cu(d), _cu(zt), _cu(o_org.astype(np.int32)), _cu(o_tau))
    assert np.max(np.abs(UM.cpu().numpy() - UM_ref)) <= 8 * N * EPS
    assert np.max(np.abs(VM.cpu().numpy() - VM_ref)) <= 8 * N * EPS


def _defl_case(m, seed):
    rng = np.random.default_rng(seed)
    d = np.concatenate(([0.0], np.sort(rng.uniform(0, 1, m - 1))))
    z = rng.uniform(-0.5, 0.5, m)
    # plant every case: small z, values close to d_0 = 0, close pairs and a chain
    k = max(m // 10, 1)
    z[rng.choice(np.arange(1, m), k, replace=False)] = 1e-19
    d[1:4] = [1e-18, 2e-18, 3e-18]
    for j in range(10, m - 3, 37):
        d[j + 1] = d[j] + 1e-17
        d[j + 2] = d[j + 1] + 2e-17
    d = np.maximum.accumulate(d)
    return d, z


@pytest.mark.parametrize("m,seed", [(3, 1), (50, 2), (1000, 3), (5000, 4)])
def test_deflation_decisions_bit_exact(bdc, m, seed):
    d, z = _defl_case(m, seed) if m > 3 else (np.array([0.0, 0.5, 0.5000000000000001]), np.array([0.2, 0.3, 0.4]))
    tol = merge.deflation_tol(d, 0.5, 0.5)
    ref = merge.deflate(d, z, tol)
    keep, zout, dval = bdc.deflate(_cu(d), _cu(z), tol)
    keep = keep.cpu().numpy().astype(bool)
    ref_keep = np.zeros(m, bool)
    ref_keep[ref["keep"]] = True
    assert np.array_equal(keep, ref_keep)                         # integer decisions: exact
    zk = zout.cpu().numpy()[keep]
    assert np.allclose(zk, ref["zkeep"], rtol=4 * EPS, atol=0)
    dv = dval.cpu().numpy()
    assert np.array_equal(dv[ref["defl"]], ref["dval"])


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (65, 70, 33), (300, 257, 190), (128, 128, 1000)])
def test_gemm_fp64(bdc, M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    C = bdc.gemm(_cu(A), _cu(B), "fp64").cpu().numpy()
    ref = A @ B
    bound = 2 * K * EPS * (np.abs(A) @ np.abs(B))
    assert np.all(np.abs(C - ref) <= bound + 1e-300)
