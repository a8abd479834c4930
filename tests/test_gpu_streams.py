"""The solve's second stream.

After each merge's prep the gather, the A-operand slicing of the split-BF16
products and the node finish run on a side stream while the caller's stream
finds the roots (Sec. 4.2, Algorithm 2: none of them needs the roots, except
the finish, which is forked after them); the caller's stream waits for the
side stream before the products.  Merges of order >= 4096 also form their
merged order and z over a grid before the prep.  These tests check that the
overlap changes nothing:

* the same call captured into a CUDA graph (the side stream joins the
  capture through the fork event) replays to the eager call's bits, twice;
* the overlapped solve equals, bit for bit, the serial one the stage profiler
  runs (every stage on the caller's stream), and both meet the oracle.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2508_11467_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bdc():
    from paper_2508_11467_gb300 import bdc as b
    from paper_2508_11467_gb300 import build
    build.build()
    b.lib()
    return b


class _Call:
    """bdc_svd_ex on fixed device buffers (capturable: no host sync)."""

    def __init__(self, bdc, d, e, prec):
        self.bdc, self.n = bdc, len(d)
        n = self.n
        self.dc, self.ec = torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda()
        self.o = bdc.make_opts(prec, 0)
        lw = bdc.workspace_bytes(n, self.o)
        self.work = torch.empty(lw + 256, dtype=torch.uint8, device="cuda")
        self.U = torch.empty((n, n), dtype=torch.float64, device="cuda")
        self.VT = torch.empty((n, n), dtype=torch.float64, device="cuda")
        self.S = torch.empty(n, dtype=torch.float64, device="cuda")
        self.info = torch.zeros(1, dtype=torch.int32, device="cuda")

    def __call__(self, stream=None):
        b, n = self.bdc, self.n
        st = stream if stream is not None else torch.cuda.current_stream()
        return b.lib().bdc_svd_ex(n, b._ptr(self.dc), b._ptr(self.ec), b._ptr(self.U), b._ptr(self.S),
                                  b._ptr(self.VT), n, n, ctypes.byref(self.o),
                                  ctypes.c_void_p(self.work.data_ptr()), self.work.numel(), b._ptr(self.info),
                                  ctypes.c_void_p(st.cuda_stream))

    def result(self):
        torch.cuda.synchronize()
        assert int(self.info.item()) == 0
        return self.S.clone(), self.U.clone(), self.VT.clone()


def _check_oracle(d, e, S):
    ref = np.sort(np.asarray(oracle.sigma_only(d, e)))[::-1]
    s = S.cpu().numpy()
    assert np.max(np.abs(s - ref)) <= 1e-13 * len(d) * ref[0]


@pytest.mark.parametrize("prec", ["fp64", "exact"])
def test_graph_replay_equals_eager(bdc, prec):
    n = 4096                              # the root merge takes the grid-wide merged order
    d, e = inputs.uniform(n, 21)
    call = _Call(bdc, d, e, prec)
    assert call() == 0
    S0, U0, VT0 = call.result()
    _check_oracle(d, e, S0)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        assert call(torch.cuda.current_stream()) == 0
    for _ in range(2):
        call.S.zero_()
        call.U.zero_()
        call.VT.zero_()
        call.info.fill_(-7)
        g.replay()
        S1, U1, VT1 = call.result()
        assert torch.equal(S1, S0) and torch.equal(U1, U0) and torch.equal(VT1, VT0)
    del g
    torch.cuda.synchronize()


@pytest.mark.parametrize("kind", ["uniform", "graded"])
def test_overlap_equals_serial_stage_order(bdc, kind):
    n = 6000                              # heights with split-BF16 products and the grid-wide merged order
    d, e = inputs.make(kind, n, 5)
    call = _Call(bdc, d, e, "exact")
    assert call() == 0
    S0, U0, VT0 = call.result()
    bdc.profile_begin()                   # the stage profiler keeps every stage on the caller's stream
    try:
        assert call() == 0
        S1, U1, VT1 = call.result()
    finally:
        bdc.profile_end()
    assert torch.equal(S1, S0) and torch.equal(U1, U0) and torch.equal(VT1, VT0)
    _check_oracle(d, e, S0)
