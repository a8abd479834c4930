"""Merge-step oracle for bidiagonal divide-and-conquer, numpy FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Every function follows
the paper's Sec. 4.2.1 in its notation; 0-based indices replace the paper's
1-based ones (paper index i is index i-1 here).

* ``secular_roots``  -- the N roots omega_i of the secular equation
  (Eq. M-svd-val), f(w) = 1 + sum_j z_j^2 / (d_j^2 - w^2), with d_0 = 0 <
  d_1 < ... < d_{N-1}.  Root i lies in (d_i, d_{i+1}); the last one in
  (d_{N-1}, sqrt(d_{N-1}^2 + |z|^2)).  Plain bisection on f, with each root
  held as w = d_org + tau (org = the nearer pole) so that d_j - w is formed
  as (d_j - d_org) - tau without cancellation.
* ``lowner_ztilde`` -- |z~_i| of Eq. (bdc-zi), sign taken from z_i.
* ``m_vectors``      -- the normalised singular vectors u_i, v_i of M~
  (Eq. M-svd-vec).
* ``deflate``        -- the deflation of Sec. 4.2.1: small z components
  (z_0 clamped up to tol, z_i for i >= 1 zeroed) and close singular values
  (one-sided rotation against d_0 = 0, two-sided rotation otherwise).
* ``bdc_svd``        -- Algorithm 2 end to end: split, leaves by QR iteration,
  bottom-up merges, final sort.  A slow model of the whole method used to pin
  the merge algebra against the QR oracle.

Readings where the paper is silent are listed with each function.
"""
from __future__ import annotations

import numpy as np

EPS = np.finfo(np.float64).eps  # 2^-52


# --------------------------------------------------------------------------
# secular equation (Eq. M-svd-val)
# --------------------------------------------------------------------------
def _f_shifted(d, z, org, tau):
    """f(w) at w = d[org] + tau, all roots at once (rows = roots)."""
    do = d[org][:, None]
    t = tau[:, None]
    delta = (d[None, :] - do) - t          # d_j - w
    sigma = d[None, :] + do + t            # d_j + w
    return 1.0 + np.sum((z * z)[None, :] / (delta * sigma), axis=1)


def secular_roots(d, z, max_iter: int = 400):
    """Roots of Eq. (M-svd-val) by bisection.

    Returns (org, tau, omega): omega_i = d[org_i] + tau_i.
    Reading: origin = the pole nearer to the root, decided by the sign of f
    at the interval midpoint (f increases on each interval).
    """
    d = np.asarray(d, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    N = d.shape[0]
    if N == 0:
        return np.zeros(0, np.int64), np.zeros(0), np.zeros(0)
    zz = float(np.dot(z, z))
    upper = np.empty(N)
    upper[:-1] = d[1:]
    upper[-1] = np.sqrt(d[-1] * d[-1] + zz)
    lower = d.copy()
    # midpoint sign decides the origin
    mid = 0.5 * (lower + upper)
    left = np.ones(N, dtype=bool)           # root in the left half -> origin d_i
    if N > 1:                               # (the last root is measured from d_{N-1})
        left[:-1] = _f_shifted(d, z, np.arange(N - 1), (mid - lower)[:-1]) >= 0.0
    org = np.where(left, np.arange(N), np.minimum(np.arange(N) + 1, N - 1))
    # bracket for tau around the origin
    lo = np.where(left, 0.0, -(upper - mid))
    hi = np.where(left, mid - lower, 0.0)
    # the last interval's length sqrt(d^2 + |z|^2) - d as |z|^2 / (sqrt(d^2 +
    # |z|^2) + d): the difference cancels to 0 when |z|^2 is below d^2 eps
    hi[-1] = zz / (upper[-1] + d[-1]) if zz > 0.0 else 0.0
    for _ in range(max_iter):
        m = 0.5 * (lo + hi)
        moving = (m > lo) & (m < hi)
        if not np.any(moving):
            break
        fm = _f_shifted(d, z, org, m)
        go_left = fm > 0.0
        hi = np.where(moving & go_left, m, hi)
        lo = np.where(moving & ~go_left, m, lo)
    tau = 0.5 * (lo + hi)
    omega = d[org] + tau
    return org.astype(np.int64), tau, omega


def secular_f(d, z, org, tau):
    """Value of f at the given roots and the sum of |terms| (its scale)."""
    d = np.asarray(d, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    do = d[org][:, None]
    t = np.asarray(tau)[:, None]
    den = ((d[None, :] - do) - t) * (d[None, :] + do + t)
    terms = (z * z)[None, :] / den
    return 1.0 + terms.sum(axis=1), 1.0 + np.abs(terms).sum(axis=1)


# --------------------------------------------------------------------------
# Gu-Eisenstat / Loewner recomputation of z (Eq. bdc-zi)
# --------------------------------------------------------------------------
def _w_minus_d(d, org, tau, i):
    """omega_k - d_i for all k, formed as (d_org(k) - d_i) + tau_k."""
    return (d[org] - d[i]) + tau


def lowner_ztilde(d, z, org, tau):
    """z~ of Eq. (bdc-zi).

    |z~_i|^2 = (w_{N-1}^2 - d_i^2) prod_{k<i} (w_k^2 - d_i^2)/(d_k^2 - d_i^2)
                                   prod_{k=i}^{N-2} (w_k^2 - d_i^2)/(d_{k+1}^2 - d_i^2)
    Reading: the sign is that of z_i (the paper leaves it free; M~ must stay
    O(eps)-close to M for the merged vectors to belong to B).
    """
    d = np.asarray(d, dtype=np.float64)
    N = d.shape[0]
    omega = d[org] + tau
    zt = np.empty(N)
    for i in range(N):
        wm = _w_minus_d(d, org, tau, i)          # w_k - d_i
        wp = omega + d[i]                        # w_k + d_i
        w2 = wm * wp                             # w_k^2 - d_i^2
        prod = w2[N - 1]
        for k in range(i):
            prod *= w2[k] / ((d[k] - d[i]) * (d[k] + d[i]))
        for k in range(i, N - 1):
            prod *= w2[k] / ((d[k + 1] - d[i]) * (d[k + 1] + d[i]))
        zt[i] = np.sqrt(abs(prod))
    return np.where(np.asarray(z) < 0.0, -zt, zt)


def m_vectors(d, zt, org, tau):
    """Singular vectors of M~ (Eq. M-svd-vec), columns i = 0..N-1.

    v_i = [z~_j / (d_j^2 - w_i^2)]_j / norm,
    u_i = [-1, d_1 v_i1, ..., d_{N-1} v_i,N-1] / norm   (before normalising v).
    """
    d = np.asarray(d, dtype=np.float64)
    zt = np.asarray(zt, dtype=np.float64)
    N = d.shape[0]
    VM = np.empty((N, N))
    UM = np.empty((N, N))
    for i in range(N):
        o = org[i]
        den = ((d - d[o]) - tau[i]) * (d + d[o] + tau[i])   # d_j^2 - w_i^2
        v = zt / den
        u = d * v
        u[0] = -1.0
        VM[:, i] = v / np.linalg.norm(v)
        UM[:, i] = u / np.linalg.norm(u)
    return UM, VM


# --------------------------------------------------------------------------
# deflation (Sec. 4.2.1, Eq. M-condition and the four N = 3 cases)
# --------------------------------------------------------------------------
def deflation_tol(d, alpha, beta):
    """Reading of 'eps ||M||_2, eps a small multiple of machine precision':
    tol = 8 eps max(max|d|, |alpha|, |beta|, 2^-400).  The floor only matters
    for an all-zero node, where it keeps tol^2 a normal number."""
    return 8.0 * EPS * max(float(np.max(np.abs(d))) if len(d) else 0.0, abs(alpha), abs(beta), 2.0 ** -400)


def deflate(d, z, tol):
    """Deflation of M = [z; 0 diag(d_1..)] with d sorted ascending, d_0 = 0.

    Returns a dict:
      keep     -- indices (into the sorted arrays) of the surviving entries,
                  ascending, always starting with 0
      zkeep    -- z of the survivors after rotations (z_0 clamped to >= tol)
      defl     -- indices of deflated entries, ascending
      dval     -- their singular values (d_i; 0 for the one-sided case)
      rots     -- list of (kind, p, q, c, s) in application order:
                  kind 'R' one-sided on the right vectors only, column 0 and q:
                       V0 <- c V0 + s Vq ; Vq <- -s V0 + c Vq
                  kind 'B' two-sided on both, p deflated into q:
                       Xp <- c Xp - s Xq ; Xq <- s Xp + c Xq
    Reading of the close-value case: entries are scanned in increasing d;
    when the current survivor is within tol of the previous one the previous
    one is zeroed (chains within clusters end on the largest).
    """
    d = np.asarray(d, dtype=np.float64)
    z = np.array(z, dtype=np.float64)
    m = d.shape[0]
    rots = []
    defl, dval = [], []
    if abs(z[0]) < tol:                      # small z_0: clamp up to tol
        z[0] = tol if z[0] >= 0.0 else -tol
    jprev = 0
    for p in range(1, m):
        if abs(z[p]) <= tol:                 # small z_i, i >= 1: set to zero
            z[p] = 0.0
            defl.append(p)
            dval.append(d[p])
            continue
        if jprev == 0 and abs(d[p] - d[0]) <= tol:
            # close to d_0 = 0: right-side rotation zeroes z_p, d_p -> 0
            r = np.hypot(z[0], z[p])
            c, s = z[0] / r, z[p] / r
            z[0], z[p] = r, 0.0
            rots.append(("R", 0, p, c, s))
            defl.append(p)
            dval.append(0.0)
            continue
        if jprev != 0 and abs(d[p] - d[jprev]) <= tol:
            # close pair: two-sided rotation zeroes the earlier z
            r = np.hypot(z[jprev], z[p])
            c, s = z[p] / r, z[jprev] / r
            z[p], z[jprev] = r, 0.0
            rots.append(("B", jprev, p, c, s))
            defl.append(jprev)
            dval.append(d[jprev])
        jprev = p
    order = np.argsort(np.array(defl, dtype=np.int64), kind="stable")
    defl = np.array(defl, dtype=np.int64)[order]
    dval = np.array(dval, dtype=np.float64)[order]
    dset = set(defl.tolist())
    keep = np.array([i for i in range(m) if i not in dset], dtype=np.int64)
    return {"keep": keep, "zkeep": z[keep], "defl": defl, "dval": dval, "rots": rots, "z": z}


def apply_rotations(rots, Ucols, Vcols):
    """Apply the deflation rotations to column blocks (in place, copies in)."""
    U = Ucols.copy()
    V = Vcols.copy()
    for kind, p, q, c, s in rots:
        if kind == "R":
            v0, vq = V[:, p].copy(), V[:, q].copy()
            V[:, p] = c * v0 + s * vq
            V[:, q] = -s * v0 + c * vq
        else:
            for X in (U, V):
                xp, xq = X[:, p].copy(), X[:, q].copy()
                X[:, p] = c * xp - s * xq
                X[:, q] = s * xp + c * xq
    return U, V


# --------------------------------------------------------------------------
# Algorithm 2 end to end
# --------------------------------------------------------------------------
def _rect_leaf(d, e, sqre):
    """SVD of the m x (m+sqre) upper bidiagonal leaf by QR iteration.

    Returns (W, D, Qfull): B = W [diag(D) 0] Qfull^T, Qfull (m+sqre) square;
    for sqre = 1 the last column of Qfull is the right null vector q.
    Reading (the paper only says 'QR iteration'): for sqre = 1 the extra
    column is first rotated away by right rotations, bottom to top.
    """
    from . import bdsqr
    m = d.shape[0]
    d = d.astype(np.float64).copy()
    e = e.astype(np.float64).copy()
    R = np.eye(m + sqre)
    if sqre:
        x = e[m - 1]                          # entry (m-1, m)
        e = e[: m - 1].copy() if m > 1 else np.zeros(0)
        for j in range(m - 1, -1, -1):        # rotate columns (j, m)
            r = np.hypot(d[j], x)
            c, s = (1.0, 0.0) if r == 0.0 else (d[j] / r, x / r)
            d[j] = r
            rj, rm = R[:, j].copy(), R[:, m].copy()
            R[:, j] = c * rj + s * rm
            R[:, m] = -s * rj + c * rm
            if j > 0:
                x = -s * e[j - 1]
                e[j - 1] = c * e[j - 1]
    s, U, VT = bdsqr(d, e[: max(m - 1, 0)]) if m > 0 else (np.zeros(0), np.zeros((0, 0)), np.zeros((0, 0)))
    Qsq = VT.T
    Qfull = R.copy()
    Qfull[:, :m] = R[:, :m] @ Qsq
    return U, s, Qfull


def _node(d, e, sqre, leaf):
    """Recursive BDC of the m x (m+sqre) bidiagonal (d[m], e[m-1+sqre])."""
    m = d.shape[0]
    if m <= leaf:
        return _rect_leaf(d, e, sqre)
    nl = m // 2                               # left child rows; row nl couples
    if nl < 1:
        nl = 1
    nr = m - nl - 1
    alpha, beta = d[nl], e[nl]
    U1, D1, V1 = _node(d[:nl], e[:nl], 1, leaf)
    U2, D2, V2 = _node(d[nl + 1:], e[nl + 1: nl + 1 + nr - 1 + sqre], sqre, leaf)
    return merge(U1, D1, V1, U2, D2, V2, alpha, beta, sqre)


def merge(U1, D1, V1, U2, D2, V2, alpha, beta, sqre):
    """One merge (lasd1 = lasd2 + lasd3) following Sec. 4.2.1.

    Children: B_1 = U1 [D1 0] V1^T (nl x nl+1, last column of V1 = q_1),
              B_2 = U2 [D2 0] V2^T (nr x nr+sqre).
    Node rows: 0..nl-1 (B_1), nl (coupling: alpha at column nl, beta at column
    nl+1), nl+1..m-1 (B_2).
    Reading for two rectangular children (paper silent): the two null-vector
    components alpha*lambda_1 and beta*phi_2 are combined by one rotation into
    z_0; the rotated partner is the node's new null vector q.
    """
    nl, nr = D1.shape[0], D2.shape[0]
    m = nl + 1 + nr
    mc = m + sqre
    # basis columns before deflation (index 0 = the d_0 = 0 column)
    Upre = np.zeros((m, m))
    Vpre = np.zeros((mc, m))
    dpre = np.zeros(m)
    zpre = np.zeros(m)
    Upre[nl, 0] = 1.0
    Upre[:nl, 1:nl + 1] = U1
    Upre[nl + 1:, nl + 1:] = U2
    Vpre[:nl + 1, 1:nl + 1] = V1[:, :nl]
    Vpre[nl + 1:, nl + 1:] = V2[:, :nr]
    dpre[1:nl + 1] = D1
    dpre[nl + 1:] = D2
    zpre[1:nl + 1] = alpha * V1[nl, :nl]
    zpre[nl + 1:] = beta * V2[0, :nr]
    q1 = np.zeros(mc)
    q1[:nl + 1] = V1[:, nl]
    z0 = alpha * V1[nl, nl]
    qnew = None
    if sqre:
        q2 = np.zeros(mc)
        q2[nl + 1:] = V2[:, nr]
        b0 = beta * V2[0, nr]
        r = np.hypot(z0, b0)
        c, s = (1.0, 0.0) if r == 0.0 else (z0 / r, b0 / r)
        Vpre[:, 0] = c * q1 + s * q2
        qnew = -s * q1 + c * q2
        z0 = r
    else:
        Vpre[:, 0] = q1
    zpre[0] = z0
    # sort ascending (index 0 stays first: d_0 = 0 <= all others)
    order = np.argsort(dpre, kind="stable")
    order = np.concatenate(([0], order[order != 0]))
    ds, zs = dpre[order], zpre[order]
    Us, Vs = Upre[:, order], Vpre[:, order]
    tol = deflation_tol(ds, alpha, beta)
    df = deflate(ds, zs, tol)
    Ur, Vr = apply_rotations(df["rots"], Us, Vs)
    keep, defl = df["keep"], df["defl"]
    dk, zk = ds[keep], df["zkeep"]
    org, tau, omega = secular_roots(dk, zk)
    zt = lowner_ztilde(dk, zk, org, tau)
    UM, VM = m_vectors(dk, zt, org, tau)
    Unode = np.zeros((m, m))
    Vnode = np.zeros((mc, mc))
    N = keep.shape[0]
    Unode[:, :N] = Ur[:, keep] @ UM
    Vnode[:, :N] = Vr[:, keep] @ VM
    Unode[:, N:] = Ur[:, defl]
    Vnode[:, N:m] = Vr[:, defl]
    if sqre:
        Vnode[:, m] = qnew
    Dnode = np.concatenate((omega, df["dval"]))
    return Unode, Dnode, Vnode


def bdc_svd(d, e, leaf: int = 16):
    """Algorithm 2: SVD of the n x n upper bidiagonal (d, e), s descending.

    Reading: the input is scaled by max|d, e| before and unscaled after (the
    paper is silent on scaling).  Returns (s, U, VT).
    """
    d = np.asarray(d, dtype=np.float64)
    n = d.shape[0]
    e = np.asarray(e, dtype=np.float64)[: max(n - 1, 0)]
    if n == 0:
        return np.zeros(0), np.zeros((0, 0)), np.zeros((0, 0))
    scale = max(float(np.max(np.abs(d))), float(np.max(np.abs(e))) if e.size else 0.0)
    if scale == 0.0:
        return np.zeros(n), np.eye(n), np.eye(n)
    U, D, V = _node(d / scale, np.concatenate((e / scale, [0.0])), 0, max(int(leaf), 1))
    neg = D < 0.0
    D = np.abs(D)
    V[:, :n][:, neg] *= -1.0
    order = np.argsort(-D, kind="stable")
    return D[order] * scale, U[:, order], V[:, order].T
