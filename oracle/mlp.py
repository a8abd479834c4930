"""Oracle of the root-start estimate and its MLP: features, analytic
estimate, network, loss gradient, Adam.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  The paper has no
learned component; what is written out here is the extension the library
adds to the secular solve of Eq. (M-svd-val): a start point for each root,
made of an analytic local estimate y_q and a small network g that corrects
it, and the training that fits g.  Everything is numpy FP64 and follows the
plain definitions:

* ``analytic(d, z, i)`` -- y_q: in t = (w^2 - d_i^2) / D2 the secular
  function is c(t) - a/t + b/(1-t) (a = z_i^2/D2, b = z_{i+1}^2/D2, c = 1 +
  the other poles' terms); c frozen at the interval midpoint m gives a
  quadratic whose root in (0, 1) is y_q = ln(t/(1-t)).  c is the exact sum
  over the 8 nearest other poles on each side plus, for the farther poles
  of each side, the second-order moment estimate M/(mu - m^2) (1 + var/(mu -
  m^2)^2) of their sum (M = sum z^2, mu, var = z^2-weighted mean and
  variance of d^2).
* ``features(d, z, i)`` -- the eleven network inputs (see the function).
* ``logit(d, omega, i)`` -- y = ln(t / (1 - t)) of a converged root;
  ``target`` = y - y_q clamped to [-40, 40], what the network learns.
* ``forward`` / ``loss_and_grad`` -- the 11 -> 64 -> 64 -> 1 tanh network
  and the gradient of loss = mean h(g - r) (h = Huber with threshold
  ``huber``, or r^2/2 when huber <= 0) by the chain rule, layer by layer.
  Pinned by central finite differences of ``loss`` (tests).
* ``adam_step`` -- one Adam update with bias correction (Kingma & Ba, 2015);
  the normalisation entries are left alone.

Parameter layout (one flat vector, the same as the library's):
  [0, 11) means, [11, 22) inverse deviations, W1 64x11, b1 64, W2 64x64,
  b2 64, W3 64, b3.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, NEAR = 11, 64, 8
OFF_MEAN, OFF_ISTD = 0, N_IN
OFF_W1 = 2 * N_IN
OFF_B1 = OFF_W1 + N_H * N_IN
OFF_W2 = OFF_B1 + N_H
OFF_B2 = OFF_W2 + N_H * N_H
OFF_W3 = OFF_B2 + N_H
OFF_B3 = OFF_W3 + N_H
N_PARAMS = OFF_B3 + 1


def _clamp(v):
    return float(min(40.0, max(-40.0, v)))


def _log(v):
    return np.log(v) if v > 0 else -np.inf


def _far(z2, d2, m2):
    """Second-moment estimate of sum z2 / (d2 - m2) over one far side."""
    M = float(np.sum(z2))
    if not M > 0:
        return 0.0
    mu = float(np.sum(z2 * d2)) / M
    var = max(float(np.sum(z2 * d2 * d2)) / M - mu * mu, 0.0)
    den = mu - m2
    if den == 0.0:
        return 0.0
    return M / den * (1.0 + var / (den * den))


def background(d, z, i):
    """(near, far): the exact sum of z_j^2 / (d_j^2 - m^2) over the other
    poles within NEAR places of the interval, and the moment estimate of the
    rest (j <= i-NEAR-1 and j >= i+NEAR+2), m the interval midpoint."""
    d = np.asarray(d, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    N = d.shape[0]
    m = 0.5 * (d[i] + d[i + 1])
    near = 0.0
    for j in range(max(i - NEAR, 0), min(i + 1 + NEAR, N - 1) + 1):
        if j not in (i, i + 1):
            near += z[j] ** 2 / ((d[j] - m) * (d[j] + m))
    L = np.arange(0, max(i - NEAR, 0))
    R = np.arange(i + NEAR + 2, N)
    far = _far(z[L] ** 2, d[L] ** 2, m * m) + _far(z[R] ** 2, d[R] ** 2, m * m)
    return near, far


def analytic(d, z, i):
    """y_q of root i (unclamped, limited to +-700)."""
    d = np.asarray(d, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    D2 = (d[i + 1] - d[i]) * (d[i + 1] + d[i])
    a, b = z[i] ** 2 / D2, z[i + 1] ** 2 / D2
    near, far = background(d, z, i)
    c = 1.0 + near + far
    # c t^2 - (c + a + b) t + a = 0: the root in (0, 1) and s = 1 - t (which
    # solves -c s^2 - (a + b - c) s + b = 0), each by the form without
    # cancellation for the sign of its linear coefficient
    p, q = c + a + b, a + b - c
    rp = np.sqrt(max(p * p - 4 * c * a, 0.0))
    rq = np.sqrt(max(q * q + 4 * c * b, 0.0))
    t = 2 * a / (p + rp) if p >= 0 else (p - rp) / (2 * c)
    s = 2 * b / (q + rq) if q >= 0 else (q - rq) / (-2 * c)
    y = _log(t) - _log(s)
    if not np.isfinite(y):
        y = 700.0 if y > 0 else -700.0
    return float(min(700.0, max(-700.0, y)))


def features(d, z, i):
    """The eleven inputs of root i (0 <= i < N-1), rho = sum z^2, D2 =
    d_{i+1}^2 - d_i^2, gap_k = d_{k+1} - d_k, a = z_i^2/D2, b = z_{i+1}^2/D2:

      f0 = ln a   f1 = ln b   f2 = ln(rho / D2)
      f3 = ln(gap_{i-1}/gap_i)   (0 when i = 0)
      f4 = ln(gap_{i+1}/gap_i)   (0 when i = N-2)
      f5 = ln(z_{i-1}^2 / D2)    (-40 when i = 0)
      f6 = ln(z_{i+2}^2 / D2)    (-40 when i = N-2)
      f7 = asinh(near)   f8 = asinh(far)   (``background``)
      f9 = y_q           f10 = d_i / d_{i+1}
    each clamped to [-40, 40]."""
    d = np.asarray(d, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    N = d.shape[0]
    assert 0 <= i < N - 1
    dl, du = d[i], d[i + 1]
    D2 = (du - dl) * (du + dl)
    gap = du - dl
    rho = float(np.sum(z * z))
    near, far = background(d, z, i)
    f = np.empty(N_IN)
    f[0] = _clamp(_log(z[i] ** 2 / D2))
    f[1] = _clamp(_log(z[i + 1] ** 2 / D2))
    f[2] = _clamp(_log(rho / D2))
    f[3] = _clamp(_log((dl - d[i - 1]) / gap)) if i >= 1 else 0.0
    f[4] = _clamp(_log((d[i + 2] - du) / gap)) if i + 2 < N else 0.0
    f[5] = _clamp(_log(z[i - 1] ** 2 / D2)) if i >= 1 else -40.0
    f[6] = _clamp(_log(z[i + 2] ** 2 / D2)) if i + 2 < N else -40.0
    f[7] = _clamp(np.arcsinh(near))
    f[8] = _clamp(np.arcsinh(far))
    f[9] = _clamp(analytic(d, z, i))
    f[10] = dl / du
    return f


def all_features(d, z):
    N = len(d)
    return np.array([features(d, z, i) for i in range(N - 1)]).reshape(-1, N_IN)


def logit(d, omega, i):
    """y = ln(t / (1 - t)), t = (omega_i^2 - d_i^2) / (d_{i+1}^2 - d_i^2)."""
    dl, du, w = d[i], d[i + 1], omega[i]
    a = (w - dl) * (w + dl)
    b = (du - w) * (du + w)
    return float(_log(a) - _log(b))


def target(d, z, omega, i):
    """The network's training target y - y_q, clamped to [-40, 40]."""
    return _clamp(logit(d, omega, i) - analytic(d, z, i))


def unpack(P):
    P = np.asarray(P, dtype=np.float64)
    return dict(
        mean=P[OFF_MEAN:OFF_MEAN + N_IN], istd=P[OFF_ISTD:OFF_ISTD + N_IN],
        W1=P[OFF_W1:OFF_B1].reshape(N_H, N_IN), b1=P[OFF_B1:OFF_W2],
        W2=P[OFF_W2:OFF_B2].reshape(N_H, N_H), b2=P[OFF_B2:OFF_W3],
        W3=P[OFF_W3:OFF_B3], b3=P[OFF_B3])


def forward(P, X):
    """g for feature rows X (S x N_IN) and the intermediate activations."""
    p = unpack(P)
    Xn = (np.asarray(X, dtype=np.float64) - p["mean"]) * p["istd"]
    H1 = np.tanh(Xn @ p["W1"].T + p["b1"])
    H2 = np.tanh(H1 @ p["W2"].T + p["b2"])
    y = H2 @ p["W3"] + p["b3"]
    return y, (Xn, H1, H2)


def _huber(r, huber):
    """Loss terms and their derivatives in r."""
    if huber <= 0:
        return 0.5 * r * r, r
    big = np.abs(r) > huber
    val = np.where(big, huber * (np.abs(r) - 0.5 * huber), 0.5 * r * r)
    der = np.where(big, huber * np.sign(r), r)
    return val, der


def loss(P, X, y, huber=0.0):
    yhat, _ = forward(P, X)
    r = yhat - np.asarray(y, dtype=np.float64)
    return float(np.mean(_huber(r, huber)[0]))


def loss_and_grad(P, X, y, huber=0.0):
    """loss = mean_s h(yhat_s - y_s) and d loss / d P (the normalisation
    entries get 0)."""
    p = unpack(P)
    yhat, (Xn, H1, H2) = forward(P, X)
    S = Xn.shape[0]
    r = yhat - np.asarray(y, dtype=np.float64)
    val, der = _huber(r, huber)
    L = float(np.mean(val))
    g_y = der / S                                 # d L / d yhat
    g_W3 = H2.T @ g_y
    g_b3 = np.sum(g_y)
    g_Z2 = np.outer(g_y, p["W3"]) * (1.0 - H2 * H2)
    g_W2 = g_Z2.T @ H1
    g_b2 = g_Z2.sum(axis=0)
    g_Z1 = (g_Z2 @ p["W2"]) * (1.0 - H1 * H1)
    g_W1 = g_Z1.T @ Xn
    g_b1 = g_Z1.sum(axis=0)
    G = np.zeros(N_PARAMS)
    G[OFF_W1:OFF_B1] = g_W1.ravel()
    G[OFF_B1:OFF_W2] = g_b1
    G[OFF_W2:OFF_B2] = g_W2.ravel()
    G[OFF_B2:OFF_W3] = g_b2
    G[OFF_W3:OFF_B3] = g_W3
    G[OFF_B3] = g_b3
    return L, G


def adam_step(P, G, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update of entries [OFF_W1, N_PARAMS); returns new (P, m, v)."""
    P = np.array(P, dtype=np.float64)
    m = np.array(m, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    s = slice(OFF_W1, N_PARAMS)
    m[s] = b1 * m[s] + (1 - b1) * G[s]
    v[s] = b2 * v[s] + (1 - b2) * G[s] ** 2
    mh = m[s] / (1 - b1 ** step)
    vh = v[s] / (1 - b2 ** step)
    P[s] = P[s] - lr * mh / (np.sqrt(vh) + eps)
    return P, m, v
