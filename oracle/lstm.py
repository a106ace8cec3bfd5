"""FP64 oracle of the MDHP-LSTM cell (test infrastructure only).

Plain numpy forward pass and backpropagation through time of the cell of the
paper's MDHP-LSTM equation (Sec. "MDHP-LSTM"), for sequences b = 0..B-1 of L
steps, inputs x [B][L][D], hidden size H:

  hks  = tanh(A vec(alpha) - Bm (beta T_span) + C mu)        one per sequence
  i    = sigmoid(W_i x_t + U_i h_{t-1} + b_i)
  f    = sigmoid(W_f x_t + U_f h_{t-1} + b_f)
  g    = tanh   (W_c x_t + U_c h_{t-1} + b_c)                (the paper's c~)
  o    = sigmoid(W_o x_t + U_o h_{t-1} + b_o)
  c_t  = hks * (f * c_{t-1} + i * g)
  h_t  = o * tanh(c_t)
  y_t  = Wy h_t
with h_{-1} = c_{-1} = 0.  W [4H][D], U [4H][H], b [4H] stack the gates in
the order i, f, g, o.  alpha [B][M][M] (row-major vec), beta [B][nb] (nb = 1
or M: beta T_span is a vector of nb values), mu [B][M] (the paper's theta),
A [H][M*M], Bm [H][nb], C [H][M], Wy [O][H].

Readings: the paper indexes the step's input as x^{t-1} and writes y^t = Wy
h^{t-1}; here step t consumes x_t and emits y_t = Wy h_t (the standard cell).

`forward` returns the outputs and a cache; `backward` the gradients of
sum(y * dy) with respect to every input.  The CPU tests pin both against
central finite differences.  Shares no code with the CUDA path.
"""
from __future__ import annotations

import numpy as np


def _sig(z):
    with np.errstate(over="ignore"):  # exp(-z) = inf for very negative z: sigmoid 0
        return 1.0 / (1.0 + np.exp(-z))


def forward(x, mu, alpha, beta, T, W, U, b, A, Bm, C, Wy):
    x = np.asarray(x, np.float64)
    B_, L, D = x.shape
    H = U.shape[1]
    vecA = np.asarray(alpha, np.float64).reshape(B_, -1)
    bT = np.asarray(beta, np.float64).reshape(B_, -1) * np.asarray(T, np.float64).reshape(B_, 1)
    pre_h = vecA @ A.T - bT @ Bm.T + np.asarray(mu, np.float64) @ C.T
    hks = np.tanh(pre_h)
    h = np.zeros((B_, H))
    c = np.zeros((B_, H))
    hs, cs, gates, ys = [], [], [], []
    for t in range(L):
        z = x[:, t] @ W.T + h @ U.T + b
        i, f, g, o = _sig(z[:, :H]), _sig(z[:, H:2 * H]), np.tanh(z[:, 2 * H:3 * H]), _sig(z[:, 3 * H:])
        c = hks * (f * c + i * g)
        h = o * np.tanh(c)
        hs.append(h); cs.append(c); gates.append(np.concatenate([i, f, g, o], axis=1)); ys.append(h @ Wy.T)
    y = np.stack(ys, axis=1)
    cache = dict(x=x, vecA=vecA, bT=bT, mu=np.asarray(mu, np.float64), hks=hks, h=np.stack(hs, 1),
                 c=np.stack(cs, 1), gates=np.stack(gates, 1), W=W, U=U, A=A, Bm=Bm, C=C, Wy=Wy,
                 beta=np.asarray(beta, np.float64).reshape(B_, -1), T=np.asarray(T, np.float64))
    return y, cache


def backward(cache, dy):
    """Gradients of sum(y * dy)."""
    x, hks, hs, cs, G = cache["x"], cache["hks"], cache["h"], cache["c"], cache["gates"]
    W, U, Wy = cache["W"], cache["U"], cache["Wy"]
    B_, L, D = x.shape
    H = U.shape[1]
    dy = np.asarray(dy, np.float64)
    dW = np.zeros_like(W); dU = np.zeros_like(U); db = np.zeros(4 * H); dWy = np.zeros_like(Wy)
    dx = np.zeros_like(x)
    dhks = np.zeros((B_, H))
    dh_next = np.zeros((B_, H)); dc_next = np.zeros((B_, H))
    for t in range(L - 1, -1, -1):
        i, f, g, o = G[:, t, :H], G[:, t, H:2 * H], G[:, t, 2 * H:3 * H], G[:, t, 3 * H:]
        c = cs[:, t]
        c_prev = cs[:, t - 1] if t > 0 else np.zeros((B_, H))
        h_prev = hs[:, t - 1] if t > 0 else np.zeros((B_, H))
        dWy += dy[:, t].T @ hs[:, t]
        dh = dh_next + dy[:, t] @ Wy
        tc = np.tanh(c)
        dc = dc_next + dh * o * (1 - tc ** 2)
        do = dh * tc
        inner = f * c_prev + i * g
        dhks += dc * inner
        dinner = dc * hks
        di, df, dg = dinner * g, dinner * c_prev, dinner * i
        dz = np.concatenate([di * i * (1 - i), df * f * (1 - f), dg * (1 - g ** 2), do * o * (1 - o)], 1)
        dW += dz.T @ x[:, t]
        dU += dz.T @ h_prev
        db += dz.sum(0)
        dx[:, t] = dz @ W
        dh_next = dz @ U
        dc_next = dinner * f
    dpre = dhks * (1 - hks ** 2)
    dA = dpre.T @ cache["vecA"]
    dBm = -dpre.T @ cache["bT"]
    dC = dpre.T @ cache["mu"]
    dalpha = (dpre @ cache["A"]).reshape(B_, -1)
    dbT = -(dpre @ cache["Bm"])
    dbeta = dbT * cache["T"].reshape(B_, 1)
    dmu = dpre @ cache["C"]
    return dict(dx=dx, dW=dW, dU=dU, db=db, dA=dA, dBm=dBm, dC=dC, dWy=dWy, dmu=dmu,
                dalpha=dalpha, dbeta=dbeta)
