"""FP64 oracle of the learned initializer (test infrastructure only).

Plain numpy restatement of what include/mdhp.h documents for the
initializer: the per-window features (type shares, 32-bin log-gap histograms
per ordered type pair, log N, log T, beta), the 4-layer ReLU MLP, the head and
the training loss with its gradient, and one AdamW step.  The reference is the
exact FP64 function (``bf16=False``): the CPU tests pin it by central finite
differences and closed forms, and the GPU tests compare the BF16 kernels with
it at tolerances derived from BF16 rounding.  ``bf16=True`` rounds inputs,
weights and hidden activations to bfloat16 (round to nearest even) and is kept
only as a diagnostic.  History: this oracle was written after the GPU kernels
of the initializer, unlike the likelihood oracle; its pins stand on their own.
Shares no code with the CUDA path.
"""
from __future__ import annotations

import numpy as np

BINS = 32


def feature_dim(M: int) -> int:
    K = M + BINS * M * M + 3
    return (K + 63) // 64 * 64


def bf16(x):
    """Round float64/float32 values to the nearest bfloat16 (ties to even)."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def layout(M: int, hidden: int):
    """Offsets of W_l [out][in] and b_l [out] in the flat parameter vector."""
    dims = [feature_dim(M), hidden, hidden, hidden, M + M * M]
    off, offs = 0, []
    for l in range(4):
        ow = off
        off += dims[l] * dims[l + 1]
        off = (off + 255) // 256 * 256
        ob = off
        off += dims[l + 1]
        off = (off + 255) // 256 * 256
        offs.append((ow, ob, dims[l], dims[l + 1]))
    return offs, off


def unpack(params, M, hidden):
    offs, _ = layout(M, hidden)
    p = np.asarray(params, dtype=np.float64)
    return [(p[ow:ow + din * dout].reshape(dout, din), p[ob:ob + dout]) for ow, ob, din, dout in offs]


def features(t, ids, T, beta, M):
    """Feature row of one window (float64, before bf16 rounding) and mu_cold."""
    t = np.asarray(t, dtype=np.float64)
    ids = np.asarray(ids, dtype=np.int64)
    N = len(t)
    hist = np.zeros((M, M, BINS))
    last = np.full(M, -np.inf)
    scale = N / T if (T > 0 and N > 0) else 1.0
    n = 0
    while n < N:  # one tie group at a time: members see only strictly earlier events
        g = n
        while g < N and t[g] == t[n]:
            g += 1
        for k in range(n, g):
            i = ids[k]
            for j in range(M):
                if last[j] > -np.inf:
                    gap = (t[k] - last[j]) * scale
                    b = int(np.floor(np.log2(gap))) + BINS // 2 if gap > 0 else 0
                    hist[i, j, min(max(b, 0), BINS - 1)] += 1
        for k in range(n, g):
            last[ids[k]] = t[k]
        n = g
    row = np.zeros(feature_dim(M))
    cnt = np.bincount(ids, minlength=M).astype(np.float64)
    row[:M] = cnt / N if N > 0 else 0.0
    tot = hist.sum(axis=2, keepdims=True)
    h = np.divide(hist, tot, out=np.zeros_like(hist), where=tot > 0)
    row[M:M + M * M * BINS] = h.reshape(-1)
    row[M + M * M * BINS] = np.log(max(N, 1))
    row[M + M * M * BINS + 1] = np.log(T if T > 0 else 1.0)
    row[M + M * M * BINS + 2] = beta
    mu_cold = 0.5 * np.maximum(cnt, 1.0) / T
    return row, mu_cold


def forward(params, X, M, hidden, bf=True):
    """Returns (y, cache); X [B, K] as float."""
    layers = unpack(params, M, hidden)
    r = bf16 if bf else (lambda v: np.asarray(v, dtype=np.float64))
    a = r(X)
    cache = [a]
    h = None
    for l, (W, b) in enumerate(layers):
        h = a @ r(W).T + b
        if l < 3:
            h = np.maximum(h, 0.0)
            a = r(h)
            cache.append((h, a))
        else:
            cache.append((h, None))
    return h, cache


def softplus(x):
    return np.where(x > 20, x, np.log1p(np.exp(np.minimum(x, 20))))


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def loss_and_grad(params, X, mu_cold, beta, mu_t, alpha_t, M, hidden, bf=True):
    """Training loss (mean over windows) and its gradient w.r.t. the flat params.
    beta: [B] or [B, M]; mu_t [B, M], alpha_t [B, M, M]."""
    B = X.shape[0]
    layers = unpack(params, M, hidden)
    r = bf16 if bf else (lambda v: np.asarray(v, dtype=np.float64))
    y, cache = forward(params, X, M, hidden, bf)
    beta = np.asarray(beta, dtype=np.float64)
    bj = np.broadcast_to(beta.reshape(B, -1), (B, M))
    z = np.clip(np.log(np.maximum(mu_t, 1e-20) / mu_cold), -6, 6)
    e_mu = y[:, :M] - z
    # column j of alpha is scaled by beta_j
    bent = np.broadcast_to(bj[:, None, :], (B, M, M)).reshape(B, M * M)
    a = alpha_t.reshape(B, M * M) * M / bent
    ya = y[:, M:M + M * M]
    e_al = softplus(ya) - a
    loss = (np.sum(e_mu ** 2) + np.sum(e_al ** 2)) / B
    dY = np.zeros_like(y)
    dY[:, :M] = 2 * e_mu / B
    dY[:, M:M + M * M] = 2 * e_al * sigmoid(ya) / B
    offs, n = layout(M, hidden)
    g = np.zeros(n)
    d = dY
    for l in range(3, -1, -1):
        W, b = layers[l]
        ow, ob, din, dout = offs[l]
        inp = cache[0] if l == 0 else cache[l][1]
        db_ = r(d)
        g[ow:ow + din * dout] = (db_.T @ inp).reshape(-1)
        g[ob:ob + dout] = d.sum(axis=0)
        if l > 0:
            dh = db_ @ r(W)
            h_prev = cache[l][0]
            d = np.where(h_prev > 0, dh, 0.0)
    return loss, g


def head(y, mu_cold, beta, M):
    B = y.shape[0]
    bj = np.broadcast_to(np.asarray(beta, dtype=np.float64).reshape(B, -1), (B, M))
    mu = mu_cold * np.exp(np.clip(y[:, :M], -6, 6))
    alpha = (bj[:, None, :] / M) * softplus(y[:, M:M + M * M]).reshape(B, M, M)
    return mu, alpha


def adamw_step(params, grad, m, v, step, lr, wd, M, hidden, b1=0.9, b2=0.999, eps=1e-8):
    """One AdamW step; decay on the weight matrices only (biases undecayed)."""
    offs, _ = layout(M, hidden)
    is_mat = np.zeros(len(params), dtype=bool)
    for ow, ob, din, dout in offs:
        is_mat[ow:ow + din * dout] = True
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    c1, c2 = 1 - b1 ** step, 1 - b2 ** step
    w = np.where(is_mat, params - lr * wd * params, params)
    w = w - lr * (m / c1) / (np.sqrt(v / c2) + eps)
    return w, m, v
