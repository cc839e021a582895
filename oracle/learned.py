"""FP64 reference of the learned FastFCA initialiser: features, network, loss and gradients.

TEST INFRASTRUCTURE ONLY (see oracle/fastfca.py): the product path never imports it.  The
GPU path computes the same quantities with BF16 tensor-core products accumulated in FP32;
the tests compare its forward outputs, loss and gradients with these.

The initialiser is not in the paper (its initialisation is mask-based, Sec. VII).  It maps
per-frequency mixture statistics to a starting point (W, L, H) of Algorithm 1:

features phi_f (16 values) of one frequency's frames x_t (t < T):
  R = (1/T) sum_t x_t x_t^H, tr = Re tr R; the M(M+1)/2 upper-triangle entries of R/tr as
  reals (diagonal real parts, then (re, im) of each a < b pair), ln(tr/M), the mean and the
  standard deviation over t of p_t = ln(||x_t||^2 / M), f/(F-1), 1, then zeros to 16.
network: h1 = gelu(W1 phi + b1), h2 = gelu(W2 h1 + b2), o = W3 h2 + b3 (hidden 256,
  gelu(z) = z Phi(z) with the normal CDF Phi).  o[0:2M^2] = W (row-major complex, (re, im)),
  o[2M^2 : 2M^2+MN] = ln L (m-major), o[2M^2+MN : 2M^2+MN+N] = per-source bias b_n of ln v.
per-frame powers: ln v_nt = c_n + b_n + sum_j k_nj q_{t+j-(K-1)/2}, q_t = p_t - mean_t p,
  zero outside [0, T) (a 1-D convolution over t with N output channels, shared weights k, c).
loss of one frequency against a target (W*, L*, H*) from converged FastFCA:
  w-hat = columns scaled to unit norm, with row m of L divided by ||w_m||^2 so that the
  covariances of the model are unchanged; l[m,n] = ln L - mean_m ln L (per n);
  h[n,t] = ln v + mean_m ln L[:, n]  (the scale shared by L[:, n] and H[n, :] removed);
  sigma = the channel permutation minimising sum_m (1 - |w-hat[:, sigma(m)]^H w-hat*[:, m]|^2);
  pi = the source permutation minimising sum_{m,n} (l[sigma(m), pi(n)] - l*[m, n])^2
       + sum_n (mean_t h[pi(n), .] - mean_t h*[n, .])^2  (ties: the first in itertools order);
  loss = sum_m (1 - |...|^2)_sigma + sum_{m,n} (l[sigma(m), pi(n)] - l*[m, n])^2
         + (1/T) sum_{n,t} (h[pi(n), t] - h*[n, t])^2.
The batch loss is the mean over the frequencies of the batch.
prediction (the starting point handed to Algorithm 1): W with unit columns (the loss fixes
  only their directions, and l refers to unit columns), L = exp(ln L), v = exp(ln v).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

D_IN = 16
HIDDEN = 256


def out_dim(M, N):
    return 2 * M * M + M * N + N


def gelu(z):
    return z * 0.5 * (1.0 + np.vectorize(math.erf)(z / math.sqrt(2.0)))


def gelu_grad(z):
    cdf = 0.5 * (1.0 + np.vectorize(math.erf)(z / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    return cdf + z * pdf


def features(x, f, F):
    """phi (16,) and the centred log-power trace q (T,) of one frequency; x (T, M)."""
    x = np.asarray(x, dtype=np.complex128)
    T, M = x.shape
    R = (x.T @ x.conj()) / T
    tr = float(np.real(np.trace(R)))
    Rn = R / tr
    vals = [float(np.real(Rn[a, a])) for a in range(M)]
    for a in range(M):
        for b in range(a + 1, M):
            vals += [float(np.real(Rn[a, b])), float(np.imag(Rn[a, b]))]
    p = np.log((np.abs(x) ** 2).sum(axis=1) / M)
    vals += [math.log(tr / M), float(p.mean()), float(p.std()), f / max(F - 1, 1), 1.0]
    phi = np.zeros(D_IN)
    phi[: len(vals)] = vals
    return phi, p - p.mean()


def forward(params, phi):
    """MLP forward for rows phi (S, 16): returns (o, cache)."""
    W1, b1, W2, b2, W3, b3 = (params[k] for k in ("W1", "b1", "W2", "b2", "W3", "b3"))
    z1 = phi @ W1.T + b1
    h1 = gelu(z1)
    z2 = h1 @ W2.T + b2
    h2 = gelu(z2)
    o = h2 @ W3.T + b3
    return o, (phi, z1, h1, z2, h2)


def backward(params, cache, do):
    """Gradients of the MLP parameters for output gradient do (S, out)."""
    phi, z1, h1, z2, h2 = cache
    g = {}
    g["W3"] = do.T @ h2
    g["b3"] = do.sum(axis=0)
    dh2 = do @ params["W3"]
    dz2 = dh2 * gelu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ params["W2"]
    dz1 = dh1 * gelu_grad(z1)
    g["W1"] = dz1.T @ phi
    g["b1"] = dz1.sum(axis=0)
    return g


def conv_logv(kw, c, b, q):
    """ln v (N, T) from the conv weights kw (N, K), offsets c (N,), biases b (N,), trace q (T,)."""
    N, K = kw.shape
    T = q.shape[0]
    half = (K - 1) // 2
    qp = np.concatenate([np.zeros(half), q, np.zeros(half)])
    out = np.zeros((N, T))
    for n in range(N):
        for j in range(K):
            out[n] += kw[n, j] * qp[j: j + T]
        out[n] += c[n] + b[n]
    return out


def _w_unit(o, M):
    W = (o[0: 2 * M * M: 2] + 1j * o[1: 2 * M * M: 2]).reshape(M, M)
    return W / np.linalg.norm(W, axis=0, keepdims=True), W


def canon_target(W, L, H):
    """Scale-free target (w-hat*, l*, h*) from a converged (W, L, H) of one frequency.

    Scaling column m of W by d scales the variance of w_m^H x by |d|^2, so with unit columns
    row m of L is divided by ||w_m||^2: (w-hat, L', H) give the same covariances as (W, L, H).
    """
    norms = np.linalg.norm(W, axis=0)
    Wn = W / norms[None, :]
    lnL = np.log(L) - 2.0 * np.log(norms)[:, None]
    mean = lnL.mean(axis=0)
    return Wn, lnL - mean[None, :], np.log(H) + mean[:, None]


def choose_perms(o, lnv, target, M, N):
    """(sigma, pi) as defined in the module docstring."""
    Wt, lt, ht = target
    Wh, _ = _w_unit(o, M)
    best = None
    for sig in itertools.permutations(range(M)):
        val = sum(1.0 - abs(Wh[:, sig[m]].conj() @ Wt[:, m]) ** 2 for m in range(M))
        if best is None or val < best[0]:
            best = (val, sig)
    sigma = best[1]
    lnL = o[2 * M * M: 2 * M * M + M * N].reshape(M, N)
    mean = lnL.mean(axis=0)
    lp = lnL - mean[None, :]
    hbar = lnv.mean(axis=1) + mean
    htbar = ht.mean(axis=1)
    best = None
    for pi in itertools.permutations(range(N)):
        val = sum((lp[sigma[m], pi[n]] - lt[m, n]) ** 2 for m in range(M) for n in range(N))
        val += sum((hbar[pi[n]] - htbar[n]) ** 2 for n in range(N))
        if best is None or val < best[0]:
            best = (val, pi)
    return sigma, best[1]


def loss_and_grads(o, lnv, target, M, N):
    """Loss of one frequency and its gradients w.r.t. o (out_dim) and ln v (N, T)."""
    Wt, lt, ht = target
    T = lnv.shape[1]
    sigma, pi = choose_perms(o, lnv, target, M, N)
    do = np.zeros_like(o)
    dlnv = np.zeros_like(lnv)
    loss = 0.0
    # W term: 1 - |u^H t|^2 with u = w / |w|
    Wh, W = _w_unit(o, M)
    for m in range(M):
        col = sigma[m]
        w = W[:, col]
        nw = np.linalg.norm(w)
        u = w / nw
        s = u.conj() @ Wt[:, m]
        loss += 1.0 - abs(s) ** 2
        # f = 1 - |s|^2 with s = u^H t, u = w/|w|:  df/d conj(w_a) = -(conj(s)/|w|) (t_a - s u_a);
        # for a real f the gradient w.r.t. (Re w_a, Im w_a) is 2 (Re, Im) of that.
        for a in range(M):
            gz = -np.conj(s) * (Wt[a, m] - s * u[a]) / nw
            idx = 2 * (a * M + col)
            do[idx] += 2.0 * np.real(gz)
            do[idx + 1] += 2.0 * np.imag(gz)
    # L and H terms
    base = 2 * M * M
    lnL = o[base: base + M * N].reshape(M, N)
    mean = lnL.mean(axis=0)
    lp = lnL - mean[None, :]
    dlp = np.zeros((M, N))
    dmean = np.zeros(N)
    for m in range(M):
        for n in range(N):
            r = lp[sigma[m], pi[n]] - lt[m, n]
            loss += r * r
            dlp[sigma[m], pi[n]] += 2.0 * r
    for n in range(N):
        r = lnv[pi[n]] + mean[pi[n]] - ht[n]
        loss += (r * r).sum() / T
        dlnv[pi[n]] += 2.0 * r / T
        dmean[pi[n]] += 2.0 * r.sum() / T
    # lp = lnL - mean_m lnL ; mean also feeds h
    dlnL = dlp - dlp.mean(axis=0, keepdims=True) + dmean[None, :] / M
    do[base: base + M * N] = dlnL.reshape(-1)
    return loss, do, dlnv, (sigma, pi)


def conv_grads(kw, dlnv, q):
    """Gradients of the conv weights, offsets and per-source biases from d ln v (N, T)."""
    N, K = kw.shape
    T = q.shape[0]
    half = (K - 1) // 2
    qp = np.concatenate([np.zeros(half), q, np.zeros(half)])
    dk = np.zeros_like(kw)
    for n in range(N):
        for j in range(K):
            dk[n, j] = (dlnv[n] * qp[j: j + T]).sum()
    dc = dlnv.sum(axis=1)
    return dk, dc, dlnv.sum(axis=1)


def batch_loss_and_grads(params, conv, phis, qs, targets, M, N):
    """Mean loss over S frequency samples and the gradients of all parameters."""
    S = phis.shape[0]
    o, cache = forward(params, phis)
    base = 2 * M * M + M * N
    do_all = np.zeros_like(o)
    dk = np.zeros_like(conv["k"])
    dc = np.zeros_like(conv["c"])
    total = 0.0
    for s in range(S):
        lnv = conv_logv(conv["k"], conv["c"], o[s, base: base + N], qs[s])
        loss, do, dlnv, _ = loss_and_grads(o[s], lnv, targets[s], M, N)
        total += loss
        dks, dcs, db = conv_grads(conv["k"], dlnv, qs[s])
        dk += dks
        dc += dcs
        do[base: base + N] += db
        do_all[s] = do
    do_all /= S
    g = backward(params, cache, do_all)
    g["k"] = dk / S
    g["c"] = dc / S
    return total / S, g, o


def predict(params, conv, phi, q, M, N):
    """Starting point (W (M, M), L (M, N), H (N, T)) of one frequency from its features."""
    o, _ = forward(params, phi[None, :])
    o = o[0]
    Wn, _ = _w_unit(o, M)
    base = 2 * M * M
    lnL = o[base: base + M * N].reshape(M, N)
    lnv = conv_logv(conv["k"], conv["c"], o[base + M * N: base + M * N + N], q)
    return Wn, np.exp(lnL), np.exp(lnv)
