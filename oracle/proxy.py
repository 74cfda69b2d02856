"""The learned proxy in float64 (oracle; test infrastructure only).

A small MLP reads each tuple's pooled last-layer document state (saved by the
offline KV-cache creation) and predicts the operator's label; tuples whose
confidence falls below a threshold tau are marked unsure and fall back to the
full KV-cached operator.  That is a two-stage cascade in the sense of the
accept / reject / unsure recurrences of Sec. 4.1: stage 1 (the proxy) decides
the confident tuples, stage 2 (the full operator) the unsure ones.  The paper
uses an embedding filter as its cheap first stage; this proxy plays that role.

Network: ``Linear(d_in, h1) - GELU - Linear(h1, h2) - GELU - Linear(h2, 2)``,
GELU in its erf form, softmax cross-entropy averaged over the batch, Adam with
bias correction.  Parameters are ``W [out][in]`` and ``b [out]``.  Two
precisions: exact contractions, and BF16 contractions with exact accumulation
(the learned-proxy configuration's "BF16, FP32 accum": every matrix product
reads its operands rounded to bfloat16; ``bf=True``).
"""
from __future__ import annotations

from typing import Dict, List

import numpy as np
from scipy.special import erf

F64 = np.float64
_SQRT2 = np.sqrt(2.0)
_INV_SQRT_2PI = 1.0 / np.sqrt(2.0 * np.pi)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / _SQRT2))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / _SQRT2)) + x * _INV_SQRT_2PI * np.exp(-0.5 * x * x)


def bf16(x):
    """Round to the nearest bfloat16 value (ties to even), returned in float64.

    bfloat16 keeps the sign, the 8 exponent bits and the top 7 mantissa bits of
    an IEEE single: the value is first rounded to single precision, then its
    low 16 bits are rounded away (half-way cases to the even upper half)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    out = u.astype(np.uint32).view(np.float32).astype(F64)
    return np.where(np.isfinite(f), out, f.astype(F64))


def _op(a, bf):
    """A contraction operand: as given, or rounded to bfloat16 (BF16 contractions)."""
    return bf16(a) if bf else np.asarray(a, dtype=F64)


def forward(params: Dict[str, np.ndarray], x: np.ndarray, bf: bool = False):
    """Returns (logits [B, 2], cache of pre-activations for backward).

    ``bf``: every contraction reads its two operands rounded to bfloat16 (the
    weights, the input and the GELU outputs); bias, GELU and accumulation stay
    exact."""
    x = np.asarray(x, dtype=F64)
    a1 = _op(x, bf) @ _op(params["w1"], bf).T + params["b1"].astype(F64)
    h1 = gelu(a1)
    a2 = _op(h1, bf) @ _op(params["w2"], bf).T + params["b2"].astype(F64)
    h2 = gelu(a2)
    z = _op(h2, bf) @ _op(params["w3"], bf).T + params["b3"].astype(F64)
    return z, (x, a1, h1, a2, h2)


def softmax(z):
    z = z - z.max(axis=1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=1, keepdims=True)


def loss_and_grads(params, x, y, bf: bool = False):
    """Mean softmax cross-entropy against integer labels y in {0, 1}, and its gradients.

    ``bf``: BF16 contractions, forward and backward -- each product's two
    operands (activation, weight or gradient) rounded to bfloat16; the bias
    gradients (column sums) and the GELU derivative stay exact."""
    y = np.asarray(y, dtype=np.int64)
    z, (x, a1, h1, a2, h2) = forward(params, x, bf)
    B = z.shape[0]
    p = softmax(z)
    loss = -np.mean(np.log(p[np.arange(B), y]))
    dz = p.copy()
    dz[np.arange(B), y] -= 1.0
    dz /= B
    g = {}
    g["w3"] = _op(dz, bf).T @ _op(h2, bf)
    g["b3"] = dz.sum(axis=0)
    dh2 = _op(dz, bf) @ _op(params["w3"], bf)
    da2 = dh2 * gelu_grad(a2)
    g["w2"] = _op(da2, bf).T @ _op(h1, bf)
    g["b2"] = da2.sum(axis=0)
    dh1 = _op(da2, bf) @ _op(params["w2"], bf)
    da1 = dh1 * gelu_grad(a1)
    g["w1"] = _op(da1, bf).T @ _op(x, bf)
    g["b1"] = da1.sum(axis=0)
    return loss, g


class Adam:
    """Adam with bias correction: m, v moments; w -= lr * mhat / (sqrt(vhat) + eps)."""

    def __init__(self, params, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.m = {k: np.zeros_like(v, dtype=F64) for k, v in params.items()}
        self.v = {k: np.zeros_like(v, dtype=F64) for k, v in params.items()}
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        for k in params:
            g = grads[k]
            self.m[k] = self.b1 * self.m[k] + (1.0 - self.b1) * g
            self.v[k] = self.b2 * self.v[k] + (1.0 - self.b2) * g * g
            mhat = self.m[k] / (1.0 - self.b1 ** self.t)
            vhat = self.v[k] / (1.0 - self.b2 ** self.t)
            params[k] = params[k].astype(F64) - self.lr * mhat / (np.sqrt(vhat) + self.eps)
        return params


def train(params, x, y, batches: List[np.ndarray], lr=1e-3, bf: bool = False):
    """Adam over the given mini-batches (index arrays into x, y); returns params, losses."""
    params = {k: np.asarray(v, dtype=F64).copy() for k, v in params.items()}
    opt = Adam(params, lr=lr)
    losses = []
    for bi in batches:
        loss, g = loss_and_grads(params, x[bi], y[bi], bf)
        params = opt.step(params, g)
        losses.append(loss)
    return params, np.array(losses)


def confidence_and_label(params, x, bf: bool = False):
    """Confidence = max softmax probability; proxy label = its argmax (ties -> 0)."""
    z, _ = forward(params, x, bf)
    p = softmax(z)
    return p.max(axis=1), np.argmax(p, axis=1).astype(np.int32)


def cascade(proxy_label, proxy_conf, tau, full_label):
    """Two-stage cascade merge: stage 1 decides where conf >= tau, stage 2 decides the rest.

    ``full_label`` is consulted only where stage 1 is unsure (conf < tau);
    returns (final labels, unsure mask of stage 1).
    """
    unsure = np.asarray(proxy_conf) < tau
    out = np.where(unsure, np.asarray(full_label), np.asarray(proxy_label)).astype(np.int32)
    return out, unsure


def cascade_soft(picks, accepts, rejects, costs=None):
    """Accept / reject / unsure recurrences of Sec. 4.1 for one tuple over a pipeline.

    ``picks[i]`` is the pick factor of operator i (1 or 0 when selected or not;
    a value in [0, 1] in the continuous relaxation); ``accepts[i]`` /
    ``rejects[i]`` are the operator's own (possibly soft) decisions for the tuple.
    Starting from unsure = 1:
    ``accept_i = accept_{i-1} + unsure_{i-1} * pick_i * accepts_i`` (same for reject),
    ``unsure_i = 1 - accept_i - reject_i``.  The per-tuple cost charges operator i
    for the unsure mass it sees, weighted by its pick factor (with picks in
    {0, 1} this is the printed cost equation, where unselected operators are
    skipped).  Returns (accept, reject, unsure, cost).
    """
    acc, rej, uns, cost = 0.0, 0.0, 1.0, 0.0
    for i in range(len(picks)):
        if costs is not None:
            cost += uns * picks[i] * costs[i]
        acc_new = acc + uns * picks[i] * accepts[i]
        rej_new = rej + uns * picks[i] * rejects[i]
        acc, rej = acc_new, rej_new
        uns = 1.0 - acc - rej
    return acc, rej, uns, cost
