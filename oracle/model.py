"""Llama-style decoder primitives in float64 (oracle; test infrastructure only).

The paper runs Llama-3.1 models (Sec. 6, "Operators") and does not restate the
architecture; the primitives below are the standard pre-norm decoder with the
readings fixed for this project:

* RMSNorm without gains: ``x / sqrt(mean(x^2) + eps)``, eps = 1e-5.
* RoPE, "rotate-half" pairing of dimension i with i + hd/2, frequency
  ``theta^(-2i/hd)``, theta = 10000.
* Attention scaled by ``1/sqrt(hd)``; grouped-query mapping of query head h to
  key/value head ``h // G`` with ``G = Hq / Hkv``.
* SwiGLU FFN ``(silu(h Wg^T) * (h Wu^T)) Wd^T``.
Weights are ``[out][in]``, so a projection is ``x @ W.T``.
"""
from __future__ import annotations

import numpy as np

F64 = np.float64


def rmsnorm(x: np.ndarray, eps: float) -> np.ndarray:
    """Root-mean-square normalisation over the last axis (no gain)."""
    x = np.asarray(x, dtype=F64)
    return x / np.sqrt(np.mean(x * x, axis=-1, keepdims=True) + eps)


def rope_inv_freq(hd: int, theta: float) -> np.ndarray:
    """Frequencies theta^(-2i/hd), i = 0 .. hd/2-1."""
    i = np.arange(hd // 2, dtype=F64)
    return np.power(F64(theta), -2.0 * i / hd)


def rope(x: np.ndarray, pos: np.ndarray, theta: float) -> np.ndarray:
    """Rotate ``x[n, H, hd]`` by the angles ``pos[n] * inv_freq``.

    Dimension i and i + hd/2 form one rotation pair:
    ``(a, b) -> (a cos - b sin, b cos + a sin)``.
    """
    x = np.asarray(x, dtype=F64)
    hd = x.shape[-1]
    ang = np.asarray(pos, dtype=F64)[:, None] * rope_inv_freq(hd, theta)[None, :]
    c = np.cos(ang)[:, None, :]
    s = np.sin(ang)[:, None, :]
    a = x[..., : hd // 2]
    b = x[..., hd // 2:]
    return np.concatenate([a * c - b * s, b * c + a * s], axis=-1)


def silu(x: np.ndarray) -> np.ndarray:
    return x / (1.0 + np.exp(-x))


def attention(q: np.ndarray, k: np.ndarray, v: np.ndarray, visible: np.ndarray) -> np.ndarray:
    """Grouped-query softmax attention.

    q: [nq, Hq, hd]; k, v: [nk, Hkv, hd]; visible: bool [nq, nk] (same mask for
    every head).  Query head h reads key/value head h // (Hq/Hkv).
    Returns [nq, Hq, hd].  Every query row must see at least one key.
    """
    nq, hq, hd = q.shape
    hkv = k.shape[1]
    g = hq // hkv
    out = np.empty((nq, hq, hd), dtype=F64)
    scale = 1.0 / np.sqrt(F64(hd))
    for h in range(hq):
        kv = h // g
        s = (q[:, h, :] @ k[:, kv, :].T) * scale
        s = np.where(visible, s, -np.inf)
        m = np.max(s, axis=1, keepdims=True)
        p = np.exp(s - m)
        p = p / np.sum(p, axis=1, keepdims=True)
        out[:, h, :] = p @ v[:, kv, :]
    return out


def qkv_pre(cfg, lw: dict, x: np.ndarray):
    """Pre-norm projections of one layer, before RoPE: q [n, Hq, hd], k and v [n, Hkv, hd]."""
    h = rmsnorm(x, cfg.eps)
    n = x.shape[0]
    q = (h @ lw["wq"].T.astype(F64)).reshape(n, cfg.hq, cfg.hd)
    k = (h @ lw["wk"].T.astype(F64)).reshape(n, cfg.hkv, cfg.hd)
    v = (h @ lw["wv"].T.astype(F64)).reshape(n, cfg.hkv, cfg.hd)
    return q, k, v


def qkv(cfg, lw: dict, x: np.ndarray, pos: np.ndarray):
    """Pre-norm projections of one layer with RoPE applied to q and k."""
    q, k, v = qkv_pre(cfg, lw, x)
    return rope(q, pos, cfg.rope_theta), rope(k, pos, cfg.rope_theta), v


def attn_out_and_ffn(cfg, lw: dict, x: np.ndarray, o: np.ndarray) -> np.ndarray:
    """Residual add of the attention output projection, then the SwiGLU FFN block."""
    n = x.shape[0]
    x = x + o.reshape(n, cfg.hq * cfg.hd) @ lw["wo"].T.astype(F64)
    h = rmsnorm(x, cfg.eps)
    gate = h @ lw["wg"].T.astype(F64)
    up = h @ lw["wu"].T.astype(F64)
    return x + (silu(gate) * up) @ lw["wd"].T.astype(F64)


def causal_mask(n: int) -> np.ndarray:
    return np.tril(np.ones((n, n), dtype=bool))


def forward(cfg, w: dict, tokens: np.ndarray, collect: bool = False, pre_rope_q: bool = False):
    """Causal forward pass over ``tokens`` at positions 0..n-1.

    Returns the final-normed hidden states ``[n][d]``; with ``collect`` also the
    per-layer post-RoPE (q, k, v), and with ``pre_rope_q`` as well the
    per-layer queries before RoPE: entries (q, k, v, q_pre).
    """
    tokens = np.asarray(tokens, dtype=np.int64)
    n = tokens.shape[0]
    x = w["embed"][tokens].astype(F64)
    pos = np.arange(n, dtype=F64)
    mask = causal_mask(n)
    per_layer = []
    for lw in w["layers"]:
        q_pre, k_pre, v = qkv_pre(cfg, lw, x)
        q, k = rope(q_pre, pos, cfg.rope_theta), rope(k_pre, pos, cfg.rope_theta)
        if collect:
            per_layer.append((q, k, v, q_pre) if pre_rope_q else (q, k, v))
        o = attention(q, k, v, mask)
        x = attn_out_and_ffn(cfg, lw, x, o)
    xf = rmsnorm(x, cfg.eps)
    return (xf, per_layer) if collect else xf


def label_logits(w: dict, xf_last: np.ndarray, label_ids) -> np.ndarray:
    """Logits of the label tokens only: rows ``label_ids`` of the LM head."""
    return w["w_lm"][np.asarray(label_ids, dtype=np.int64)].astype(F64) @ xf_last
