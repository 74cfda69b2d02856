"""Alternative retention scores for the scoring ablation, in float64 (oracle;
test infrastructure only).

The paper keeps a query-agnostic retention (Expected Attention, Sec. 5
"Offline: KV Cache Creation") and contrasts it with query-specific pruning
that optimises the cache for one query.  The default score of ``operator.py``
("EA-lite") takes the statistics of the post-RoPE document queries.  This
module adds the two sides of the ablation:

``ea_full_scores`` -- Expected Attention with the RoPE rotation averaged over
    the future positions.  For layer l and kv head g let mu and Sigma be the
    mean and the (population, full) covariance of the PRE-RoPE queries of the
    G query heads of the group over all document positions.  Future queries
    sit at positions L .. L+F-1 (F, the horizon, is a parameter); their
    rotation is replaced by the average Rbar = (1/F) sum_p R(p) of the RoPE
    rotation matrices, so the expected post-RoPE query is Gaussian with mean
    m = Rbar mu and covariance M = Rbar Sigma Rbar^T.  The score of slot j is
    the log of E_q[exp(q . k_j / sqrt(hd))] * ||v_j|| under that Gaussian::

        m . k_j / sqrt(hd) + k_j^T M k_j / (2 hd) + ln(||v_j|| + 1e-12)

    (the moment generating function of a Gaussian; the keys are the stored
    post-RoPE keys).  Parity unpinned against the cited method's own code,
    which the paper does not give; pinned here by the closed form of the
    averaged rotation, a Monte-Carlo estimate of the expectation, and the
    one-position, zero-variance special case.

``query_scores`` -- query-specific: the score of a document slot is the total
    attention probability that the operator's prompt queries (every prompt
    position, every query head of the group) put on it when the prompt is
    forwarded against the full (r = 1) cache, softmax over the document slots
    and the visible prompt keys.  Not reusable across operators: that is the
    contrast the ablation measures.  Pinned against the attention of a
    from-scratch causal pass over document + prompt, and by the uniform case.
"""
from __future__ import annotations

import math

import numpy as np

from .model import F64, attention, attn_out_and_ffn, forward, qkv, rope_inv_freq
from .operator import KVCache


def rope_matrix(p: float, hd: int, theta: float) -> np.ndarray:
    """The RoPE rotation at position p as an explicit [hd, hd] matrix (dimension
    i pairs with i + hd/2; x -> R x)."""
    h = hd // 2
    ang = float(p) * rope_inv_freq(hd, theta)
    R = np.zeros((hd, hd), dtype=F64)
    for i in range(h):
        c, s = math.cos(ang[i]), math.sin(ang[i])
        R[i, i], R[i, i + h] = c, -s
        R[i + h, i], R[i + h, i + h] = s, c
    return R


def avg_rotation(L: int, F: int, hd: int, theta: float) -> np.ndarray:
    """Rbar = mean of rope_matrix(p) over the future positions p = L .. L+F-1."""
    R = np.zeros((hd, hd), dtype=F64)
    for p in range(L, L + F):
        R += rope_matrix(p, hd, theta)
    return R / F


def ea_full_scores(q_pre_group: np.ndarray, k: np.ndarray, v: np.ndarray, L: int, F: int, theta: float):
    """Full Expected Attention scores of every slot of one (layer, kv head).

    q_pre_group: [L, G, hd] pre-RoPE queries of the group; k, v: [L, hd]
    (post-RoPE keys, values).  Returns (scores [L], m [hd], M [hd, hd]).
    """
    hd = k.shape[-1]
    qs = np.asarray(q_pre_group, dtype=F64).reshape(-1, hd)
    mu = qs.mean(axis=0)
    dev = qs - mu
    sigma = dev.T @ dev / qs.shape[0]
    Rbar = avg_rotation(L, F, hd, theta)
    m = Rbar @ mu
    M = Rbar @ sigma @ Rbar.T
    k = np.asarray(k, dtype=F64)
    v = np.asarray(v, dtype=F64)
    quad = np.einsum("ja,ab,jb->j", k, M, k)
    s = (k @ m) / math.sqrt(hd) + quad / (2.0 * hd) + np.log(np.sqrt(np.sum(v * v, axis=1)) + 1e-12)
    return s, m, M


def kv_build_ea_full(cfg, w: dict, doc_tokens, F: int) -> KVCache:
    """``operator.kv_build`` with the full Expected Attention scores (horizon F)."""
    doc_tokens = np.asarray(doc_tokens, dtype=np.int64)
    L = doc_tokens.shape[0]
    xf, per_layer = forward(cfg, w, doc_tokens, collect=True, pre_rope_q=True)
    G = cfg.hq // cfg.hkv
    K, V, S, QS = [], [], [], []
    for (q, k, v, q_pre) in per_layer:
        kl, vl, sl, ql = [], [], [], []
        for g in range(cfg.hkv):
            s, m, M = ea_full_scores(q_pre[:, g * G:(g + 1) * G, :], k[:, g, :], v[:, g, :], L, F,
                                     cfg.rope_theta)
            kl.append(k[:, g, :].copy())
            vl.append(v[:, g, :].copy())
            sl.append(s)
            ql.append((m, M))
        K.append(kl), V.append(vl), S.append(sl), QS.append(ql)
    return KVCache(L, K, V, S, xf.mean(axis=0), QS)


def query_scores(cfg, w: dict, cache: KVCache, prompt):
    """Query-specific scores ``[l][g] -> [L]``: the attention probability the
    prompt's queries put on each document slot, the prompt forwarded against
    the full cache (positions L..L+P-1, the document slots visible to every
    prompt row, the prompt causal on itself)."""
    prompt = np.asarray(prompt, dtype=np.int64)
    P, L = prompt.shape[0], cache.L
    G = cfg.hq // cfg.hkv
    x = w["embed"][prompt].astype(F64)
    pos = np.arange(L, L + P, dtype=F64)
    scale = 1.0 / math.sqrt(cfg.hd)
    out = []
    for l, lw in enumerate(w["layers"]):
        q, k, v = qkv(cfg, lw, x, pos)
        kd = np.stack(cache.k[l], axis=1)            # [L, Hkv, hd]
        vd = np.stack(cache.v[l], axis=1)
        kc = np.concatenate([kd, k], axis=0)
        vc = np.concatenate([vd, v], axis=0)
        vis = np.concatenate([np.ones((P, L), dtype=bool), np.tril(np.ones((P, P), dtype=bool))], axis=1)
        per_g = []
        for g in range(cfg.hkv):
            mass = np.zeros(L, dtype=F64)
            for h in range(g * G, (g + 1) * G):
                s = np.where(vis, (q[:, h, :] @ kc[:, g, :].T) * scale, -np.inf)
                p = np.exp(s - s.max(axis=1, keepdims=True))
                p /= p.sum(axis=1, keepdims=True)
                mass += p[:, :L].sum(axis=0)
            per_g.append(mass)
        out.append(per_g)
        x = attn_out_and_ffn(cfg, lw, x, attention(q, kc, vc, vis))
    return out
