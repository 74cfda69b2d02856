"""The KV-cache semantic operator, step by step in float64 (oracle; test infrastructure only).

Steps, in the paper's order (Sec. 5):

1. ``kv_build``  -- offline KV-cache creation: each tuple's document is run
   through the decoder once (causal prefill at positions 0..L-1); the post-RoPE
   keys and values of every layer and kv head are kept, together with the
   retention scores and the pooled last-layer document state (input of the
   learned proxy).
2. ``n_keep`` / ``retain``  -- query-agnostic compression to a retained
   fraction r (compression ratio 1 - r, Sec. 6 "Operators"): per (layer, kv
   head) the n_keep(L, r) slots with the highest score are kept, in rank order
   (score descending, index ascending on ties).
3. ``op_eval``  -- online execution: the operator's prompt is appended after
   the cached document (positions L..L+P-1) and forwarded through the decoder
   attending to the retained cache; the logits of the label tokens are read at
   the last prompt position.
4. ``decide_filter`` / ``decide_classify``  -- the filter decision from the
   log-odds of the '1'/'0' label tokens with thresholds theta+ / theta-
   (Sec. 5 "Online: Query Execution"; soft-threshold equation of Sec. 4.1 at
   temperature 0); the classify generalisation is an argmax over biased label
   logits.

Retention score ("EA-lite", parity unpinned against the cited Expected
Attention method, whose formula the paper does not give): for layer l and kv
head g let mu and sigma^2 be the per-dimension mean and population variance of
the post-RoPE queries of the G query heads of the group over all document
positions.  The score of slot j with key k_j and value v_j is the logarithm of
``E_q[exp(q . k_j / sqrt(hd))] * ||v_j||`` for q ~ N(mu, diag sigma^2)::

    mu . k_j / sqrt(hd) + sum_c sigma_c^2 k_jc^2 / (2 hd) + ln(||v_j|| + 1e-12)
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence

import numpy as np

from . import fp8 as _fp8
from .model import (F64, attention, attn_out_and_ffn, forward, label_logits, qkv,
                    rmsnorm)

ACCEPT, REJECT, UNSURE = 1, 0, 2


class KVCache:
    """Per-tuple cache: ``k[l][g]``, ``v[l][g]`` are ``[L, hd]`` float64 arrays
    (post-RoPE, original slot order); ``scores[l][g]`` is ``[L]``; ``pooled`` is
    ``[d]``; ``qstats[l][g] = (mu, sigma2)``."""

    def __init__(self, L, k, v, scores, pooled, qstats):
        self.L, self.k, self.v, self.scores, self.pooled, self.qstats = L, k, v, scores, pooled, qstats


def ea_scores(q_group: np.ndarray, k: np.ndarray, v: np.ndarray):
    """EA-lite scores of every slot of one (layer, kv head).

    q_group: [L, G, hd] post-RoPE queries of the group; k, v: [L, hd].
    Returns (scores [L], mu [hd], sigma2 [hd]).
    """
    hd = k.shape[-1]
    qs = np.asarray(q_group, dtype=F64).reshape(-1, hd)
    mu = qs.mean(axis=0)
    sigma2 = ((qs - mu) ** 2).mean(axis=0)
    k = np.asarray(k, dtype=F64)
    v = np.asarray(v, dtype=F64)
    s = (k @ mu) / math.sqrt(hd) + (k * k) @ sigma2 / (2.0 * hd) \
        + np.log(np.sqrt(np.sum(v * v, axis=1)) + 1e-12)
    return s, mu, sigma2


def kv_build(cfg, w: dict, doc_tokens) -> KVCache:
    """Offline KV-cache creation for one document (Sec. 5, "Offline: KV Cache Creation")."""
    doc_tokens = np.asarray(doc_tokens, dtype=np.int64)
    L = doc_tokens.shape[0]
    xf, per_layer = forward(cfg, w, doc_tokens, collect=True)
    G = cfg.hq // cfg.hkv
    K, V, S, QS = [], [], [], []
    for (q, k, v) in per_layer:
        kl, vl, sl, ql = [], [], [], []
        for g in range(cfg.hkv):
            s, mu, s2 = ea_scores(q[:, g * G:(g + 1) * G, :], k[:, g, :], v[:, g, :])
            kl.append(k[:, g, :].copy())
            vl.append(v[:, g, :].copy())
            sl.append(s)
            ql.append((mu, s2))
        K.append(kl), V.append(vl), S.append(sl), QS.append(ql)
    pooled = xf.mean(axis=0)
    return KVCache(L, K, V, S, pooled, QS)


def n_keep(L: int, r: float) -> int:
    """Retained slot count: clamp(floor(r*L + 0.5), 1, L), r taken as the IEEE double of the given value."""
    if not (r > 0.0 and r <= 1.0):
        raise ValueError("retention r must lie in (0, 1]")
    rl = float(r) * float(L)          # one rounding, then the add: no fused multiply-add
    n = math.floor(rl + 0.5)
    return int(min(max(n, 1), L))


def rank_order(scores: np.ndarray) -> np.ndarray:
    """All slot indices sorted by (score descending, index ascending)."""
    scores = np.asarray(scores)
    if np.isnan(scores).any():
        raise ValueError("NaN retention score")
    idx = np.arange(scores.shape[0])
    return np.lexsort((idx, -scores.astype(np.float64)))


def retain(scores: np.ndarray, r: float) -> np.ndarray:
    """Indices of the retained slots, in rank order (Sec. 5, query-agnostic compression)."""
    return rank_order(scores)[: n_keep(len(scores), r)]


def retained_kv(cache: KVCache, r: float, idx: Optional[list] = None, kv_fp8: bool = False,
                fp8_arith: str = "f64", fp8_profile_r: Optional[float] = None):
    """Gather the retained keys / values of every (layer, kv head).

    ``idx[l][g]`` overrides the retained index lists (to evaluate the operator on
    an externally chosen set); ``kv_fp8`` replaces each by its per-block E4M3
    dequantisation.

    ``fp8_profile_r`` (with ``kv_fp8``): the operator reads an E4M3 profile
    retained at this larger ratio (one profile shared by operators of smaller
    r, the retained sets being nested prefixes of one rank order, Sec. 5): the
    64-slot blocks and their scales are those of the profile's set, quantised
    first, and the operator reads the first n_keep(L, r) of its rows (the last
    block's scale then covers slots the operator does not read).  ``idx``, if
    given, holds the profile's sets.
    """
    Kr, Vr, I = [], [], []
    for l in range(len(cache.k)):
        kl, vl, il = [], [], []
        for g in range(len(cache.k[l])):
            r_set = fp8_profile_r if (kv_fp8 and fp8_profile_r is not None) else r
            sel = retain(cache.scores[l][g], r_set) if idx is None else np.asarray(idx[l][g])
            k = cache.k[l][g][sel]
            v = cache.v[l][g][sel]
            if kv_fp8:
                k = _fp8.quantize_blocks(k, fp8_arith)[2]
                v = _fp8.quantize_blocks(v, fp8_arith)[2]
            if r_set != r:
                n = n_keep(cache.L, r)
                sel, k, v = sel[:n], k[:n], v[:n]
            kl.append(k), vl.append(v), il.append(sel)
        Kr.append(kl), Vr.append(vl), I.append(il)
    return Kr, Vr, I


def op_eval(cfg, w: dict, L: int, Kr, Vr, prompt, label_ids) -> np.ndarray:
    """Online evaluation of one operator on one tuple (Sec. 5, "Online: Query Execution").

    ``Kr[l][g]`` / ``Vr[l][g]``: retained post-RoPE keys / values ``[n, hd]``
    (any order); ``L``: the document length (the prompt sits at positions
    L..L+P-1 whatever was pruned).  Returns the label logits ``[n_labels]``.
    """
    return label_logits(w, prompt_state(cfg, w, L, Kr, Vr, prompt), label_ids)


def prompt_state(cfg, w: dict, L: int, Kr, Vr, prompt) -> np.ndarray:
    """Final-normed hidden state of the last prompt position, the prompt sitting
    at positions L..L+P-1 after the retained cache (visible to every prompt row)
    and attending causally to itself."""
    prompt = np.asarray(prompt, dtype=np.int64)
    P = prompt.shape[0]
    x = w["embed"][prompt].astype(F64)
    pos = np.arange(L, L + P, dtype=F64)
    for l, lw in enumerate(w["layers"]):
        q, k, v = qkv(cfg, lw, x, pos)
        n = Kr[l][0].shape[0]
        # cached slots first (visible to every prompt row), then the prompt's own keys (causal)
        kc = np.concatenate([np.stack(Kr[l], axis=1), k], axis=0)
        vc = np.concatenate([np.stack(Vr[l], axis=1), v], axis=0)
        vis = np.concatenate([np.ones((P, n), dtype=bool), np.tril(np.ones((P, P), dtype=bool))],
                             axis=1)
        o = attention(q, kc, vc, vis)
        x = attn_out_and_ffn(cfg, lw, x, o)
    return rmsnorm(x[-1], cfg.eps)


def map_eval(cfg, w: dict, L: int, Kr, Vr, prompt, n_gen: int):
    """The map operator (Sec. 6 "Operators": generate a value per item), greedy:
    token t is the argmax over the vocabulary (ties to the lowest id) of the
    logits at the last position of prompt + tokens 0..t-1; it sits at the next
    position.  Returns (tokens [n_gen], logits [n_gen, V])."""
    seq, toks, logs = list(np.asarray(prompt, dtype=np.int64)), [], []
    w_lm = w["w_lm"].astype(F64)
    for _ in range(n_gen):
        z = w_lm @ prompt_state(cfg, w, L, Kr, Vr, seq)
        t = int(np.argmax(z))
        toks.append(t), logs.append(z), seq.append(t)
    return toks, np.stack(logs)


def map_eval_from_scratch(cfg, w: dict, doc_tokens, prompt, n_gen: int):
    """The same greedy decode without any cache: each step runs document, prompt
    and the tokens so far in one causal pass."""
    seq = list(np.asarray(doc_tokens, dtype=np.int64)) + list(np.asarray(prompt, dtype=np.int64))
    toks, logs = [], []
    w_lm = w["w_lm"].astype(F64)
    for _ in range(n_gen):
        z = w_lm @ forward(cfg, w, np.asarray(seq))[-1]
        t = int(np.argmax(z))
        toks.append(t), logs.append(z), seq.append(t)
    return toks, np.stack(logs)


def op_eval_from_scratch(cfg, w: dict, doc_tokens, prompt, label_ids) -> np.ndarray:
    """The same label logits computed without any cache: document and prompt in one causal pass."""
    seq = np.concatenate([np.asarray(doc_tokens, dtype=np.int64), np.asarray(prompt, dtype=np.int64)])
    xf = forward(cfg, w, seq)
    return label_logits(w, xf[-1], label_ids)


def decide_filter(z_accept: float, z_reject: float, theta_pos: float, theta_neg: float) -> int:
    """Accept / reject / unsure from the log-odds s = z('1') - z('0').

    Temperature-0 form of softmax[s - theta+, theta- - s, 0]: the largest entry
    wins; ties go to unsure, then reject.
    """
    s = z_accept - z_reject
    a, rj, u = s - theta_pos, theta_neg - s, 0.0
    if u >= a and u >= rj:
        return UNSURE
    if rj >= a:
        return REJECT
    return ACCEPT


def decide_classify(z: Sequence[float], bias: Optional[Sequence[float]] = None) -> int:
    """argmax_k (z_k + b_k), ties to the lowest k."""
    z = np.asarray(z, dtype=F64)
    if bias is not None:
        z = z + np.asarray(bias, dtype=F64)
    return int(np.argmax(z))


def decide(op, z) -> int:
    if op.kind == "classify":
        return decide_classify(z, op.bias)
    return decide_filter(float(z[0]), float(z[1]), op.theta_pos, op.theta_neg)


def cascade_stages(decisions: List[List[int]]):
    """Multi-stage cascade (Sec. 4.1 with any number of stages): stage k is
    consulted for a tuple only if every earlier stage left it UNSURE; the first
    stage that accepts or rejects decides; the last stage's UNSURE stays UNSURE.

    ``decisions[k][i]`` is stage k's decision for input position i (only read
    for the tuples that reach stage k).  Returns (labels, deciding stage,
    number of tuples sent to each stage)."""
    n = len(decisions[0]) if decisions else 0
    labels, stage = [UNSURE] * n, [0] * n
    counts = [0] * len(decisions)
    for i in range(n):
        for k, dk in enumerate(decisions):
            counts[k] += 1
            labels[i], stage[i] = dk[i], k
            if dk[i] != UNSURE:
                break
    return labels, stage, counts


def run_table(cfg, w, table, op, tuples: Optional[List[int]] = None, kv_fp8: bool = False,
              caches: Optional[dict] = None):
    """kv_build -> retain(r) -> op_eval -> decision for the selected tuples of a table.

    Returns (logits [n][n_labels], labels [n], caches).
    """
    tok, off = table["tokens"], table["offsets"]
    T = len(off) - 1
    tuples = list(range(T)) if tuples is None else list(tuples)
    caches = {} if caches is None else caches
    Z, D = [], []
    for t in tuples:
        if t not in caches:
            caches[t] = kv_build(cfg, w, tok[off[t]:off[t + 1]])
        c = caches[t]
        Kr, Vr, _ = retained_kv(c, op.r, kv_fp8=kv_fp8)
        z = op_eval(cfg, w, c.L, Kr, Vr, op.prompt, op.label_ids)
        Z.append(z)
        D.append(decide(op, z))
    return np.array(Z), np.array(D, dtype=np.int32), caches
