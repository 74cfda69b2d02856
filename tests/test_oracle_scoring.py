"""Pins of the scoring-ablation oracle (CPU only): the averaged RoPE rotation
against its geometric-series closed form, full Expected Attention against the
Gaussian moment generating function (Monte Carlo), a library covariance and
the one-position zero-variance case, and the query-specific scores against a
from-scratch causal pass over document + prompt and the uniform-attention
closed form."""
import math

import numpy as np
import pytest

from oracle import model as M
from oracle import operator as O
from oracle import scoring as SC
from paper_2602_04430_b300 import synth


def rng(seed=0):
    return np.random.Generator(np.random.PCG64(seed))


def tiny_cfg():
    return synth.ModelConfig(layers=2, d=32, hq=4, hkv=2, hd=8, ffn=48, vocab=64, dtype="f32", name="t")


@pytest.mark.parametrize("L,F", [(1, 1), (7, 5), (300, 64), (2040, 64)])
def test_avg_rotation_closed_form(L, F):
    """Each 2x2 block of the averaged rotation is the complex number
    (1/F) sum_p e^{i p w} = (1/F) e^{i L w} (1 - e^{i F w}) / (1 - e^{i w})."""
    hd, theta = 64, 10000.0
    R = SC.avg_rotation(L, F, hd, theta)
    h = hd // 2
    for i in range(h):
        w_i = theta ** (-2.0 * i / hd)
        e = np.exp(1j * w_i)
        z = np.exp(1j * L * w_i) * (1 - e ** F) / (1 - e) / F
        np.testing.assert_allclose([R[i, i], R[i + h, i], R[i, i + h], R[i + h, i + h]],
                                   [z.real, z.imag, -z.imag, z.real], rtol=1e-8, atol=1e-10)
    # off-pair entries are zero
    mask = np.ones_like(R, dtype=bool)
    for i in range(h):
        mask[[i, i, i + h, i + h], [i, i + h, i, i + h]] = False
    assert np.all(R[mask] == 0.0)


def test_ea_full_one_position_zero_variance():
    """F = 1 and identical document queries: the expected query is that query
    rotated to position L (model.rope, an independent routine) and the
    quadratic term vanishes."""
    g = rng(1)
    hd, L, G = 16, 37, 3
    q0 = g.standard_normal(hd)
    qg = np.tile(q0, (L, G, 1))
    k, v = g.standard_normal((L, hd)), g.standard_normal((L, hd))
    s, m, Mq = SC.ea_full_scores(qg, k, v, L, 1, 10000.0)
    qL = M.rope(q0[None, None, :], np.array([float(L)]), 10000.0)[0, 0]
    np.testing.assert_allclose(m, qL, rtol=1e-12, atol=1e-14)
    assert np.abs(Mq).max() < 1e-24
    ref = k @ qL / math.sqrt(hd) + np.log(np.linalg.norm(v, axis=1) + 1e-12)
    np.testing.assert_allclose(s, ref, rtol=1e-12, atol=1e-12)


def test_ea_full_moments_match_library_covariance():
    """m and M are the mean and the population covariance of the rotated
    queries Rbar q (linearity of the mean; np.cov with bias=True)."""
    g = rng(2)
    hd, L, G, F = 8, 23, 2, 9
    qg = g.standard_normal((L, G, hd)) * 0.7 + 0.3
    k, v = g.standard_normal((L, hd)), g.standard_normal((L, hd))
    _, m, Mq = SC.ea_full_scores(qg, k, v, L, F, 500.0)
    Y = qg.reshape(-1, hd) @ SC.avg_rotation(L, F, hd, 500.0).T
    np.testing.assert_allclose(m, Y.mean(axis=0), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(Mq, np.cov(Y.T, bias=True), rtol=1e-10, atol=1e-13)


def test_ea_full_is_log_expected_exp_monte_carlo():
    """score - ln||v|| = ln E_q[exp(q.k/sqrt(hd))] for q ~ N(m, M): checked by a
    Monte-Carlo estimate (400k draws, tolerance well above its spread)."""
    g = rng(3)
    hd, L, G, F = 8, 40, 2, 6
    qg = g.standard_normal((L, G, hd)) * 0.8
    k, v = g.standard_normal((5, hd)), g.standard_normal((5, hd))
    s, m, Mq = SC.ea_full_scores(qg, np.vstack([k, np.zeros((L - 5, hd))]),
                                 np.vstack([v, np.ones((L - 5, hd))]), L, F, 10000.0)
    w_, U = np.linalg.eigh(Mq)
    A = U * np.sqrt(np.clip(w_, 0, None))
    q = m + g.standard_normal((400_000, hd)) @ A.T
    est = np.log(np.mean(np.exp(q @ k.T / math.sqrt(hd)), axis=0))
    ref = s[:5] - np.log(np.linalg.norm(v, axis=1) + 1e-12)
    np.testing.assert_allclose(est, ref, atol=2e-2)
    # the quadratic term matters at this scale (the test would fail without it)
    assert np.abs(ref - k @ m / math.sqrt(hd)).max() > 0.1


def test_kv_build_ea_full_keeps_cache():
    """The full-EA build changes only the scores: K, V and the pooled state are
    operator.kv_build's."""
    cfg = tiny_cfg()
    w = synth.make_weights(cfg, seed=4, std=0.3)
    doc = rng(5).integers(0, cfg.vocab, 19)
    a, b = O.kv_build(cfg, w, doc), SC.kv_build_ea_full(cfg, w, doc, 8)
    for l in range(cfg.layers):
        for g in range(cfg.hkv):
            np.testing.assert_array_equal(a.k[l][g], b.k[l][g])
            np.testing.assert_array_equal(a.v[l][g], b.v[l][g])
            assert a.scores[l][g].shape == b.scores[l][g].shape
    np.testing.assert_array_equal(a.pooled, b.pooled)


def _scratch_prompt_mass(cfg, w, doc, prompt):
    """Attention mass of the last P rows on the first L columns in one causal
    pass over document + prompt (no cache)."""
    seq = np.concatenate([doc, prompt]).astype(np.int64)
    n, L, P = len(seq), len(doc), len(prompt)
    G = cfg.hq // cfg.hkv
    x = w["embed"][seq].astype(np.float64)
    pos = np.arange(n, dtype=np.float64)
    mask = M.causal_mask(n)
    out = []
    for lw in w["layers"]:
        q, k, v = M.qkv(cfg, lw, x, pos)
        per_g = []
        for g in range(cfg.hkv):
            tot = np.zeros(L)
            for h in range(g * G, (g + 1) * G):
                sc = np.where(mask, q[:, h, :] @ k[:, g, :].T / math.sqrt(cfg.hd), -np.inf)
                p = np.exp(sc - sc.max(axis=1, keepdims=True))
                p /= p.sum(axis=1, keepdims=True)
                tot += p[L:, :L].sum(axis=0)
            per_g.append(tot)
        out.append(per_g)
        x = M.attn_out_and_ffn(cfg, lw, x, M.attention(q, k, v, mask))
    return out


def test_query_scores_equal_from_scratch_attention():
    cfg = tiny_cfg()
    w = synth.make_weights(cfg, seed=6, std=0.3)
    g = rng(7)
    for L, P in ((1, 3), (17, 5)):
        doc, prompt = g.integers(0, cfg.vocab, L), g.integers(0, cfg.vocab, P)
        qs = SC.query_scores(cfg, w, O.kv_build(cfg, w, doc), prompt)
        ref = _scratch_prompt_mass(cfg, w, doc, prompt)
        for l in range(cfg.layers):
            for gg in range(cfg.hkv):
                np.testing.assert_allclose(qs[l][gg], ref[l][gg], rtol=1e-11, atol=1e-14)
                G = cfg.hq // cfg.hkv
                assert 0 < qs[l][gg].sum() < G * P


def test_query_scores_uniform_when_queries_vanish():
    """Zero query weights: every visible key gets probability 1/(L + p + 1) at
    prompt row p, so each document slot gets G * sum_p 1/(L + p + 1)."""
    cfg = tiny_cfg()
    w = synth.make_weights(cfg, seed=8, std=0.3)
    for lw in w["layers"]:
        lw["wq"] = np.zeros_like(lw["wq"])
    L, P = 11, 4
    g = rng(9)
    doc, prompt = g.integers(0, cfg.vocab, L), g.integers(0, cfg.vocab, P)
    qs = SC.query_scores(cfg, w, O.kv_build(cfg, w, doc), prompt)
    G = cfg.hq // cfg.hkv
    want = G * sum(1.0 / (L + p + 1) for p in range(P))
    for l in range(cfg.layers):
        for gg in range(cfg.hkv):
            np.testing.assert_allclose(qs[l][gg], np.full(L, want), rtol=1e-13)
