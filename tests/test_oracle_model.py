"""Pins of the oracle's decoder primitives (CPU only).

Each check compares the oracle with something other than itself: torch fp64
library routines, hand-computed closed forms, or invariants of the mathematics.
"""
import math

import numpy as np
import pytest
import torch

from oracle import model as M
from paper_2602_04430_b300 import synth


def rng(seed=0):
    return np.random.Generator(np.random.PCG64(seed))


def test_rmsnorm_matches_torch_and_hand_case():
    x = rng().standard_normal((7, 33))
    ref = torch.nn.functional.rms_norm(torch.from_numpy(x), (33,), eps=1e-5).numpy()
    np.testing.assert_allclose(M.rmsnorm(x, 1e-5), ref, rtol=1e-14, atol=1e-14)
    # (3, 4): mean square 12.5
    v = M.rmsnorm(np.array([3.0, 4.0]), 0.0)
    np.testing.assert_allclose(v, [3 / math.sqrt(12.5), 4 / math.sqrt(12.5)], rtol=1e-15)


def test_silu_matches_torch():
    x = np.linspace(-30, 30, 1001)
    np.testing.assert_allclose(M.silu(x), torch.nn.functional.silu(torch.from_numpy(x)).numpy(),
                               rtol=1e-13, atol=1e-300)


def test_rope_hand_cases():
    # hd = 2: one pair rotated by angle pos * theta^0 = pos
    x = np.array([[[0.3, -1.2]]])
    for p in (0.0, 1.0, 5.5):
        out = M.rope(x, np.array([p]), 10000.0)[0, 0]
        np.testing.assert_allclose(out, [0.3 * math.cos(p) + 1.2 * math.sin(p),
                                         -1.2 * math.cos(p) + 0.3 * math.sin(p)], rtol=1e-14)
    # hd = 4, theta = 100: frequencies (1, 0.1); pairs are (0, 2) and (1, 3)
    x = np.array([[[1.0, 2.0, 3.0, 4.0]]])
    p = 2.0
    out = M.rope(x, np.array([p]), 100.0)[0, 0]
    a0, a1 = p * 1.0, p * 0.1
    exp = [1 * math.cos(a0) - 3 * math.sin(a0), 2 * math.cos(a1) - 4 * math.sin(a1),
           3 * math.cos(a0) + 1 * math.sin(a0), 4 * math.cos(a1) + 2 * math.sin(a1)]
    np.testing.assert_allclose(out, exp, rtol=1e-14)


def test_rope_relative_position_and_norm():
    r = rng(1)
    q = r.standard_normal((1, 1, 64))
    k = r.standard_normal((1, 1, 64))
    def dot(m, n):
        return float(np.sum(M.rope(q, np.array([m]), 1e4) * M.rope(k, np.array([n]), 1e4)))
    for delta in (0.0, 17.0, 1000.0):
        assert abs(dot(5 + delta, 2 + delta) - dot(5, 2)) < 1e-11
    np.testing.assert_allclose(np.linalg.norm(M.rope(q, np.array([123.0]), 1e4)),
                               np.linalg.norm(q), rtol=1e-14)


def _sdpa_ref(q, k, v, vis):
    # torch fp64 scaled_dot_product_attention with the kv heads repeated per group
    G = q.shape[1] // k.shape[1]
    qt = torch.from_numpy(q).permute(1, 0, 2)[None]
    kt = torch.from_numpy(np.repeat(k, G, axis=1)).permute(1, 0, 2)[None]
    vt = torch.from_numpy(np.repeat(v, G, axis=1)).permute(1, 0, 2)[None]
    o = torch.nn.functional.scaled_dot_product_attention(qt, kt, vt, attn_mask=torch.from_numpy(vis))
    return o[0].permute(1, 0, 2).numpy()


def test_attention_matches_torch_sdpa_gqa():
    r = rng(2)
    nq, nk, hq, hkv, hd = 9, 23, 8, 2, 16
    q, k, v = (r.standard_normal((nq, hq, hd)), r.standard_normal((nk, hkv, hd)),
               r.standard_normal((nk, hkv, hd)))
    vis = r.random((nq, nk)) < 0.6
    vis[:, 0] = True
    np.testing.assert_allclose(M.attention(q, k, v, vis), _sdpa_ref(q, k, v, vis),
                               rtol=1e-12, atol=1e-13)


def test_attention_two_key_closed_form():
    hd = 4
    q = np.array([[[1.0, 0, 0, 0]]])
    k = np.array([[[2.0, 0, 0, 0]], [[0.0, 0, 0, 0]]])
    v = np.array([[[1.0, 0, 0, 0]], [[0.0, 1, 0, 0]]])
    o = M.attention(q, k, v, np.ones((1, 2), dtype=bool))[0, 0]
    w1 = 1.0 / (1.0 + math.exp(-(2.0 / math.sqrt(hd))))
    np.testing.assert_allclose(o, [w1, 1 - w1, 0, 0], rtol=1e-14)
    # a single visible key returns its value
    o = M.attention(q, k, v, np.array([[False, True]]))[0, 0]
    np.testing.assert_allclose(o, [0, 1, 0, 0], atol=0)


def _tiny_cfg(hq=4, hkv=2):
    return synth.ModelConfig(layers=2, d=32, hq=hq, hkv=hkv, hd=8, ffn=48, vocab=64,
                             dtype="f32", name="t")


def test_gqa_mapping_is_h_div_g():
    """A GQA model equals the MHA model whose kv head h is the GQA kv head h // G."""
    cfg = _tiny_cfg(4, 2)
    w = synth.make_weights(cfg, seed=3, std=0.2)
    cfg_mha = _tiny_cfg(4, 4)
    w_mha = {"embed": w["embed"], "w_lm": w["w_lm"], "layers": []}
    for lw in w["layers"]:
        l2 = dict(lw)
        for key in ("wk", "wv"):
            blocks = lw[key].reshape(2, cfg.hd, cfg.d)
            l2[key] = np.concatenate([blocks[h // 2] for h in range(4)], axis=0)
        w_mha["layers"].append(l2)
    toks = rng(4).integers(0, 64, 11)
    np.testing.assert_allclose(M.forward(cfg, w, toks), M.forward(cfg_mha, w_mha, toks),
                               rtol=1e-12, atol=1e-12)


def test_zero_blocks_reduce_to_embedding_head():
    """With Wo = Wd = 0 every layer is the identity: logits = W_lm[labels] . rmsnorm(E[last])."""
    cfg = _tiny_cfg()
    w = synth.make_weights(cfg, seed=5, std=0.2)
    for lw in w["layers"]:
        lw["wo"] = np.zeros_like(lw["wo"])
        lw["wd"] = np.zeros_like(lw["wd"])
    toks = rng(6).integers(0, 64, 9)
    xf = M.forward(cfg, w, toks)
    e = w["embed"][toks[-1]].astype(np.float64)
    e = e / math.sqrt(float(np.mean(e * e)) + cfg.eps)
    z = M.label_logits(w, xf[-1], [3, 7])
    np.testing.assert_allclose(z, [w["w_lm"][3] @ e, w["w_lm"][7] @ e], rtol=1e-12)


def test_forward_is_causal():
    cfg = _tiny_cfg()
    w = synth.make_weights(cfg, seed=7, std=0.2)
    toks = rng(8).integers(0, 64, 12)
    a = M.forward(cfg, w, toks)
    toks2 = toks.copy()
    toks2[8:] = (toks2[8:] + 1) % 64
    b = M.forward(cfg, w, toks2)
    np.testing.assert_array_equal(a[:8], b[:8])
    assert np.abs(a[8:] - b[8:]).max() > 1e-6
