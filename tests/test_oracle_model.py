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


# ---------------------------------------------------------------- decoder block
# The two functions that compose a layer (qkv_pre, attn_out_and_ffn) are pinned
# against (a) a 2-element case worked out by hand with scalar arithmetic and
# (b) a pre-norm Llama block written independently from torch.nn.functional
# primitives in float64 (RoPE there as a complex rotation of the (i, i + hd/2)
# pairs, attention by scaled_dot_product_attention with grouped kv heads).
# Planted mistakes -- gate / up swapped, the FFN reading the pre-attention
# residual, a projection applied transposed -- must each fail them.

def _hand_cfg():
    return synth.ModelConfig(layers=1, d=2, hq=1, hkv=1, hd=2, ffn=2, vocab=4, dtype="f32",
                             name="hand", eps=1e-5)


_HAND_LW = {
    "wo": np.array([[1.0, 2.0], [3.0, 4.0]]),      # [out][in]
    "wg": np.array([[1.0, 0.0], [0.5, -1.0]]),
    "wu": np.array([[0.5, 0.5], [1.0, 0.0]]),
    "wd": np.array([[2.0, -1.0], [0.0, 1.0]]),
}


def _hand_expected():
    """x = (1, -2), attention output o = (0.5, 0.25), weights above, eps 1e-5."""
    sg = lambda t: t / (1.0 + math.exp(-t))
    # residual after the output projection: x + Wo o
    x0 = 1.0 + (1.0 * 0.5 + 2.0 * 0.25)          # 2.0
    x1 = -2.0 + (3.0 * 0.5 + 4.0 * 0.25)         # 0.5
    inv = 1.0 / math.sqrt((x0 * x0 + x1 * x1) / 2.0 + 1e-5)
    h0, h1 = x0 * inv, x1 * inv
    g0, g1 = 1.0 * h0 + 0.0 * h1, 0.5 * h0 - 1.0 * h1
    u0, u1 = 0.5 * h0 + 0.5 * h1, 1.0 * h0 + 0.0 * h1
    a0, a1 = sg(g0) * u0, sg(g1) * u1
    return np.array([x0 + (2.0 * a0 - 1.0 * a1), x1 + (0.0 * a0 + 1.0 * a1)])


def test_swiglu_residual_hand_case():
    cfg = _hand_cfg()
    out = M.attn_out_and_ffn(cfg, _HAND_LW, np.array([[1.0, -2.0]]), np.array([[[0.5, 0.25]]]))
    np.testing.assert_allclose(out[0], _hand_expected(), rtol=1e-14, atol=1e-15)


def test_swiglu_hand_case_catches_a_gate_up_swap():
    cfg = _hand_cfg()
    lw = dict(_HAND_LW, wg=_HAND_LW["wu"], wu=_HAND_LW["wg"])
    out = M.attn_out_and_ffn(cfg, lw, np.array([[1.0, -2.0]]), np.array([[[0.5, 0.25]]]))
    assert np.abs(out[0] - _hand_expected()).max() > 1e-3


def _torch_rope(x, pos, theta):
    """x [n, H, hd] float64 torch; rotate-half pairs as complex numbers a + i b."""
    hd = x.shape[-1]
    half = hd // 2
    inv = theta ** (-torch.arange(0, half, dtype=torch.float64) * 2.0 / hd)
    ang = pos[:, None].to(torch.float64) * inv[None, :]
    rot = torch.polar(torch.ones_like(ang), ang)[:, None, :]           # e^{i ang}
    z = torch.complex(x[..., :half], x[..., half:]) * rot
    return torch.cat([z.real, z.imag], dim=-1)


def _torch_llama_layer(cfg, lw, x, pos, kv_prefix=None):
    """One pre-norm Llama block in torch float64.  ``kv_prefix`` = (K, V) of
    cached slots [m, Hkv, hd] visible to every row; the rows attend causally to
    themselves.  Returns (x_out, q, k, v) with q/k post-RoPE."""
    F = torch.nn.functional
    t = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64))
    n = x.shape[0]
    h = F.rms_norm(x, (cfg.d,), eps=cfg.eps)
    q = F.linear(h, t(lw["wq"])).view(n, cfg.hq, cfg.hd)
    k = F.linear(h, t(lw["wk"])).view(n, cfg.hkv, cfg.hd)
    v = F.linear(h, t(lw["wv"])).view(n, cfg.hkv, cfg.hd)
    q, k = _torch_rope(q, pos, cfg.rope_theta), _torch_rope(k, pos, cfg.rope_theta)
    kc, vc = k, v
    mask = torch.tril(torch.ones(n, n, dtype=torch.bool))
    if kv_prefix is not None:
        kc = torch.cat([kv_prefix[0], k], 0)
        vc = torch.cat([kv_prefix[1], v], 0)
        mask = torch.cat([torch.ones(n, kv_prefix[0].shape[0], dtype=torch.bool), mask], 1)
    o = F.scaled_dot_product_attention(q.transpose(0, 1)[None], kc.transpose(0, 1)[None],
                                       vc.transpose(0, 1)[None], attn_mask=mask, enable_gqa=True)
    o = o[0].transpose(0, 1).reshape(n, cfg.hq * cfg.hd)
    x = x + F.linear(o, t(lw["wo"]))
    h = F.rms_norm(x, (cfg.d,), eps=cfg.eps)
    x = x + F.linear(F.silu(F.linear(h, t(lw["wg"]))) * F.linear(h, t(lw["wu"])), t(lw["wd"]))
    return x, q, k, v


def _block_cfg():
    # q width (Hq*hd = 48) differs from d (40), so a transposed projection cannot go unnoticed
    return synth.ModelConfig(layers=2, d=40, hq=6, hkv=2, hd=8, ffn=56, vocab=64, dtype="f32",
                             name="blk")


def test_decoder_layer_matches_torch_llama_block():
    cfg = _block_cfg()
    w = synth.make_weights(cfg, seed=21, std=0.3)
    r = rng(22)
    x = r.standard_normal((7, cfg.d))
    pos = np.arange(3, 10, dtype=np.float64)
    for lw in w["layers"]:
        xt, qt, kt, vt = _torch_llama_layer(cfg, lw, torch.from_numpy(x), torch.from_numpy(pos))
        q_pre, k_pre, v = M.qkv_pre(cfg, lw, x)
        q, k = M.rope(q_pre, pos, cfg.rope_theta), M.rope(k_pre, pos, cfg.rope_theta)
        np.testing.assert_allclose(q, qt.numpy(), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(k, kt.numpy(), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(v, vt.numpy(), rtol=1e-12, atol=1e-12)
        o = M.attention(q, k, v, M.causal_mask(len(x)))
        out = M.attn_out_and_ffn(cfg, lw, x, o)
        np.testing.assert_allclose(out, xt.numpy(), rtol=1e-12, atol=1e-12)
        x = out


def test_forward_and_cached_prompt_match_torch_llama_stack():
    """Whole stack: the oracle's causal forward over a document and its cached
    prompt state against the torch block applied layer by layer."""
    from oracle import operator as O
    cfg = _block_cfg()
    w = synth.make_weights(cfg, seed=23, std=0.3)
    doc = rng(24).integers(0, cfg.vocab, 9)
    prompt = rng(25).integers(0, cfg.vocab, 4)
    xt = torch.from_numpy(w["embed"][doc].astype(np.float64))
    pos = torch.arange(len(doc), dtype=torch.float64)
    kvs = []
    for lw in w["layers"]:
        xt, _, k, v = _torch_llama_layer(cfg, lw, xt, pos)
        kvs.append((k, v))
    ref = torch.nn.functional.rms_norm(xt, (cfg.d,), eps=cfg.eps).numpy()
    np.testing.assert_allclose(M.forward(cfg, w, doc), ref, rtol=1e-12, atol=1e-12)
    # the prompt after the cache: positions L..L+P-1, every cached slot visible
    xp = torch.from_numpy(w["embed"][prompt].astype(np.float64))
    pp = torch.arange(len(doc), len(doc) + len(prompt), dtype=torch.float64)
    for lw, kv in zip(w["layers"], kvs):
        xp, _, _, _ = _torch_llama_layer(cfg, lw, xp, pp, kv_prefix=kv)
    ref_last = torch.nn.functional.rms_norm(xp[-1], (cfg.d,), eps=cfg.eps).numpy()
    c = O.kv_build(cfg, w, doc)
    Kr, Vr, _ = O.retained_kv(c, 1.0)
    np.testing.assert_allclose(O.prompt_state(cfg, w, c.L, Kr, Vr, prompt), ref_last,
                               rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("mistake", ["gate_up_swap", "ffn_reads_pre_attention_residual",
                                     "output_projection_transposed", "ffn_without_norm"])
def test_planted_block_mistakes_fail_the_torch_pin(monkeypatch, mistake):
    """Each planted mistake in the oracle's block makes it disagree with the
    torch block by far more than the pin's tolerance."""
    cfg = _block_cfg()
    if mistake == "output_projection_transposed":
        cfg = synth.ModelConfig(layers=1, d=48, hq=6, hkv=2, hd=8, ffn=56, vocab=64, dtype="f32",
                                name="blk_sq")    # Wo square, so the transposed product runs
    w = synth.make_weights(cfg, seed=26, std=0.3)
    lw = w["layers"][0]
    x = rng(27).standard_normal((5, cfg.d))
    pos = np.arange(5, dtype=np.float64)
    xt = _torch_llama_layer(cfg, lw, torch.from_numpy(x), torch.from_numpy(pos))[0].numpy()
    good = M.attn_out_and_ffn

    def planted(cfg_, lw_, x_, o_):
        n = x_.shape[0]
        if mistake == "gate_up_swap":
            return good(cfg_, dict(lw_, wg=lw_["wu"], wu=lw_["wg"]), x_, o_)
        if mistake == "output_projection_transposed":
            return good(cfg_, dict(lw_, wo=lw_["wo"].T.copy()), x_, o_)
        xa = x_ + o_.reshape(n, -1) @ lw_["wo"].T
        src = x_ if mistake == "ffn_reads_pre_attention_residual" else xa
        h = src if mistake == "ffn_without_norm" else M.rmsnorm(src, cfg_.eps)
        return xa + (M.silu(h @ lw_["wg"].T) * (h @ lw_["wu"].T)) @ lw_["wd"].T

    monkeypatch.setattr(M, "attn_out_and_ffn", planted)
    q_pre, k_pre, v = M.qkv_pre(cfg, lw, x)
    q, k = M.rope(q_pre, pos, cfg.rope_theta), M.rope(k_pre, pos, cfg.rope_theta)
    out = M.attn_out_and_ffn(cfg, lw, x, M.attention(q, k, v, M.causal_mask(5)))
    assert np.abs(out - xt).max() > 1e-6, mistake
