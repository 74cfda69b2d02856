"""The seeded input generators follow the stated recipe: bfloat16 rounding is
round-to-nearest-even (torch's cast), weights are N(0, 0.02^2) in the
documented draw order, table lengths follow the configured lognormal or
bounded-Zipf law inside their bounds, token ids follow Zipf(1.1) over ranks,
a smaller table is a prefix of the larger one, and every draw is reproducible
from its seed.  Statistical checks use the exact distribution (pmf sums,
quantiles) on samples large enough for tight bounds."""
import math

import numpy as np

from paper_2602_04430_b300 import synth


def test_bf16_rounding_matches_torch_including_ties():
    import torch
    rng = np.random.Generator(np.random.PCG64(1))
    a = (rng.standard_normal(100000) * 3).astype(np.float32)
    # exact ties: the low 16 bits 0x8000 with an even and an odd kept mantissa
    ties = np.array([0x3F808000, 0x3F818000, 0xBF808000, 0x40490000 | 0x8000], dtype=np.uint32).view(np.float32)
    a = np.concatenate([a, ties, np.array([0.0, -0.0, 1e-40, 3.0e38], dtype=np.float32)])
    got = synth.to_bf16_f32(a)
    want = torch.from_numpy(a).to(torch.bfloat16).float().numpy()
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    assert not np.any(got.view(np.uint32) & 0xFFFF)


def test_weights_distribution_and_draw_order():
    cfg = synth.MODELS["tiny_f32"]
    w1 = synth.make_weights(cfg, seed=11)
    w2 = synth.make_weights(cfg, seed=11)
    assert np.array_equal(w1["embed"], w2["embed"]) and np.array_equal(w1["w_lm"], w2["w_lm"])
    # the documented order: embed first, then layer 0's wq from the same stream
    rng = np.random.Generator(np.random.PCG64(11))
    e = rng.standard_normal((cfg.vocab, cfg.d), dtype=np.float32) * np.float32(0.02)
    q = rng.standard_normal((cfg.hq * cfg.hd, cfg.d), dtype=np.float32) * np.float32(0.02)
    assert np.array_equal(w1["embed"], e) and np.array_equal(w1["layers"][0]["wq"], q)
    allw = np.concatenate([w1["embed"].ravel(), w1["w_lm"].ravel()] +
                          [m.ravel() for L in w1["layers"] for m in L.values()])
    n = allw.size
    assert abs(allw.mean()) < 4 * 0.02 / math.sqrt(n)
    assert abs(allw.std() / 0.02 - 1) < 4 / math.sqrt(2 * n)
    # a bf16 model's weights are bf16 values
    cb = synth.ModelConfig(layers=1, d=64, hq=2, hkv=1, hd=32, ffn=128, vocab=256, dtype="bf16")
    wb = synth.make_weights(cb, seed=3)
    assert not np.any(wb["layers"][0]["wd"].view(np.uint32) & 0xFFFF)


def test_lognormal_lengths_follow_the_c2_recipe():
    t = synth.make_table(synth.TABLES["c2"], 32000, seed=1000)
    L = t["lengths"]
    assert len(L) == 4096 and L.min() >= 64 and L.max() <= 2048
    assert np.array_equal(np.diff(t["offsets"]), L) and t["offsets"][0] == 0
    assert len(t["tokens"]) == t["offsets"][-1]
    # median: the clipping bounds lie outside the central mass, so the sample
    # median estimates exp(mu) = 512; its standard error is about
    # sigma * 512 * sqrt(pi / 2 / n) = 6 tokens
    assert abs(np.median(L) - 512) < 30
    # the fraction below 512 * e^(+-0.6) (one sigma) is Phi(1) - Phi(-1) = 0.683
    inside = np.mean((L > 512 * math.exp(-0.6)) & (L < 512 * math.exp(0.6)))
    assert abs(inside - 0.6827) < 0.03


def test_zipf_token_ids_and_lengths():
    rng = np.random.Generator(np.random.PCG64(5))
    ids = synth.zipf_ids(rng, 400000, 1.1, 32000)
    assert ids.min() >= 0 and ids.max() < 32000
    c = np.bincount(ids, minlength=32000)
    assert c.argmax() == 0
    # P(rank 1) / P(rank 2) = 2^1.1
    assert abs(c[0] / c[1] - 2 ** 1.1) < 0.1
    # bounded Zipf(1.1) lengths on [32, 8192]: the sample mean against the pmf's mean
    t = synth.make_table(synth.TABLES["c4"], 32000, seed=44, n_tuples=32768)
    L = t["lengths"]
    assert L.min() >= 32 and L.max() <= 8192
    k = np.arange(32, 8193, dtype=np.float64)
    p = k ** -1.1
    p /= p.sum()
    mean, sd = float((k * p).sum()), float(np.sqrt(((k - (k * p).sum()) ** 2 * p).sum()))
    assert abs(L.mean() - mean) < 4 * sd / math.sqrt(len(L))


def test_tables_are_prefixes_and_seeded():
    full = synth.make_table(synth.TABLES["c2"], 32000, seed=7)
    part = synth.make_table(synth.TABLES["c2"], 32000, seed=7, n_tuples=100)
    assert np.array_equal(part["lengths"], full["lengths"][:100])
    assert np.array_equal(part["tokens"], full["tokens"][:part["offsets"][-1]])
    other = synth.make_table(synth.TABLES["c2"], 32000, seed=8, n_tuples=100)
    assert not np.array_equal(other["lengths"], part["lengths"])
    t = synth.make_table_from_lengths([1, 5, 0, 3], 50, seed=2, ids="zipf")
    assert list(t["offsets"]) == [0, 1, 6, 6, 9] and t["tokens"].max() < 50


def test_prompt_and_sample_helpers():
    a = synth.make_prompt(32, 1000, seed=9, label_ids=(4, 2), r=0.25)
    b = synth.make_prompt(32, 1000, seed=9, label_ids=(4, 2), r=0.25)
    assert a == b and len(a.prompt) == 32 and max(a.prompt) < 1000
    assert a.label_ids == (4, 2) and a.r == 0.25 and a.kind == "filter"
    s = synth.sample_tuples(1000, 17, seed=4)
    assert len(s) == 17 and s[0] == 0 and s[-1] == 999 and s == sorted(set(s))
