"""Pins of the oracle's operator steps (CPU only): cached == from scratch (Sec. 5),
retention against brute force, EA-lite against the Gaussian moment generating
function, the log-odds identity and the decision table."""
import math

import numpy as np
import pytest
from scipy.special import log_softmax

from oracle import model as M
from oracle import operator as O
from paper_2602_04430_b300 import synth


def rng(seed=0):
    return np.random.Generator(np.random.PCG64(seed))


def tiny_cfg(hq=4, hkv=2, layers=2):
    return synth.ModelConfig(layers=layers, d=32, hq=hq, hkv=hkv, hd=8, ffn=48, vocab=64,
                             dtype="f32", name="t")


@pytest.fixture(scope="module")
def setup():
    cfg = tiny_cfg()
    w = synth.make_weights(cfg, seed=11, std=0.3)
    table = synth.make_table_from_lengths([1, 5, 13, 20], cfg.vocab, seed=12)
    op = synth.make_prompt(6, cfg.vocab, seed=13, label_ids=(1, 0))
    return cfg, w, table, op


def test_cached_equals_from_scratch(setup):
    """Operators reuse the cache and skip the prefill (Sec. 5): at r = 1 the
    cached evaluation equals the document + prompt forward pass."""
    cfg, w, table, op = setup
    tok, off = table["tokens"], table["offsets"]
    for t in range(len(off) - 1):
        doc = tok[off[t]:off[t + 1]]
        c = O.kv_build(cfg, w, doc)
        Kr, Vr, _ = O.retained_kv(c, 1.0)
        z_cached = O.op_eval(cfg, w, c.L, Kr, Vr, op.prompt, op.label_ids)
        z_scratch = O.op_eval_from_scratch(cfg, w, doc, op.prompt, op.label_ids)
        np.testing.assert_allclose(z_cached, z_scratch, rtol=1e-12, atol=1e-13)


def test_r1_is_unpruned_any_order(setup):
    cfg, w, table, op = setup
    tok, off = table["tokens"], table["offsets"]
    doc = tok[off[3]:off[4]]
    c = O.kv_build(cfg, w, doc)
    Kr, Vr, I = O.retained_kv(c, 1.0)
    for l in range(cfg.layers):
        for g in range(cfg.hkv):
            assert sorted(I[l][g].tolist()) == list(range(c.L))
    nat = [[np.arange(c.L) for _ in range(cfg.hkv)] for _ in range(cfg.layers)]
    Kn, Vn, _ = O.retained_kv(c, 1.0, idx=nat)
    z1 = O.op_eval(cfg, w, c.L, Kr, Vr, op.prompt, op.label_ids)
    z2 = O.op_eval(cfg, w, c.L, Kn, Vn, op.prompt, op.label_ids)
    np.testing.assert_allclose(z1, z2, rtol=1e-12, atol=1e-13)


def test_kv_build_matches_forward_states(setup):
    cfg, w, table, _ = setup
    doc = table["tokens"][table["offsets"][2]:table["offsets"][3]]
    c = O.kv_build(cfg, w, doc)
    xf = M.forward(cfg, w, doc)
    np.testing.assert_allclose(c.pooled, xf.mean(axis=0), rtol=1e-13)
    # layer-0 keys are rope(rmsnorm(E[tok]) Wk^T) at positions 0..L-1
    x = w["embed"][doc].astype(np.float64)
    k = (M.rmsnorm(x, cfg.eps) @ w["layers"][0]["wk"].T.astype(np.float64)).reshape(-1, cfg.hkv, cfg.hd)
    k = M.rope(k, np.arange(len(doc)), cfg.rope_theta)
    np.testing.assert_allclose(c.k[0][1], k[:, 1, :], rtol=1e-13, atol=1e-15)


def test_padded_masked_equals_ragged():
    """Padding the cached slots and masking them out (Sec. 5, execution-time batching)
    gives the ragged result."""
    r = rng(3)
    q = r.standard_normal((5, 4, 8))
    k = r.standard_normal((7, 2, 8))
    v = r.standard_normal((7, 2, 8))
    vis = np.ones((5, 7), dtype=bool)
    pad_k = np.concatenate([k, 1e3 * r.standard_normal((4, 2, 8))])
    pad_v = np.concatenate([v, 1e3 * r.standard_normal((4, 2, 8))])
    pad_vis = np.concatenate([vis, np.zeros((5, 4), dtype=bool)], axis=1)
    np.testing.assert_allclose(M.attention(q, pad_k, pad_v, pad_vis), M.attention(q, k, v, vis),
                               rtol=1e-13, atol=1e-14)


def brute_rank(scores):
    return sorted(range(len(scores)), key=lambda j: (-float(scores[j]), j))


def test_retention_matches_brute_force_sort():
    r = rng(4)
    for L in (1, 2, 7, 64, 65, 300):
        for trial in range(5):
            s = r.choice(np.array([-1.5, -0.0, 0.0, 0.25, 3.0, 1e-30]), size=L) if trial % 2 else \
                r.standard_normal(L).astype(np.float32)
            order = O.rank_order(s)
            assert order.tolist() == brute_rank(s)
            # O(L^2) rank count: slot j's rank = #(better slots)
            for j in range(L):
                better = sum(1 for i in range(L) if (s[i] > s[j]) or (s[i] == s[j] and i < j))
                assert order[better] == j
            for rr in (0.1, 0.25, 0.5, 1.0):
                n = O.n_keep(L, rr)
                assert O.retain(s, rr).tolist() == brute_rank(s)[:n]


def test_retention_nested_in_r_and_identity_at_1():
    s = rng(5).standard_normal(101)
    prev = []
    for rr in (0.05, 0.1, 0.3, 0.5, 0.77, 1.0):
        cur = O.retain(s, rr).tolist()
        assert cur[:len(prev)] == prev
        prev = cur
    assert sorted(prev) == list(range(101))


def test_signed_zero_ties_and_nan():
    s = np.array([0.0, -0.0, 0.0, -0.0])
    assert O.rank_order(s).tolist() == [0, 1, 2, 3]
    with pytest.raises(ValueError):
        O.rank_order(np.array([1.0, np.nan]))


def test_n_keep_cases():
    assert O.n_keep(10, 1.0) == 10
    assert O.n_keep(1, 0.01) == 1
    assert O.n_keep(10, 0.25) == 3      # floor(2.5 + 0.5)
    assert O.n_keep(10, 0.05) == 1      # floor(0.5 + 0.5)
    assert O.n_keep(7, 0.5) == 4        # floor(3.5 + 0.5)
    assert O.n_keep(1000, 0.1) == 100   # 0.1 is slightly above 1/10 as a double
    assert O.n_keep(2048, 0.1) == 205   # 204.8 -> 205
    for bad in (0.0, -0.1, 1.0000001, float("nan")):
        with pytest.raises(ValueError):
            O.n_keep(10, bad)


def test_ea_score_is_gaussian_mgf():
    """score_j - ln||v_j|| = ln E[exp(q.k_j/sqrt(hd))] for Gaussian queries (Monte Carlo)."""
    r = rng(6)
    hd = 8
    mu = 0.3 * r.standard_normal(hd)
    sd = 0.2 + 0.3 * r.random(hd)
    q = mu + sd * r.standard_normal((400000, hd))
    k = r.standard_normal((5, hd))
    v = r.standard_normal((5, hd))
    s, mu_hat, s2_hat = O.ea_scores(q.reshape(-1, 2, hd), k, v)
    np.testing.assert_allclose(mu_hat, q.mean(axis=0), rtol=1e-12)
    mc = np.log(np.mean(np.exp(q @ k.T / math.sqrt(hd)), axis=0)) + np.log(np.linalg.norm(v, axis=1))
    np.testing.assert_allclose(s, mc, atol=5e-3)


def test_ea_score_invariants():
    r = rng(7)
    q = r.standard_normal((30, 2, 8))
    k = r.standard_normal((12, 8))
    v = r.standard_normal((12, 8))
    s, _, _ = O.ea_scores(q, k, v)
    perm = r.permutation(12)
    s2, _, _ = O.ea_scores(q, k[perm], v[perm])
    np.testing.assert_allclose(s2, s[perm], rtol=1e-14)
    # identical queries (sigma^2 = 0) and equal value norms: ranking by mu . k
    qc = np.tile(q[0, 0], (30, 2, 1))
    vu = v / np.linalg.norm(v, axis=1, keepdims=True)
    s3, mu, s2v = O.ea_scores(qc, k, vu)
    assert np.allclose(s2v, 0.0)
    assert O.rank_order(s3).tolist() == O.rank_order(k @ mu).tolist()


def test_log_odds_equals_full_softmax(setup):
    cfg, w, table, op = setup
    doc = table["tokens"][:5]
    seq = np.concatenate([doc, np.asarray(op.prompt)])
    xf = M.forward(cfg, w, seq)[-1]
    full = log_softmax(w["w_lm"].astype(np.float64) @ xf)
    z = M.label_logits(w, xf, [1, 0])
    assert abs((z[0] - z[1]) - (full[1] - full[0])) < 1e-12


def test_decision_table():
    A, R, U = O.ACCEPT, O.REJECT, O.UNSURE
    # s = za - zr against theta+ = 1, theta- = -1
    cases = [(2.0, 0.0, A), (1.0, 0.0, U), (0.5, 0.0, U), (0.0, 0.0, U), (-1.0, 0.0, U),
             (-1.5, 0.0, R), (-3.0, 0.0, R)]
    for za, zr, d in cases:
        assert O.decide_filter(za, zr, 1.0, -1.0) == d
    # single threshold theta+ = theta- = 0.5: s > 0.5 accept, s < 0.5 reject, tie unsure
    assert O.decide_filter(0.6, 0.0, 0.5, 0.5) == A
    assert O.decide_filter(0.4, 0.0, 0.5, 0.5) == R
    assert O.decide_filter(0.5, 0.0, 0.5, 0.5) == U
    # crossed thresholds (theta- > theta+) between them: reject beats accept on a tie
    assert O.decide_filter(0.0, 0.0, -1.0, 1.0) == R
    assert O.decide_classify([0.1, 0.3, 0.3]) == 1
    assert O.decide_classify([0.1, 0.3, 0.3], [0.0, 0.0, 1e-9]) == 2


def test_pruned_cache_equals_masked_full_sequence(setup):
    """r < 1: the cached evaluation equals one causal pass over document + prompt in
    which each prompt row, per layer and kv head, cannot see the pruned document
    slots; the prompt keeps its positions L..L+P-1 (pruning happens after prefill)."""
    cfg, w, table, op = setup
    tok, off = table["tokens"], table["offsets"]
    doc = tok[off[3]:off[4]]
    L, P = len(doc), len(op.prompt)
    c = O.kv_build(cfg, w, doc)
    Kr, Vr, I = O.retained_kv(c, 0.4)
    z_cached = O.op_eval(cfg, w, L, Kr, Vr, op.prompt, op.label_ids)
    seq = np.concatenate([doc, np.asarray(op.prompt)])
    n = L + P
    x = w["embed"][seq].astype(np.float64)
    G = cfg.hq // cfg.hkv
    for l, lw in enumerate(w["layers"]):
        q, k, v = M.qkv(cfg, lw, x, np.arange(n))
        o = np.empty_like(q)
        for g in range(cfg.hkv):
            vis = M.causal_mask(n)
            hidden = np.setdiff1d(np.arange(L), I[l][g])
            vis[L:, hidden] = False
            o[:, g * G:(g + 1) * G] = M.attention(q[:, g * G:(g + 1) * G], k[:, g:g + 1],
                                                  v[:, g:g + 1], vis)
        x = M.attn_out_and_ffn(cfg, lw, x, o)
    z_masked = M.label_logits(w, M.rmsnorm(x[-1], cfg.eps), op.label_ids)
    np.testing.assert_allclose(z_cached, z_masked, rtol=1e-12, atol=1e-13)


def test_cascade_stages_definition():
    """Multi-stage cascade oracle: the first sure stage decides, later stages
    are not consulted, the last stage's unsure stays unsure (Sec. 4.1)."""
    from oracle.operator import ACCEPT, REJECT, UNSURE, cascade_stages
    d0 = [ACCEPT, UNSURE, REJECT, UNSURE, UNSURE]
    d1 = [REJECT, REJECT, ACCEPT, UNSURE, ACCEPT]
    d2 = [ACCEPT, ACCEPT, ACCEPT, UNSURE, REJECT]
    labels, stage, counts = cascade_stages([d0, d1, d2])
    assert labels == [ACCEPT, REJECT, REJECT, UNSURE, ACCEPT]
    assert stage == [0, 1, 0, 2, 1]
    assert counts == [5, 3, 1]
    # one stage: its own decisions, unsure included
    assert cascade_stages([d0]) == (d0, [0] * 5, [5])
    # a stage that is never unsure ends the cascade
    labels, stage, counts = cascade_stages([d1[:3], d0[:3], d2[:3]])
    assert counts == [3, 0, 0] and stage == [0, 0, 0] and labels == d1[:3]


def test_map_eval_cached_equals_from_scratch():
    """Greedy decode over the cached document (r = 1) equals decoding document +
    prompt + generated tokens from scratch: the same tokens and logits (positions
    L + P + t, causal visibility of the generated tokens)."""
    from oracle.operator import kv_build, map_eval, map_eval_from_scratch, retained_kv
    from paper_2602_04430_b300 import synth
    cfg = synth.MODELS["tiny_f32"]
    w = synth.make_weights(cfg, seed=81)
    rng = np.random.Generator(np.random.PCG64(82))
    prompt = rng.integers(0, cfg.vocab, size=6)
    for L in (1, 9, 33):
        doc = rng.integers(0, cfg.vocab, size=L)
        Kr, Vr, _ = retained_kv(kv_build(cfg, w, doc), 1.0)
        toks, logs = map_eval(cfg, w, L, Kr, Vr, prompt, 5)
        toks2, logs2 = map_eval_from_scratch(cfg, w, doc, prompt, 5)
        assert toks == toks2
        np.testing.assert_allclose(logs, logs2, rtol=1e-10, atol=1e-12)
        assert all(0 <= t < cfg.vocab for t in toks)
        # every token is the argmax of its step's logits
        assert all(int(np.argmax(z)) == t for z, t in zip(logs, toks))


def test_oracle_pool_matches_serial_oracle():
    """The parallel runner adds no arithmetic: its logits, retained sets and
    scores equal serial oracle calls (up to BLAS summation order)."""
    from oracle import pool as OP
    cfg = synth.ModelConfig(layers=2, d=32, hq=4, hkv=2, hd=8, ffn=48, vocab=64, dtype="f32", name="p")
    w = synth.make_weights(cfg, seed=41, std=0.2)
    table = synth.make_table_from_lengths([5, 17, 33], cfg.vocab, seed=42)
    op = synth.make_prompt(4, cfg.vocab, seed=43, r=0.5)
    docs = {t: table["tokens"][table["offsets"][t]:table["offsets"][t + 1]] for t in range(3)}
    ops = [{"prompt": op.prompt, "label_ids": op.label_ids, "r": 0.5},
           {"prompt": op.prompt, "label_ids": op.label_ids, "r": 1.0, "kv_fp8": True}]
    with OP.OraclePool(cfg, w, workers=2) as pool:
        res = pool.run(docs, ops, want_scores=True)
    for t, doc in docs.items():
        c = O.kv_build(cfg, w, doc)
        for j, o in enumerate(ops):
            Kr, Vr, idx = O.retained_kv(c, o["r"], kv_fp8=o.get("kv_fp8", False))
            z = O.op_eval(cfg, w, c.L, Kr, Vr, op.prompt, op.label_ids)
            np.testing.assert_allclose(res[t]["logits"][j], z, rtol=1e-12, atol=1e-12)
            for l in range(cfg.layers):
                for g in range(cfg.hkv):
                    np.testing.assert_array_equal(res[t]["idx"][j][l][g], idx[l][g])
                    np.testing.assert_allclose(res[t]["scores"][l][g], c.scores[l][g], rtol=1e-12)


def test_oracle_pool_codes_from_given_values_and_shared_profiles():
    """The pool's E4M3 options: codes decided from given keys and values (here
    the oracle's own, so the result must equal its float32-arithmetic E4M3
    path), and a profile shared at a larger r (the operator reads a prefix of
    the profile's quantised set), on given index sets."""
    from oracle import pool as OP
    cfg = synth.ModelConfig(layers=2, d=32, hq=4, hkv=2, hd=8, ffn=48, vocab=64, dtype="f32", name="q")
    w = synth.make_weights(cfg, seed=51, std=0.2)
    table = synth.make_table_from_lengths([70, 150], cfg.vocab, seed=52)
    op = synth.make_prompt(4, cfg.vocab, seed=53, r=0.4)
    docs = {t: table["tokens"][table["offsets"][t]:table["offsets"][t + 1]] for t in range(2)}
    caches = {t: O.kv_build(cfg, w, d) for t, d in docs.items()}
    given = {t: (c.k, c.v) for t, c in caches.items()}
    full = {t: [[O.rank_order(c.scores[l][g]) for g in range(cfg.hkv)] for l in range(cfg.layers)]
            for t, c in caches.items()}
    ops = [{"prompt": op.prompt, "label_ids": op.label_ids, "r": 0.4, "kv_fp8": True, "codes_from_given": True,
            "fp8_profile_r": 1.0},
           {"prompt": op.prompt, "label_ids": op.label_ids, "r": 0.4, "kv_fp8": True, "fp8_profile_r": 1.0}]
    idx = {t: [full[t], full[t]] for t in docs}
    with OP.OraclePool(cfg, w, workers=2) as pool:
        res = pool.run(docs, ops, idx=idx, given=given)
    for t, c in caches.items():
        Kr, Vr, _ = O.retained_kv(c, 0.4, kv_fp8=True, fp8_arith="f32", fp8_profile_r=1.0)
        z32 = O.op_eval(cfg, w, c.L, Kr, Vr, op.prompt, op.label_ids)
        np.testing.assert_allclose(res[t]["logits"][0], z32, rtol=1e-12, atol=1e-12)
        Kr, Vr, _ = O.retained_kv(c, 0.4, kv_fp8=True, fp8_profile_r=1.0)
        z64 = O.op_eval(cfg, w, c.L, Kr, Vr, op.prompt, op.label_ids)
        np.testing.assert_allclose(res[t]["logits"][1], z64, rtol=1e-12, atol=1e-12)


def test_oracle_workers_hold_a_cache_and_match_serial_oracle():
    """Persistent workers (the benchmark's CPU legs): each builds one tuple's
    cache, then every step evaluates the operator on it; the logits equal a
    serial oracle run."""
    from oracle import pool as OP
    cfg = synth.ModelConfig(layers=2, d=32, hq=4, hkv=2, hd=8, ffn=48, vocab=64, dtype="f32", name="p")
    w = synth.make_weights(cfg, seed=44, std=0.2)
    table = synth.make_table_from_lengths([9, 23], cfg.vocab, seed=45)
    op = synth.make_prompt(4, cfg.vocab, seed=46, r=0.5)
    o = {"prompt": op.prompt, "label_ids": op.label_ids, "r": 0.5}
    docs = [table["tokens"][table["offsets"][t]:table["offsets"][t + 1]] for t in range(2)]
    wk = OP.OracleWorkers(cfg, w, workers=2)
    try:
        wk.build(docs)
        secs, lens = wk.wait_built()
        assert lens == [9, 23]
        for _ in range(2):
            dt, zs = wk.step(o)
            assert dt > 0
            for doc, z in zip(docs, zs):
                c = O.kv_build(cfg, w, doc)
                Kr, Vr, _ = O.retained_kv(c, 0.5)
                np.testing.assert_allclose(z, O.op_eval(cfg, w, c.L, Kr, Vr, op.prompt, op.label_ids),
                                           rtol=1e-12, atol=1e-12)
    finally:
        wk.close()
