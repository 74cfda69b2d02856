"""Scoring ablation on the GPU against the float64 oracle (oracle/scoring.py).

Full Expected Attention (st_set_scoring EA_FULL, horizon F): every slot's
score normwise per (layer, kv head) within 1e-4 of the oracle for the float32
tiny model and 2e-2 for the BF16 config-2 model; the retained sets are the
brute-force ranking of the GPU's own scores bit for bit and, for float32, the
oracle's ranking except at near-ties.  Query-specific scores
(st_kv_score_query) the same way, then the operator evaluated on the cache
retained by them against the oracle on the same index sets.  Switching back
to EA-lite restores the default scores bit for bit."""
import numpy as np
import pytest

from tests.util import normwise_rel

pytestmark = pytest.mark.gpu


def _env(model_name, table_cfg, n_tuples, seed, max_pos):
    import torch
    from paper_2602_04430_b300 import build, stretto, synth
    build.build()
    cfg = synth.MODELS[model_name]
    w = synth.make_weights(cfg, seed=seed)
    table = synth.make_table(synth.TABLES[table_cfg], cfg.vocab, seed=seed + 1, n_tuples=n_tuples)
    model = stretto.Model(cfg, w, max_pos=max_pos)
    kv = model.kv_alloc(table["offsets"])
    tok = torch.from_numpy(table["tokens"]).cuda()
    return dict(cfg=cfg, w=w, table=table, model=model, kv=kv, tok=tok, stretto=stretto, synth=synth,
                torch=torch)


def _views(e):
    cfg, kv, st, torch = e["cfg"], e["kv"], e["stretto"], e["torch"]
    R = int(e["table"]["offsets"][-1])
    sc = kv.read(st.ST_VIEW_SCORES, torch.float32, (cfg.layers, cfg.hkv, R)).cpu().numpy()
    rk = kv.read(st.ST_VIEW_RANK, torch.int32, (cfg.layers, cfg.hkv, R)).cpu().numpy()
    return sc, rk


def _check_sets(e, gpu_scores, rank, ref_scores, r, f32):
    """Bit-exact against the GPU's own scores; against the oracle up to near-ties (float32)."""
    from oracle import operator as O
    cfg, off = e["cfg"], e["table"]["offsets"]
    exchanged = 0
    for t in range(len(off) - 1):
        a, b = int(off[t]), int(off[t + 1])
        n = O.n_keep(b - a, r)
        for l in range(cfg.layers):
            for g in range(cfg.hkv):
                own = O.rank_order(gpu_scores[l, g, a:b].astype(np.float64))[:n]
                got = rank[l, g, a:a + n]
                np.testing.assert_array_equal(got, own)
                if not f32:
                    continue
                s = np.asarray(ref_scores[t][l][g], dtype=np.float64)
                ref = O.rank_order(s)[:n]
                diff = set(got.tolist()) ^ set(ref.tolist())
                if diff:
                    err = np.abs(gpu_scores[l, g, a:b] - s).max()
                    kth = s[ref[-1]]
                    for j in diff:
                        assert abs(s[j] - kth) <= max(1e-5 * abs(kth), 4 * err), (t, l, g, j)
                    exchanged += len(diff) // 2
    return exchanged


def _ea_full_case(model_name, table_cfg, n_tuples, seed, max_pos, F, tol, f32):
    from oracle import scoring as SC
    e = _env(model_name, table_cfg, n_tuples, seed, max_pos)
    cfg, kv, model, st, torch = e["cfg"], e["kv"], e["model"], e["stretto"], e["torch"]
    tok, off = e["table"]["tokens"], e["table"]["offsets"]
    # EA-lite scores of a first build, to check that switching back restores them
    kv.build(e["tok"])
    torch.cuda.synchronize()
    lite, _ = _views(e)
    model.set_scoring(st.ST_SCORE_EA_FULL, F)
    kv.build(e["tok"])
    kv.retain(0.5)
    torch.cuda.synchronize()
    model.status()
    sc, rk = _views(e)
    refs = []
    worst = 0.0
    for t in range(len(off) - 1):
        a, b = int(off[t]), int(off[t + 1])
        c = SC.kv_build_ea_full(cfg, e["w"], tok[a:b], F)
        refs.append(c.scores)
        for l in range(cfg.layers):
            for g in range(cfg.hkv):
                err = normwise_rel(sc[l, g, a:b], c.scores[l][g])
                worst = max(worst, err)
                assert err <= tol, (t, l, g, err)
    ex = _check_sets(e, sc, rk, refs, 0.5, f32)
    print(f"{model_name}: EA-full F={F} worst normwise score error {worst:.3e}, boundary exchanges {ex}")
    # differs from EA-lite, and EA-lite comes back bit for bit
    assert not np.array_equal(sc, lite)
    model.set_scoring(st.ST_SCORE_EA_LITE)
    kv.build(e["tok"])
    torch.cuda.synchronize()
    np.testing.assert_array_equal(_views(e)[0], lite)


def test_ea_full_tiny_f32():
    _ea_full_case("tiny_f32", "tiny", 12, 201, 512, 64, 1e-4, True)


def test_ea_full_bf16():
    _ea_full_case("c2_bf16", "c2", 6, 203, 2200, 64, 2e-2, False)


def _query_case(model_name, table_cfg, n_tuples, seed, max_pos, P, tol, f32):
    from oracle import operator as O
    from oracle import scoring as SC
    e = _env(model_name, table_cfg, n_tuples, seed, max_pos)
    cfg, kv, model, st, torch, synth = e["cfg"], e["kv"], e["model"], e["stretto"], e["torch"], e["synth"]
    tok, off = e["table"]["tokens"], e["table"]["offsets"]
    T = len(off) - 1
    kv.build(e["tok"])
    kv.retain(1.0)
    op = model.operator(synth.make_prompt(P, cfg.vocab, seed=seed + 5, r=0.5))
    kv.score_query(op)
    kv.retain(0.5)
    ids = torch.arange(T, dtype=torch.int32, device="cuda")
    lg, _ = op.eval(kv, ids)
    torch.cuda.synchronize()
    model.status()
    sc, rk = _views(e)
    lg = lg.cpu().numpy()
    refs, worst, worst_z = [], 0.0, 0.0
    for t in range(T):
        a, b = int(off[t]), int(off[t + 1])
        c = O.kv_build(cfg, e["w"], tok[a:b])
        qs = SC.query_scores(cfg, e["w"], c, op.op.prompt)
        refs.append(qs)
        for l in range(cfg.layers):
            for g in range(cfg.hkv):
                err = normwise_rel(sc[l, g, a:b], qs[l][g])
                worst = max(worst, err)
                assert err <= tol, (t, l, g, err)
        n = O.n_keep(c.L, 0.5)
        idx = [[rk[l, g, a:a + n] for g in range(cfg.hkv)] for l in range(cfg.layers)]
        Kr, Vr, _ = O.retained_kv(c, 0.5, idx=idx)
        z = O.op_eval(cfg, e["w"], c.L, Kr, Vr, op.op.prompt, op.op.label_ids)
        worst_z = max(worst_z, normwise_rel(lg[t], z))
        assert normwise_rel(lg[t], z) <= tol, (t, normwise_rel(lg[t], z))
    ex = _check_sets(e, sc, rk, refs, 0.5, f32)
    print(f"{model_name}: query-specific worst score error {worst:.3e}, logits {worst_z:.3e}, "
          f"boundary exchanges {ex}")
    # the profile is no longer r = 1: query scoring is refused
    with pytest.raises(st.StrettoError) as ei:
        kv.score_query(op)
    assert ei.value.code == st.ST_EINVAL


def test_query_scores_tiny_f32():
    _query_case("tiny_f32", "tiny", 12, 211, 512, 8, 1e-4, True)


def test_query_scores_bf16():
    _query_case("c2_bf16", "c2", 6, 213, 2200, 24, 2e-2, False)


def test_set_scoring_rejects_bad_arguments():
    from paper_2602_04430_b300 import build, stretto, synth
    build.build()
    cfg = synth.MODELS["tiny_f32"]
    model = stretto.Model(cfg, synth.make_weights(cfg, seed=221), max_pos=300)
    for mode, h in ((7, 64), (stretto.ST_SCORE_EA_FULL, 0), (stretto.ST_SCORE_EA_FULL, 300)):
        with pytest.raises(stretto.StrettoError) as ei:
            model.set_scoring(mode, h)
        assert ei.value.code == stretto.ST_EINVAL
    # a 256-token document + horizon 64 exceeds max_pos 300: the build is refused
    import torch
    table = synth.make_table(synth.TABLES["tiny"], cfg.vocab, seed=222, n_tuples=2)
    kv = model.kv_alloc(table["offsets"])
    model.set_scoring(stretto.ST_SCORE_EA_FULL, 64)
    with pytest.raises(stretto.StrettoError) as ei:
        kv.build(torch.from_numpy(table["tokens"]).cuda())
    assert ei.value.code == stretto.ST_EINVAL
