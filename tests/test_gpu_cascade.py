"""Multi-stage cascade (st_cascade_run) against the cascade definition.

Each stage's decision for a tuple does not depend on which other tuples the
stage evaluates (batch independence is tested bit for bit elsewhere), so the
executor's labels, deciding stages and per-stage counts must equal the oracle's
cascade definition applied to every stage's decisions over all tuples.  Stage
thresholds are set from the stages' own margin quantiles so that about 40 % of
the tuples reaching a stage stay unsure.  Two set-ups: three stages of growing
r on one BF16 decoder and cache, and a two-model cascade (the float32 tiny
decoder first, the BF16 config-2 decoder second) over one token table."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _with_band(synth, base, margins, lo_q=0.3, hi_q=0.7):
    th_neg, th_pos = float(np.quantile(margins, lo_q)), float(np.quantile(margins, hi_q))
    return synth.Operator(prompt=base.prompt, label_ids=base.label_ids, r=base.r, theta_pos=th_pos,
                          theta_neg=th_neg, kind="filter", bias=None)


def _stage_ops(models_kvs, bases, synth, torch):
    """Per stage: an operator with an unsure band, and its decisions over all tuples."""
    ops, decisions = [], []
    for (model, kv), base in zip(models_kvs, bases):
        ids = torch.arange(kv.T, dtype=torch.int32, device="cuda")
        lg, _ = model.operator(base).eval(kv, ids)
        lg = lg.cpu().numpy()
        op = model.operator(_with_band(synth, base, lg[:, 0] - lg[:, 1]))
        _, lb = op.eval(kv, ids)
        torch.cuda.synchronize()
        ops.append(op)
        decisions.append(lb.cpu().tolist())
    return ops, decisions


def _check(models_kvs, ops, decisions, stretto, torch):
    from oracle.operator import cascade_stages
    T = models_kvs[0][1].T
    ids = torch.arange(T, dtype=torch.int32, device="cuda")
    stages = [(m, kv, op) for (m, kv), op in zip(models_kvs, ops)]
    labels, stage, counts, ms = stretto.cascade_run(stages, ids)
    torch.cuda.synchronize()
    for m, _ in models_kvs:
        m.status()
    ref_l, ref_s, ref_c = cascade_stages(decisions)
    assert labels.cpu().tolist() == ref_l
    assert stage.cpu().tolist() == ref_s
    assert counts == ref_c
    assert all(c > 0 for c in counts) and counts[-1] < counts[0]
    assert all(t > 0 for t in ms)
    return counts


def test_three_stages_growing_r():
    import torch
    from paper_2602_04430_b300 import build, stretto, synth
    build.build()
    cfg = synth.MODELS["c2_bf16"]
    table = synth.make_table(synth.TABLES["c2"], cfg.vocab, seed=61, n_tuples=700)
    model = stretto.Model(cfg, synth.make_weights(cfg, seed=62), max_pos=2112)
    kv = model.kv_alloc(table["offsets"])
    kv.build(torch.from_numpy(table["tokens"]).cuda())
    kv.retain(1.0)
    bases = [synth.make_prompt(32, cfg.vocab, seed=63, r=r) for r in (0.1, 0.3, 1.0)]
    mk = [(model, kv)] * 3
    ops, dec = _stage_ops(mk, bases, synth, torch)
    counts = _check(mk, ops, dec, stretto, torch)
    print("tuples per stage", counts)


def test_two_models():
    import torch
    from paper_2602_04430_b300 import build, stretto, synth
    build.build()
    small, big = synth.MODELS["tiny_f32"], synth.MODELS["c2_bf16"]
    # token ids valid for both vocabularies
    table = synth.make_table(synth.TABLES["c2"], small.vocab, seed=64, n_tuples=300)
    m1 = stretto.Model(small, synth.make_weights(small, seed=65), max_pos=2112)
    m2 = stretto.Model(big, synth.make_weights(big, seed=66), max_pos=2112)
    tok = torch.from_numpy(table["tokens"]).cuda()
    mk = []
    for m in (m1, m2):
        kv = m.kv_alloc(table["offsets"])
        kv.build(tok)
        kv.retain(0.5)
        mk.append((m, kv))
    bases = [synth.make_prompt(16, small.vocab, seed=67, r=0.5), synth.make_prompt(32, small.vocab, seed=68, r=0.5)]
    ops, dec = _stage_ops(mk, bases, synth, torch)
    _check(mk, ops, dec, stretto, torch)


def test_cascade_rejects_classify(tmp_path):
    import torch
    from paper_2602_04430_b300 import build, stretto, synth
    build.build()
    cfg = synth.MODELS["tiny_f32"]
    table = synth.make_table(synth.TABLES["tiny"], cfg.vocab, seed=69)
    m = stretto.Model(cfg, synth.make_weights(cfg, seed=70), max_pos=512)
    kv = m.kv_alloc(table["offsets"])
    kv.build(torch.from_numpy(table["tokens"]).cuda())
    kv.retain(1.0)
    op = m.operator(synth.make_prompt(8, cfg.vocab, seed=71, label_ids=(1, 2, 3), kind="classify"))
    with pytest.raises(stretto.StrettoError):
        stretto.cascade_run([(m, kv, op)], torch.arange(kv.T, dtype=torch.int32, device="cuda"))


def test_proxy_cascade_with_e4m3_band_then_bf16():
    """st_proxy_cascade: the proxy (trained a few steps on the FP8 operator's
    labels) as stage 0, then an operator over an E4M3 profile with an unsure
    band, then the same operator over the BF16 profile of the same cache (two
    profiles resident at once).  Labels, deciding stages and counts must equal
    the cascade definition applied to the proxy's decisions (UNSURE below tau)
    and to each stage's decisions over all tuples, on a shuffled subset of the
    table's tuples."""
    import torch
    from oracle.operator import UNSURE, cascade_stages
    from paper_2602_04430_b300 import build, stretto, synth
    build.build()
    cfg = synth.MODELS["c2_bf16"]
    table = synth.make_table(synth.TABLES["c2"], cfg.vocab, seed=72, n_tuples=600)
    model = stretto.Model(cfg, synth.make_weights(cfg, seed=73), max_pos=2112)
    kv = model.kv_alloc(table["offsets"])
    kv.build(torch.from_numpy(table["tokens"]).cuda())
    kv.retain(0.5, stretto.ST_BF16)
    prof = kv.profile(0.5)
    prof.retain(0.5, stretto.ST_E4M3)
    T = kv.T
    all_ids = torch.arange(T, dtype=torch.int32, device="cuda")
    base = synth.make_prompt(32, cfg.vocab, seed=74, r=0.5)
    lg, _ = model.operator(base).eval(prof, all_ids)
    m = (lg[:, 0] - lg[:, 1]).cpu().numpy()
    theta = float(np.median(m))
    band = synth.Operator(prompt=base.prompt, label_ids=base.label_ids, r=0.5,
                          theta_pos=float(np.quantile(m, 0.6)), theta_neg=float(np.quantile(m, 0.4)))
    plain = synth.Operator(prompt=base.prompt, label_ids=base.label_ids, r=0.5, theta_pos=theta, theta_neg=theta)
    op8, op16 = model.operator(band), model.operator(plain)
    x = kv.read(stretto.ST_VIEW_POOLED, torch.float32, (T, cfg.d))
    px = stretto.Proxy(model, synth.make_proxy_weights(cfg.d, 512, 128, seed=75))
    y = torch.from_numpy((m > theta).astype(np.int32)).cuda()
    for b in synth.minibatches(T, 128, 2, seed=76):
        px.train_step(x, y, torch.from_numpy(b).cuda(), lr=1e-3)
    rng = np.random.Generator(np.random.PCG64(77))
    sub = rng.permutation(T)[:450].astype(np.int32)
    ids = torch.from_numpy(sub).cuda()
    conf, plab = px.eval(x, rows=ids)
    tau = float(np.quantile(conf.cpu().numpy(), 0.5))
    d_proxy = np.where(conf.cpu().numpy() < np.float32(tau), UNSURE, plab.cpu().numpy()).tolist()
    d8 = op8.eval(prof, ids)[1].cpu().tolist()
    d16 = op16.eval(kv, ids)[1].cpu().tolist()
    labels, stage, counts = stretto.proxy_cascade(px, x, tau, [(model, prof, op8), (model, kv, op16)], ids)
    torch.cuda.synchronize()
    model.status()
    ref_l, ref_s, ref_c = cascade_stages([d_proxy, d8, d16])
    assert labels.cpu().tolist() == ref_l
    assert stage.cpu().tolist() == ref_s
    assert counts == ref_c
    assert counts[0] > counts[1] > counts[2] > 0, counts
    print("proxy cascade: tuples per stage", counts)
