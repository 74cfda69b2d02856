"""Map operator (greedy decode, st_map_eval) against the float64 oracle.

Every step's full-vocabulary logits are compared with the oracle's greedy
decode over the same retained slots (the GPU's own retained index sets, so the
comparison isolates the decode), normwise: float32 model <= 1e-4, BF16 model
<= 2e-2, E4M3 cache <= 5e-2.  Tokens must agree until the first step whose oracle logits have a
near-tie at the top (gap below the tolerance times the largest logit): from
there on the sequences may legitimately differ, and the comparison stops for
that tuple.  Also: decoding n tokens gives the first n tokens of a longer
decode, bit for bit (prefix property), and the E4M3 retained cache decodes."""
import numpy as np
import pytest

from tests.util import normwise_rel

pytestmark = pytest.mark.gpu


def _env(model_name, table_cfg, n_tuples, seed, max_pos):
    import torch
    from oracle import operator as O
    from paper_2602_04430_b300 import build, stretto, synth
    build.build()
    cfg = synth.MODELS[model_name]
    w = synth.make_weights(cfg, seed=seed)
    table = synth.make_table(synth.TABLES[table_cfg], cfg.vocab, seed=seed + 1, n_tuples=n_tuples)
    model = stretto.Model(cfg, w, max_pos=max_pos)
    kv = model.kv_alloc(table["offsets"])
    kv.build(torch.from_numpy(table["tokens"]).cuda())
    torch.cuda.synchronize()
    off = table["offsets"]
    caches = {t: O.kv_build(cfg, w, table["tokens"][off[t]:off[t + 1]]) for t in range(len(off) - 1)}
    return dict(cfg=cfg, w=w, table=table, model=model, kv=kv, caches=caches, stretto=stretto, synth=synth)


def _compare(e, r, P, n_gen, tol, fp8=False):
    import torch
    from oracle import operator as O
    cfg, w, kv, model, st = e["cfg"], e["w"], e["kv"], e["model"], e["stretto"]
    off = e["table"]["offsets"]
    T = len(off) - 1
    kv.retain(r, st.ST_E4M3 if fp8 else None)
    R = int(off[-1])
    rank = kv.read(st.ST_VIEW_RANK, torch.int32, (cfg.layers, cfg.hkv, R)).cpu().numpy()
    op = model.operator(e["synth"].make_prompt(P, cfg.vocab, seed=91, r=r))
    ids = torch.arange(T, dtype=torch.int32, device="cuda")
    toks, logs = op.map(kv, ids, n_gen, with_logits=True)
    torch.cuda.synchronize()
    model.status()
    toks, logs = toks.cpu().numpy(), logs.cpu().numpy()
    full, steps = 0, 0
    for t in range(T):
        c = e["caches"][t]
        n = O.n_keep(c.L, r)
        idx = [[rank[l, g, off[t]:off[t] + n] for g in range(cfg.hkv)] for l in range(cfg.layers)]
        Kg, Vg, _ = O.retained_kv(c, r, idx=idx, kv_fp8=fp8)
        ref_t, ref_z = O.map_eval(cfg, w, c.L, Kg, Vg, op.op.prompt, n_gen)
        ok = True
        for s in range(n_gen):
            assert normwise_rel(logs[t, s], ref_z[s]) <= tol, (t, s, normwise_rel(logs[t, s], ref_z[s]))
            steps += 1
            if toks[t, s] != ref_t[s]:
                top2 = np.sort(ref_z[s])[-2:]
                assert top2[1] - top2[0] <= tol * max(1.0, np.abs(ref_z[s]).max()), (t, s)
                ok = False
                break
            assert int(np.argmax(logs[t, s])) == toks[t, s]
        full += ok
    return full, T, steps


def test_map_f32_matches_oracle():
    e = _env("tiny_f32", "tiny", 24, 92, 512)
    for r in (1.0, 0.5):
        full, T, steps = _compare(e, r, P=8, n_gen=6, tol=1e-4)
        print(f"r={r}: {full}/{T} tuples decoded identically, {steps} steps compared")
        assert full >= T - 2


def test_map_bf16_matches_oracle():
    e = _env("c2_bf16", "c2", 6, 93, 2200)
    full, T, steps = _compare(e, 1.0, P=16, n_gen=4, tol=2e-2)
    print(f"bf16: {full}/{T} tuples decoded identically, {steps} steps compared")
    assert steps >= T


def test_map_e4m3_matches_oracle():
    """E4M3 retained cache: the oracle decodes over the same slots dequantised
    per 64-slot block; logits within the E4M3 tolerance 5e-2."""
    e = _env("c2_bf16", "c2", 6, 96, 2200)
    full, T, steps = _compare(e, 0.5, P=16, n_gen=4, tol=5e-2, fp8=True)
    print(f"e4m3: {full}/{T} tuples decoded identically, {steps} steps compared")
    assert steps >= T


def test_map_prefix_and_e4m3():
    import torch
    e = _env("c2_bf16", "c2", 40, 94, 2200)
    st, kv, model = e["stretto"], e["kv"], e["model"]
    op = model.operator(e["synth"].make_prompt(24, e["cfg"].vocab, seed=95, r=0.5))
    ids = torch.arange(kv.T, dtype=torch.int32, device="cuda")
    for code in (st.ST_BF16, st.ST_E4M3):
        kv.retain(0.5, code)
        long = op.map(kv, ids, 6)
        short = op.map(kv, ids, 3)
        torch.cuda.synchronize()
        model.status()
        assert torch.equal(long[:, :3], short)
        assert int(long.min()) >= 0 and int(long.max()) < e["cfg"].vocab
    with pytest.raises(st.StrettoError):
        op.map(kv, ids, 0)
