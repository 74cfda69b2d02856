"""Retained-profile repository (st_kv_export / st_kv_import): a profile saved
from one cache and loaded into a fresh, never-built cache of the same table
evaluates operators bit for bit like the original (BF16 and E4M3 profiles,
operators at the profile's r and below, pooled states included); blobs of
another table or model, truncated or corrupted blobs are refused."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _setup(model_name, table_cfg, n, seed, max_pos):
    import torch
    from paper_2602_04430_b300 import build, stretto, synth
    build.build()
    cfg = synth.MODELS[model_name]
    table = synth.make_table(synth.TABLES[table_cfg], cfg.vocab, seed=seed, n_tuples=n)
    model = stretto.Model(cfg, synth.make_weights(cfg, seed=seed + 1), max_pos=max_pos)
    kv = model.kv_alloc(table["offsets"])
    kv.build(torch.from_numpy(table["tokens"]).cuda())
    return cfg, table, model, kv, stretto, synth, torch


def _evals(model, kv, ops, torch):
    ids = torch.arange(kv.T, dtype=torch.int32, device="cuda")
    out = []
    for op in ops:
        lg, lb = op.eval(kv, ids)
        out.append((lg.clone(), lb.clone()))
    torch.cuda.synchronize()
    model.status()
    return out


@pytest.mark.parametrize("model_name,table_cfg,codes", [("c2_bf16", "c2", ("bf16", "e4m3")),
                                                         ("tiny_f32", "tiny", ("f32",))])
def test_profile_roundtrip_is_bit_exact(tmp_path, model_name, table_cfg, codes):
    cfg, table, model, kv, st, synth, torch = _setup(model_name, table_cfg, 48, 401, 2200)
    code_of = {"bf16": st.ST_BF16, "e4m3": st.ST_E4M3, "f32": st.ST_F32}
    ops = [model.operator(synth.make_prompt(16, cfg.vocab, seed=402, r=r)) for r in (0.5, 0.25)]
    for name in codes:
        kv.retain(0.5, code_of[name])
        want = _evals(model, kv, ops, torch)
        path = str(tmp_path / f"profile_{name}.bin")
        kv.save_profile(path)
        fresh = model.kv_alloc(table["offsets"])
        fresh.load_profile(path)
        got = _evals(model, fresh, ops, torch)
        for (a, b), (c, d) in zip(want, got):
            assert torch.equal(a, c) and torch.equal(b, d)
        P1 = kv.read(st.ST_VIEW_POOLED, torch.float32, (kv.T, cfg.d))
        P2 = fresh.read(st.ST_VIEW_POOLED, torch.float32, (kv.T, cfg.d))
        assert torch.equal(P1, P2)
        # the profile holds no full cache: retaining again needs a build
        with pytest.raises(st.StrettoError) as ei:
            fresh.retain(0.25)
        assert ei.value.code == st.ST_EINVAL


def test_profile_blobs_are_validated():
    cfg, table, model, kv, st, synth, torch = _setup("c2_bf16", "c2", 24, 411, 2200)
    kv.retain(0.5)
    blob = kv.export_profile()
    fresh = model.kv_alloc(table["offsets"])

    def refused(b, target=fresh):
        with pytest.raises(st.StrettoError) as ei:
            target.import_profile(b)
        assert ei.value.code == st.ST_EINVAL

    refused(blob[:-1])                           # truncated
    bad = blob.copy()
    bad[0] ^= 0xFF                               # magic
    refused(bad)
    other = synth.make_table(synth.TABLES["c2"], cfg.vocab, seed=412, n_tuples=24)
    refused(blob, model.kv_alloc(other["offsets"]))   # another table
    # a retained count beyond its document: header 128 B, offsets and padded
    # offsets (T+1 int64 each), then the int32 counts
    T = kv.T
    bad = blob.copy()
    nk = bad[128 + 16 * (T + 1):128 + 16 * (T + 1) + 4 * T].view(np.int32)
    nk[0] = int(table["offsets"][1] - table["offsets"][0]) + 1
    refused(bad)
    # another model shape
    tiny = synth.MODELS["tiny_f32"]
    m2 = st.Model(tiny, synth.make_weights(tiny, seed=413), max_pos=2200)
    refused(blob, m2.kv_alloc(table["offsets"]))
    # the intact blob still loads
    fresh.import_profile(blob)


def test_second_profile_of_one_cache():
    """st_kv_profile_alloc: a BF16 profile in the cache itself and an E4M3
    profile in a second handle over the same full cache, resident at once, each
    evaluate bit for bit like the cache re-retained in that dtype; the profile
    refuses r above its r_max, a build, an import and query scoring."""
    cfg, table, model, kv, st, synth, torch = _setup("c2_bf16", "c2", 48, 411, 2200)
    ops = [model.operator(synth.make_prompt(16, cfg.vocab, seed=412, r=r)) for r in (0.5, 0.25)]
    kv.retain(0.5, st.ST_E4M3)
    want_e4m3 = _evals(model, kv, ops, torch)
    kv.retain(0.5, st.ST_BF16)
    want_bf16 = _evals(model, kv, ops, torch)
    prof = kv.profile(0.5)
    prof.retain(0.5, st.ST_E4M3)
    for _ in range(2):      # interleaved: neither retained cache disturbs the other
        got_e4m3 = _evals(model, prof, ops, torch)
        got_bf16 = _evals(model, kv, ops, torch)
        for (a, b), (c, d) in zip(got_e4m3 + got_bf16, want_e4m3 + want_bf16):
            assert torch.equal(a, c) and torch.equal(b, d)
    with pytest.raises(st.StrettoError):
        prof.retain(0.75, st.ST_E4M3)
    with pytest.raises(st.StrettoError):
        prof.build(torch.from_numpy(table["tokens"]).cuda())
    with pytest.raises(st.StrettoError):
        prof.import_profile(kv.export_profile())
    blob = prof.export_profile()
    fresh = model.kv_alloc(table["offsets"])
    fresh.import_profile(blob)
    for (a, b), (c, d) in zip(_evals(model, fresh, ops, torch), want_e4m3):
        assert torch.equal(a, c) and torch.equal(b, d)
    prof.close()
    fresh.close()
    kv.close()
    model.close()
