"""Schedule independence of the persistent kernels (a race detector).

Every work item of the attention, projection and retention kernels is computed
by one CTA in a fixed order, so a tuple's results may not depend on which
other tuples share its launch, on the order in which the persistent grid walks
the items, or on how a build or an evaluation is cut into chunks.  These tests
run the config-2 decoder over a ragged lognormal table large enough that every
CTA walks many items (prefill: about 200 per CTA; evaluation: about 10) and
compare, bit for bit:
  * the cache built in one chunk against the cache built in many small chunks;
  * the retained BF16 and E4M3 caches of the two builds;
  * operator logits and labels of one launch over all tuples against launches
    over small, reordered slices, and against a run with a small evaluation
    chunk.
A slot, barrier-phase or buffer-reuse race shows up as a mismatch (or as the
device status of a timed-out bounded wait)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N_TUPLES = 768


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2602_04430_b300 import build, stretto, synth
    build.build()
    cfg = synth.MODELS["c2_bf16"]
    w = synth.make_weights(cfg, seed=31)
    table = synth.make_table(synth.TABLES["c2"], cfg.vocab, seed=32, n_tuples=N_TUPLES)
    model = stretto.Model(cfg, w, max_pos=2112)
    tok = torch.from_numpy(table["tokens"]).cuda()
    kv_one = model.kv_alloc(table["offsets"])
    kv_one.build(tok)
    torch.cuda.synchronize()
    model.status()
    # the same table through many small build chunks
    model.reserve(build_rows=20000)
    kv_many = model.kv_alloc(table["offsets"])
    kv_many.build(tok)
    torch.cuda.synchronize()
    model.status()
    return dict(cfg=cfg, table=table, model=model, kv_one=kv_one, kv_many=kv_many, stretto=stretto,
                synth=synth)


def _views(env, kv):
    import torch
    st, cfg = env["stretto"], env["cfg"]
    R = int(env["table"]["offsets"][-1])
    return {
        "K": kv.read(st.ST_VIEW_K, torch.bfloat16, (cfg.layers, cfg.hkv, R, cfg.hd)).cpu(),
        "V": kv.read(st.ST_VIEW_V, torch.bfloat16, (cfg.layers, cfg.hkv, R, cfg.hd)).cpu(),
        "scores": kv.read(st.ST_VIEW_SCORES, torch.float32, (cfg.layers, cfg.hkv, R)).cpu(),
        "pooled": kv.read(st.ST_VIEW_POOLED, torch.float32, (N_TUPLES, cfg.d)).cpu(),
    }


def test_build_independent_of_chunking(env):
    import torch
    a, b = _views(env, env["kv_one"]), _views(env, env["kv_many"])
    for name in a:
        assert torch.equal(a[name], b[name]), f"{name} differs between one and many build chunks"


@pytest.mark.parametrize("kv_dtype", ["bf16", "e4m3"])
def test_eval_independent_of_batch_and_order(env, kv_dtype):
    import torch
    st, synth, model = env["stretto"], env["synth"], env["model"]
    code = st.ST_E4M3 if kv_dtype == "e4m3" else st.ST_BF16
    for kv in (env["kv_one"], env["kv_many"]):
        kv.retain(0.5, code)
    torch.cuda.synchronize()
    model.status()
    op = model.operator(synth.make_prompt(32, env["cfg"].vocab, seed=33, r=0.5))
    ids = torch.arange(N_TUPLES, dtype=torch.int32, device="cuda")
    ref_logits, ref_labels = op.eval(env["kv_one"], ids)
    torch.cuda.synchronize()
    model.status()
    ref_logits, ref_labels = ref_logits.cpu(), ref_labels.cpu()
    # the other build, in reversed slices of 61 tuples
    logits = torch.empty_like(ref_logits)
    labels = torch.empty_like(ref_labels)
    order = list(range(N_TUPLES))[::-1]
    for s in range(0, N_TUPLES, 61):
        sl = torch.tensor(order[s:s + 61], dtype=torch.int32, device="cuda")
        lg, lb = op.eval(env["kv_many"], sl)
        logits[sl.cpu().long()] = lg.cpu()
        labels[sl.cpu().long()] = lb.cpu()
    torch.cuda.synchronize()
    model.status()
    assert torch.equal(logits, ref_logits), "logits depend on the batch composition or order"
    assert torch.equal(labels, ref_labels)
    # one call cut into small evaluation chunks (16 tuples of 32 prompt rows)
    model.reserve(eval_rows=16 * 32)
    lg, lb = op.eval(env["kv_one"], ids)
    torch.cuda.synchronize()
    model.status()
    model.reserve(eval_rows=1 << 18)
    assert torch.equal(lg.cpu(), ref_logits), "logits depend on the evaluation chunking"
    assert torch.equal(lb.cpu(), ref_labels)


def test_retained_caches_independent_of_build_chunking(env):
    import torch
    st, cfg = env["stretto"], env["cfg"]
    for code, dt, esz in ((st.ST_BF16, torch.bfloat16, 2), (st.ST_E4M3, torch.uint8, 1)):
        views = []
        for kv in (env["kv_one"], env["kv_many"]):
            kv.retain(0.25, code)
            torch.cuda.synchronize()
            n = kv.view_bytes(st.ST_VIEW_KR) // esz
            views.append((kv.read(st.ST_VIEW_KR, dt, (n,)).cpu(), kv.read(st.ST_VIEW_VR, dt, (n,)).cpu()))
        env["model"].status()
        assert torch.equal(views[0][0], views[1][0]) and torch.equal(views[0][1], views[1][1])
