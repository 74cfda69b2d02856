"""Batched evaluation of several operators (st_op_eval_multi).

Three operators shaped like the batching workload — a binary filter with a
16-token prompt at r = 0.1, an 8-way classify with 48 tokens at r = 0.3 and a
binary filter with 64 tokens at r = 1.0 — each over its own tuple set, share
one pass over one retained profile (r = 1, rank order; each operator reads its
own n_keep prefix).  Every pair is computed exactly as by a single-operator
call, so the logits and labels must equal separate st_op_eval calls bit for
bit: on the BF16 decoder with BF16 and E4M3 retained caches (tensor-core path,
including the 64-token prompt whose 4 x 64 query rows take two 128-row
attention blocks) and on the float32 decoder (CUDA-core path)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ops(synth, vocab):
    return [
        synth.make_prompt(16, vocab, seed=41, label_ids=(1, 0), r=0.1),
        synth.make_prompt(48, vocab, seed=42, label_ids=tuple(range(2, 10)), r=0.3, kind="classify",
                          bias=[0.01 * k for k in range(8)]),
        synth.make_prompt(64, vocab, seed=43, label_ids=(3, 4), r=1.0),
    ]


def _sets(T, torch):
    ids0 = np.arange(T)
    ids1 = np.arange(T)[::3][::-1].copy()
    ids2 = np.arange(min(T, 77))
    return [torch.tensor(x, dtype=torch.int32, device="cuda") for x in (ids0, ids1, ids2)]


def _check(model, kv, ops_np, synth, stretto, torch):
    ops = [model.operator(o) for o in ops_np]
    sets = _sets(kv.T, torch)
    multi_lg, multi_lb = stretto.eval_multi(model, kv, ops, sets)
    torch.cuda.synchronize()
    model.status()
    for op, ids, lg, lb in zip(ops, sets, multi_lg, multi_lb):
        lg1, lb1 = op.eval(kv, ids)
        torch.cuda.synchronize()
        assert torch.equal(lg.cpu(), lg1.cpu()), "batched logits differ from a single-operator call"
        assert torch.equal(lb.cpu(), lb1.cpu())
    model.status()
    return multi_lg, multi_lb


@pytest.fixture(scope="module")
def bf16_env():
    import torch
    from paper_2602_04430_b300 import build, stretto, synth
    build.build()
    cfg = synth.MODELS["c2_bf16"]
    table = synth.make_table_from_lengths([1, 2, 37, 63, 64, 65, 130, 257, 600, 1000, 2048] * 9,
                                          cfg.vocab, seed=44, ids="zipf")
    model = stretto.Model(cfg, synth.make_weights(cfg, seed=45), max_pos=2200)
    kv = model.kv_alloc(table["offsets"])
    kv.build(torch.from_numpy(table["tokens"]).cuda())
    torch.cuda.synchronize()
    return dict(cfg=cfg, model=model, kv=kv, synth=synth, stretto=stretto, torch=torch)


@pytest.mark.parametrize("kv_dtype", ["bf16", "e4m3"])
def test_multi_equals_single_bf16(bf16_env, kv_dtype):
    e = bf16_env
    st = e["stretto"]
    e["kv"].retain(1.0, st.ST_E4M3 if kv_dtype == "e4m3" else st.ST_BF16)
    lg, lb = _check(e["model"], e["kv"], _ops(e["synth"], e["cfg"].vocab), e["synth"], st, e["torch"])
    # the classify operator produces classes, the filters accept / reject / unsure
    assert set(lb[1].cpu().tolist()) <= set(range(8))
    assert set(lb[0].cpu().tolist()) <= {0, 1, 2}


def test_multi_small_eval_chunks(bf16_env):
    # pairs of different operators share chunk boundaries
    e = bf16_env
    st = e["stretto"]
    e["kv"].retain(1.0, st.ST_BF16)
    e["model"].reserve(eval_rows=1000)
    try:
        _check(e["model"], e["kv"], _ops(e["synth"], e["cfg"].vocab), e["synth"], st, e["torch"])
    finally:
        e["model"].reserve(eval_rows=1 << 18)


def test_multi_equals_single_f32():
    import torch
    from paper_2602_04430_b300 import build, stretto, synth
    build.build()
    cfg = synth.MODELS["tiny_f32"]
    table = synth.make_table(synth.TABLES["tiny"], cfg.vocab, seed=46)
    model = stretto.Model(cfg, synth.make_weights(cfg, seed=47), max_pos=512)
    kv = model.kv_alloc(table["offsets"])
    kv.build(torch.from_numpy(table["tokens"]).cuda())
    kv.retain(1.0)
    torch.cuda.synchronize()
    _check(model, kv, _ops(synth, cfg.vocab), synth, stretto, torch)


def test_multi_rejects_bad_arguments(bf16_env):
    e = bf16_env
    st, torch = e["stretto"], e["torch"]
    e["kv"].retain(0.5, st.ST_BF16)
    ops = [e["model"].operator(o) for o in _ops(e["synth"], e["cfg"].vocab)]
    sets = _sets(e["kv"].T, torch)
    with pytest.raises(st.StrettoError):
        st.eval_multi(e["model"], e["kv"], ops, sets)      # r = 1.0 above the retained 0.5
    with pytest.raises(st.StrettoError):
        st.eval_multi(e["model"], e["kv"], ops[:1] * 9, sets[:1] * 9)   # more than 8 operators


def test_graph_replay_equals_eager(bf16_env):
    """A captured batched evaluation replays to the eager results, also after the
    tuple-id buffers are rewritten in place, and counts its kernels per replay."""
    e = bf16_env
    st, torch = e["stretto"], e["torch"]
    e["kv"].retain(1.0, st.ST_BF16)
    model, kv = e["model"], e["kv"]
    ops = [model.operator(o) for o in _ops(e["synth"], e["cfg"].vocab)]
    sets = _sets(kv.T, torch)
    g = st.Graph(model, kv, ops, sets)
    assert g.launches() > 0
    n0 = model.launch_count()
    for _ in range(2):
        g.launch()
    torch.cuda.synchronize()
    model.status()
    assert model.launch_count() - n0 == 2 * g.launches()
    ref_lg, ref_lb = st.eval_multi(model, kv, ops, sets)
    torch.cuda.synchronize()
    for a, b in zip(g.logits, ref_lg):
        assert torch.equal(a.cpu(), b.cpu())
    for a, b in zip(g.labels, ref_lb):
        assert torch.equal(a.cpu(), b.cpu())
    # other tuples in the same buffers
    for t in sets:
        t.copy_(torch.flip(t, [0]) % kv.T)
    g.launch()
    ref_lg, ref_lb = st.eval_multi(model, kv, ops, sets)
    torch.cuda.synchronize()
    model.status()
    for a, b in zip(g.logits, ref_lg):
        assert torch.equal(a.cpu(), b.cpu())
    g.close()


def test_autotune_schedules_agree(bf16_env):
    """Every schedule the autotuner tries gives the same results bit for bit; the
    chosen one is the fastest it timed and stays set."""
    e = bf16_env
    st, torch = e["stretto"], e["torch"]
    e["kv"].retain(1.0, st.ST_BF16)
    model, kv = e["model"], e["kv"]
    ops = [model.operator(o) for o in _ops(e["synth"], e["cfg"].vocab)]
    sets = _sets(kv.T, torch)
    st.set_schedule(model)
    ref_lg, ref_lb = st.eval_multi(model, kv, ops, sets)
    torch.cuda.synchronize()
    best, tried = st.autotune(model, kv, ops, sets)
    model.status()
    assert len(tried) >= 4 and best["ms"] == min(t["ms"] for t in tried)
    for sc in tried:
        st.set_schedule(model, sc["eval_rows"], sc["attn_nb"], sc["longest_first"], sc["split_keys"])
        lg, lb = st.eval_multi(model, kv, ops, sets)
        torch.cuda.synchronize()
        model.status()
        for a, b in zip(lg, ref_lg):
            assert torch.equal(a.cpu(), b.cpu()), f"schedule {sc} changes the logits"
    st.set_schedule(model)
