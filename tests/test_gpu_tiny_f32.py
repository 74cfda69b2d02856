"""FP32 parity of the whole path on the tiny model (2 layers, d 128, 4 heads x 32,
64 tuples of 256 tokens, 16-token prompt, r in {1.0, 0.5}) against the FP64
oracle: cache contents, retention (bit-exact on the kernel's own scores), label
logits (normwise relative error <= 1e-4) and decisions."""
import numpy as np
import pytest

from tests.util import check_retained_vs_oracle, decide_f32, normwise_rel

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def run():
    import torch
    from oracle import operator as O
    from paper_2602_04430_b300 import build, stretto, synth
    build.build()
    cfg = synth.MODELS["tiny_f32"]
    w = synth.make_weights(cfg, seed=1)
    table = synth.make_table(synth.TABLES["tiny"], cfg.vocab, seed=2)
    model = stretto.Model(cfg, w, max_pos=512)
    kv = model.kv_alloc(table["offsets"])
    tok = torch.from_numpy(table["tokens"]).cuda()
    kv.build(tok)
    torch.cuda.synchronize()
    model.status()
    caches = {}
    for t in range(table["offsets"].shape[0] - 1):
        a, b = table["offsets"][t], table["offsets"][t + 1]
        caches[t] = O.kv_build(cfg, w, table["tokens"][a:b])
    return dict(cfg=cfg, w=w, table=table, model=model, kv=kv, caches=caches, torch=torch)


def _full(run, view):
    import torch
    cfg, kv = run["cfg"], run["kv"]
    R = int(run["table"]["offsets"][-1])
    from paper_2602_04430_b300 import stretto
    if view in (stretto.ST_VIEW_K, stretto.ST_VIEW_V):
        return kv.read(view, torch.float32, (cfg.layers, cfg.hkv, R, cfg.hd)).cpu().numpy()
    if view == stretto.ST_VIEW_SCORES:
        return kv.read(view, torch.float32, (cfg.layers, cfg.hkv, R)).cpu().numpy()
    if view == stretto.ST_VIEW_RANK:
        return kv.read(view, torch.int32, (cfg.layers, cfg.hkv, R)).cpu().numpy()
    raise ValueError(view)


def test_cache_matches_oracle(run):
    from paper_2602_04430_b300 import stretto
    import torch
    cfg, off = run["cfg"], run["table"]["offsets"]
    K, V, S = (_full(run, v) for v in (stretto.ST_VIEW_K, stretto.ST_VIEW_V, stretto.ST_VIEW_SCORES))
    pooled = run["kv"].read(stretto.ST_VIEW_POOLED, torch.float32, (len(off) - 1, cfg.d)).cpu().numpy()
    for t, c in run["caches"].items():
        a, b = off[t], off[t + 1]
        for l in range(cfg.layers):
            for g in range(cfg.hkv):
                assert normwise_rel(K[l, g, a:b], c.k[l][g]) <= TOL
                assert normwise_rel(V[l, g, a:b], c.v[l][g]) <= TOL
                assert normwise_rel(S[l, g, a:b], c.scores[l][g]) <= TOL
        assert normwise_rel(pooled[t], c.pooled) <= TOL


@pytest.mark.parametrize("r", [1.0, 0.5])
def test_retention_bit_exact_and_gather(run, r):
    import torch
    from oracle import operator as O
    from paper_2602_04430_b300 import stretto
    cfg, off, kv = run["cfg"], run["table"]["offsets"], run["kv"]
    kv.retain(r)
    kv.status()
    S = _full(run, stretto.ST_VIEW_SCORES)
    K = _full(run, stretto.ST_VIEW_K)
    rank = _full(run, stretto.ST_VIEW_RANK)
    T = len(off) - 1
    offp = kv.read(stretto.ST_VIEW_OFFP, torch.int64, (T + 1,)).cpu().numpy()
    nk = kv.read(stretto.ST_VIEW_NKEEP, torch.int32, (T,)).cpu().numpy()
    rp_cap = kv.view_bytes(stretto.ST_VIEW_KR) // (4 * cfg.layers * cfg.hkv * cfg.hd)
    Kr = kv.read(stretto.ST_VIEW_KR, torch.float32, (cfg.layers, cfg.hkv, rp_cap, cfg.hd)).cpu().numpy()
    swaps = 0
    for t in range(T):
        a, b = off[t], off[t + 1]
        n = O.n_keep(b - a, r)
        assert nk[t] == n
        assert offp[t + 1] - offp[t] == (n + 63) // 64 * 64
        for l in range(cfg.layers):
            for g in range(cfg.hkv):
                seg = S[l, g, a:b]
                # (i) the kernel's ranking of its own float32 scores == brute-force sort
                assert rank[l, g, a:b].tolist() == O.rank_order(seg).tolist()
                # (ii) against the FP64 oracle's scores: equal up to boundary near-ties
                swaps += check_retained_vs_oracle(rank[l, g, a:b], run["caches"][t].scores[l][g], n)
                idx = rank[l, g, a:a + n]
                np.testing.assert_array_equal(Kr[l, g, offp[t]:offp[t] + n], K[l, g, a + idx])
                np.testing.assert_array_equal(Kr[l, g, offp[t] + n:offp[t + 1]], 0.0)
    print(f"r={r}: boundary near-tie exchanges vs oracle: {swaps}")


@pytest.mark.parametrize("r", [1.0, 0.5])
def test_op_eval_matches_oracle(run, r):
    import torch
    from oracle import operator as O
    from paper_2602_04430_b300 import stretto, synth
    cfg, w, off, kv, model = run["cfg"], run["w"], run["table"]["offsets"], run["kv"], run["model"]
    T = len(off) - 1
    op = synth.make_prompt(16, cfg.vocab, seed=3, label_ids=(1, 0), r=r, theta_pos=0.05, theta_neg=-0.05)
    kv.retain(r)
    rank = _full(run, stretto.ST_VIEW_RANK)
    opr = model.operator(op)
    ids = torch.arange(T, dtype=torch.int32, device="cuda")
    logits, labels = opr.eval(kv, ids)
    torch.cuda.synchronize()
    z = logits.cpu().numpy()
    lab = labels.cpu().numpy()
    # decisions are the kernel's float32 decisions of its own logits
    np.testing.assert_array_equal(lab, decide_f32(z, op.theta_pos, op.theta_neg))
    z_own, z_gpuidx = [], []
    for t in range(T):
        c = run["caches"][t]
        Kr, Vr, _ = O.retained_kv(c, r)
        z_own.append(O.op_eval(cfg, w, c.L, Kr, Vr, op.prompt, op.label_ids))
        n = O.n_keep(c.L, r)
        idx = [[rank[l, g, off[t]:off[t] + n] for g in range(cfg.hkv)] for l in range(cfg.layers)]
        Kg, Vg, _ = O.retained_kv(c, r, idx=idx)
        z_gpuidx.append(O.op_eval(cfg, w, c.L, Kg, Vg, op.prompt, op.label_ids))
    assert normwise_rel(z, np.array(z_gpuidx)) <= TOL
    assert normwise_rel(z, np.array(z_own)) <= TOL
    ref_lab = np.array([O.decide(op, zz) for zz in z_own])
    agree = float(np.mean(ref_lab == lab))
    assert agree >= 0.95, agree


def test_subset_and_order_of_tuple_ids(run):
    """Evaluating a permuted subset gives the same per-tuple logits as the full table."""
    import torch
    from paper_2602_04430_b300 import synth
    cfg, kv, model = run["cfg"], run["kv"], run["model"]
    kv.retain(0.5)
    op = synth.make_prompt(16, cfg.vocab, seed=3, label_ids=(1, 0), r=0.5)
    opr = model.operator(op)
    full, _ = opr.eval(kv, torch.arange(64, dtype=torch.int32, device="cuda"))
    sub = torch.tensor([63, 0, 17, 17, 5], dtype=torch.int32, device="cuda")
    part, _ = opr.eval(kv, sub)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(part.cpu().numpy(), full.cpu().numpy()[[63, 0, 17, 17, 5]])


def test_bounded_wait_timeout_is_reported_and_recoverable(run):
    """The failure path without a fault: a device wait on a barrier that nothing
    completes gives up after its cycle limit, st_status reports ST_ETIMEOUT once,
    and the context keeps working (the same operator evaluation afterwards)."""
    import torch
    from paper_2602_04430_b300 import stretto, synth
    model, kv = run["model"], run["kv"]
    model.status()                                   # clean before
    model.selftest_wait(limit_cycles=2_000_000)
    torch.cuda.synchronize()
    with pytest.raises(stretto.StrettoError) as e:
        model.status()
    assert e.value.code == stretto.ST_ETIMEOUT
    model.status()                                   # reported once, then clear
    kv.retain(1.0)
    op = model.operator(synth.make_prompt(16, run["cfg"].vocab, seed=5, r=1.0))
    ids = torch.arange(kv.T, dtype=torch.int32, device="cuda")
    lg, lb = op.eval(kv, ids)
    torch.cuda.synchronize()
    model.status()
    assert torch.isfinite(lg).all()
    with pytest.raises(stretto.StrettoError):
        model.selftest_wait(limit_cycles=10)         # limit out of range


def test_out_of_range_token_is_reported_not_read(run):
    """A token id outside [0, vocab) in the table is caught by the embedding's
    own bounds check: it embeds as zeros, st_status reports ST_EINVAL once, and
    the context keeps working."""
    import torch
    from paper_2602_04430_b300 import stretto, synth
    cfg, model = run["cfg"], run["model"]
    table = synth.make_table(synth.TABLES["tiny"], cfg.vocab, seed=7, n_tuples=4)
    tok = table["tokens"].copy()
    tok[3], tok[-1] = cfg.vocab, -1
    model.status()
    kv = model.kv_alloc(table["offsets"])
    kv.build(torch.from_numpy(tok).cuda())
    torch.cuda.synchronize()
    with pytest.raises(stretto.StrettoError) as e:
        model.status()
    assert e.value.code == stretto.ST_EINVAL
    model.status()
    kv.build(torch.from_numpy(table["tokens"]).cuda())
    kv.retain(1.0)
    op = model.operator(synth.make_prompt(16, cfg.vocab, seed=8, r=1.0))
    lg, _ = op.eval(kv, torch.arange(kv.T, dtype=torch.int32, device="cuda"))
    torch.cuda.synchronize()
    model.status()
    assert torch.isfinite(lg).all()


def test_out_of_range_tuple_id_is_reported_not_read(run):
    """A tuple id outside [0, T) is caught by the planning kernels' bounds
    check: it is evaluated as tuple 0 (no read leaves the cache), st_status
    reports ST_ERANGE once, and the other ids' results are unchanged."""
    import torch
    from paper_2602_04430_b300 import stretto, synth
    cfg, kv, model = run["cfg"], run["kv"], run["model"]
    kv.retain(1.0)
    opr = model.operator(synth.make_prompt(16, cfg.vocab, seed=9, label_ids=(1, 0), r=1.0))
    model.status()
    good = torch.tensor([5, 0, 9], dtype=torch.int32, device="cuda")
    ref, _ = opr.eval(kv, good)
    torch.cuda.synchronize()
    model.status()
    for bad in (kv.T, -1, 1 << 30):
        ids = torch.tensor([5, bad, 9], dtype=torch.int32, device="cuda")
        lg, _ = opr.eval(kv, ids)
        torch.cuda.synchronize()
        with pytest.raises(stretto.StrettoError) as e:
            model.status()
        assert e.value.code == stretto.ST_ERANGE
        model.status()                               # reported once, then clear
        np.testing.assert_array_equal(lg.cpu().numpy(), ref.cpu().numpy())


def test_kv_alloc_validates_offsets(run):
    """Empty documents, documents past max_pos - 1, a nonzero first offset and
    an empty table are refused on the host, before any device work."""
    import numpy as np
    from paper_2602_04430_b300 import stretto
    model = run["model"]                       # max_pos 512
    for off in ([0, 3, 3, 7], [0, 600], [1, 5], [0]):
        with pytest.raises(stretto.StrettoError) as ei:
            model.kv_alloc(np.asarray(off, dtype=np.int64))
        assert ei.value.code == stretto.ST_EINVAL, off
    model.kv_alloc(np.asarray([0, 1, 511], dtype=np.int64)).close()


def test_caller_owned_workspace():
    """st_workspace_size / st_set_workspace: with caller-owned build and eval
    workspaces sized for st_reserve's chunks, kv_build + retain + op_eval give
    the same results bit for bit as with library-owned workspace; a workspace
    too small for a chunk is refused with ST_ENOMEM before anything runs; NULL
    returns to library-owned workspace; a misaligned buffer is rejected."""
    import torch
    from paper_2602_04430_b300 import build, stretto, synth
    build.build()
    cfg = synth.MODELS["tiny_f32"]
    w = synth.make_weights(cfg, seed=91)
    table = synth.make_table(synth.TABLES["tiny"], cfg.vocab, seed=92, n_tuples=16)
    tok = torch.from_numpy(table["tokens"]).cuda()
    op_np = synth.make_prompt(16, cfg.vocab, seed=93, r=0.5)

    def run_model(caller_ws):
        m = stretto.Model(cfg, w, max_pos=512)
        m.reserve(build_rows=1024, eval_rows=128)     # 4 build chunks, 2 eval chunks
        if caller_ws:
            bb = m.workspace_size(stretto.ST_WS_BUILD, 1024)
            eb = m.workspace_size(stretto.ST_WS_EVAL, 128)
            assert bb > 0 and eb > 0
            m.set_workspace(stretto.ST_WS_BUILD, torch.empty(bb, dtype=torch.uint8, device="cuda"))
            m.set_workspace(stretto.ST_WS_EVAL, torch.empty(eb, dtype=torch.uint8, device="cuda"))
        kv = m.kv_alloc(table["offsets"])
        kv.build(tok)
        kv.retain(0.5)
        op = m.operator(op_np)
        lg, lb = op.eval(kv, torch.arange(kv.T, dtype=torch.int32, device="cuda"))
        torch.cuda.synchronize()
        m.status()
        return m, kv, lg.clone(), lb.clone()

    _, _, lg0, lb0 = run_model(False)
    m, kv, lg1, lb1 = run_model(True)
    assert torch.equal(lg0, lg1) and torch.equal(lb0, lb1)
    m.set_workspace(stretto.ST_WS_BUILD, torch.empty(4096, dtype=torch.uint8, device="cuda"))
    with pytest.raises(stretto.StrettoError) as e:
        kv.build(tok)
    assert e.value.code == stretto.ST_ENOMEM
    m.set_workspace(stretto.ST_WS_BUILD, None)
    kv.build(tok)
    torch.cuda.synchronize()
    m.status()
    with pytest.raises(stretto.StrettoError) as e:
        m.set_workspace(stretto.ST_WS_EVAL, torch.empty(1024, dtype=torch.uint8, device="cuda")[1:])
    assert e.value.code == stretto.ST_EINVAL


def test_kv_indices_are_the_retained_sets(run):
    """st_kv_indices: at r = 0.5, 0.25 and 1 the offsets are the prefix sums of
    n_keep(L, r) and every (layer, kv head, tuple) lists its top n_keep slots by
    (score desc, index asc) on the kernel's own scores, in that order; smaller r
    gives prefixes (nested sets); before any retain the call is refused."""
    import torch
    from oracle import operator as O
    from paper_2602_04430_b300 import stretto, synth
    cfg, model = run["cfg"], run["model"]
    table = synth.make_table_from_lengths([1, 2, 37, 64, 65, 200], cfg.vocab, seed=95)
    kv = model.kv_alloc(table["offsets"])
    kv.build(torch.from_numpy(table["tokens"]).cuda())
    with pytest.raises(stretto.StrettoError) as e:
        kv.indices(0.5)
    assert e.value.code == stretto.ST_EINVAL
    model.status()
    kv.retain(0.5)
    off_h = table["offsets"]
    R = int(off_h[-1])
    S = kv.read(stretto.ST_VIEW_SCORES, torch.float32, (cfg.layers, cfg.hkv, R)).cpu().numpy()
    prev = None
    for r in (1.0, 0.5, 0.25):
        idx, off = kv.indices(r)
        idx, off = idx.cpu().numpy(), off.cpu().numpy()
        n = [O.n_keep(int(off_h[t + 1] - off_h[t]), r) for t in range(len(off_h) - 1)]
        assert list(off) == [0] + list(np.cumsum(n))
        for l in range(cfg.layers):
            for g in range(cfg.hkv):
                for t in range(len(n)):
                    seg = S[l, g, off_h[t]:off_h[t + 1]]
                    want = np.lexsort((np.arange(len(seg)), -seg))[:n[t]]
                    got = idx[l, g, off[t]:off[t + 1]]
                    assert np.array_equal(got, want)
                    if prev is not None:
                        p_idx, p_off = prev
                        assert np.array_equal(got, p_idx[l, g, p_off[t]:p_off[t] + n[t]])
        prev = (idx, off)
    torch.cuda.synchronize()
    model.status()


def test_operator_arguments_are_validated(run):
    """st_op_create refuses, with ST_EINVAL and without touching the device,
    prompt or label ids outside [0, vocab), an empty or over-long prompt, r
    outside (0, 1], and label counts other than 2 (filter) or 2..8
    (classify); the context keeps working afterwards."""
    import dataclasses
    import torch
    from paper_2602_04430_b300 import stretto, synth
    cfg, model, kv = run["cfg"], run["model"], run["kv"]
    good = synth.make_prompt(16, cfg.vocab, seed=97, label_ids=(1, 0), r=1.0)
    bad = [
        dataclasses.replace(good, prompt=good.prompt[:-1] + (cfg.vocab,)),
        dataclasses.replace(good, prompt=(-1,) + good.prompt[1:]),
        dataclasses.replace(good, label_ids=(1, cfg.vocab)),
        dataclasses.replace(good, prompt=()),
        dataclasses.replace(good, prompt=tuple(range(257))),
        dataclasses.replace(good, r=0.0),
        dataclasses.replace(good, r=1.5),
        dataclasses.replace(good, label_ids=(1, 0, 2)),
        dataclasses.replace(good, kind="classify", label_ids=tuple(range(9)), bias=None),
        dataclasses.replace(good, kind="classify", label_ids=(3,), bias=None),
    ]
    for op in bad:
        with pytest.raises(stretto.StrettoError) as e:
            model.operator(op)
        assert e.value.code == stretto.ST_EINVAL
    kv.retain(1.0)
    lg, _ = model.operator(good).eval(kv, torch.arange(kv.T, dtype=torch.int32, device="cuda"))
    torch.cuda.synchronize()
    model.status()
    assert bool(torch.isfinite(lg).all())
