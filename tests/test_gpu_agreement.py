"""Label agreement and label-logit error against the unmodified float64 oracle.

The oracle here runs as it stands -- its own float64 cache, its own ranking of
its own scores, E4M3 codes decided from its exact keys and values -- on a
seeded subsample of a configuration's table (run over host processes by
``oracle.pool``).  The CUDA path runs the whole table in the benchmark's launch
configuration.  Compared per sampled tuple:

* decisions at the calibrated threshold: theta+ = theta- = theta, the median
  oracle margin z('1') - z('0') over the sample (the optimizer tunes log-odds
  thresholds, Sec. 4.1; the median puts the most tuples near the threshold,
  the hardest setting for agreement), and at theta = 0;
* the label logits, normwise over the sample (max |dz| / max |z_oracle|):
  the bound applies to the oracle evaluated over the GPU's retained sets (the
  ranking is an integer decision that the kernel takes in float32 from its own
  BF16 cache, so near-ties at the boundary fall either way), for the E4M3
  variant likewise (its codes decided from the oracle's exact values); the
  error against the oracle's own ranking, which adds those exchanges, is
  reported (and bounded on the 8-layer model);
* the retained sets (BF16 cache) against the oracle's ranking: an exchanged
  slot is allowed only where the two scorings can disagree, i.e. where the
  oracle score lies within twice the largest GPU-oracle score difference of the
  oracle's boundary score; the mean overlap is reported.

Bars: BF16 logits <= 2e-2 with >= 99.5 % agreement; E4M3 KV
<= 5e-2 with >= 99 % agreement, against the oracle's own E4M3 variant.
"""
import numpy as np
import pytest

from tests.util import normwise_rel

pytestmark = pytest.mark.gpu

N_C2 = 256      # sampled tuples of the 8-layer table
N_C3 = 32       # sampled tuples of the 16-layer table


def _decide(z, theta):
    from oracle import operator as O
    return np.array([O.decide_filter(float(a), float(b), theta, theta) for a, b in z], dtype=np.int32)


def _retained_overlap(rank_rows, scores_gpu, scores_or, n):
    """Per (layer, kv head): overlap of the GPU's first n ranked slots with the
    oracle's; exchanged slots must sit within the scorings' disagreement band."""
    from oracle import operator as O
    overlaps, exchanged = [], 0
    for l in range(len(rank_rows)):
        for g in range(len(rank_rows[l])):
            s = np.asarray(scores_or[l][g], dtype=np.float64)
            ref = O.rank_order(s)[:n]
            gpu = np.asarray(rank_rows[l][g][:n])
            a, b = set(gpu.tolist()), set(ref.tolist())
            overlaps.append(len(a & b) / n)
            diff = a ^ b
            if diff:
                band = 2.0 * float(np.abs(np.asarray(scores_gpu[l][g], np.float64) - s).max()) + 1e-9
                kth = s[ref[-1]]
                for j in diff:
                    assert abs(s[j] - kth) <= band, (l, g, j, s[j], kth, band)
                exchanged += len(diff) // 2
    return float(np.mean(overlaps)), exchanged


def _run(model_key, table_key, table_seed, weight_seed, op_seed, r, n_sample, sample_seed,
         n_tuples=None, max_pos=2048 + 64, shard=None):
    import torch
    from oracle import pool as OP
    from paper_2602_04430_b300 import build, stretto, synth
    build.build()
    cfg = synth.MODELS[model_key]
    table = synth.make_table(synth.TABLES[table_key], cfg.vocab, seed=table_seed, n_tuples=n_tuples)
    off, tok = table["offsets"], table["tokens"]
    T = len(table["lengths"])
    rng = np.random.Generator(np.random.PCG64(sample_seed))
    sample = np.sort(rng.choice(T if shard is None else shard, n_sample, replace=False))
    base = synth.make_prompt(32, cfg.vocab, seed=op_seed, label_ids=(1, 0), r=r)
    w = synth.make_weights(cfg, seed=weight_seed)
    docs = {int(t): tok[off[t]:off[t + 1]] for t in sample}
    # the oracle pool first (spawned workers), then the GPU
    pool = OP.OraclePool(cfg, w)
    model = stretto.Model(cfg, w, max_pos=max_pos)
    del w
    n_gpu = T if shard is None else shard
    kv = model.kv_alloc(off[:n_gpu + 1])
    kv.build(torch.from_numpy(np.ascontiguousarray(tok[:off[n_gpu]])).cuda())
    ids = torch.arange(n_gpu, dtype=torch.int32, device="cuda")
    R = int(off[n_gpu])
    gpu = {}
    for name, code in (("bf16", stretto.ST_BF16), ("e4m3", stretto.ST_E4M3)):
        kv.retain(r, code)
        lg, _ = model.operator(base).eval(kv, ids)
        torch.cuda.synchronize()
        model.status()
        kv.status()
        gpu[name] = lg.cpu().numpy()[sample]
        if name == "bf16":
            rank = kv.read(stretto.ST_VIEW_RANK, torch.int32, (cfg.layers, cfg.hkv, R)).cpu().numpy()
            scores = kv.read(stretto.ST_VIEW_SCORES, torch.float32, (cfg.layers, cfg.hkv, R)).cpu().numpy()
    # the oracle: its own ranking with exact K/V and with exact-value E4M3 codes,
    # and, for the logit bound, the GPU's retained sets with exact K/V (the
    # ranking is an integer decision the kernel takes in float32)
    from oracle import operator as O
    ops = [{"prompt": base.prompt, "label_ids": base.label_ids, "r": r},
           {"prompt": base.prompt, "label_ids": base.label_ids, "r": r, "kv_fp8": True},
           {"prompt": base.prompt, "label_ids": base.label_ids, "r": r},
           {"prompt": base.prompt, "label_ids": base.label_ids, "r": r, "kv_fp8": True}]
    idx = {}
    for t in sample:
        a, b = int(off[t]), int(off[t + 1])
        n = O.n_keep(b - a, r)
        gsets = [[rank[l, g, a:a + n].copy() for g in range(cfg.hkv)] for l in range(cfg.layers)]
        idx[int(t)] = [None, None, gsets, gsets]
    res = pool.run(docs, ops, want_scores=True, idx=idx)
    pool.close()
    z_or = np.array([res[int(t)]["logits"][0] for t in sample])
    z_or8 = np.array([res[int(t)]["logits"][1] for t in sample])
    z_orset = np.array([res[int(t)]["logits"][2] for t in sample])
    z_orset8 = np.array([res[int(t)]["logits"][3] for t in sample])
    theta = float(np.median(z_or[:, 0] - z_or[:, 1]))
    # the GPU's decisions at theta come from its label head (float32)
    from paper_2602_04430_b300 import synth as S
    op_t = S.Operator(prompt=base.prompt, label_ids=base.label_ids, r=r, theta_pos=theta, theta_neg=theta)
    labels = {}
    for name, code in (("bf16", stretto.ST_BF16), ("e4m3", stretto.ST_E4M3)):
        kv.retain(r, code)
        _, lb = model.operator(op_t).eval(kv, ids)
        torch.cuda.synchronize()
        model.status()
        labels[name] = lb.cpu().numpy()[sample]
    out = {"theta": theta, "n": len(sample)}
    d_or, d_or8 = _decide(z_or, theta), _decide(z_or8, theta)
    out["bf16_agree"] = float((labels["bf16"] == d_or).mean())
    out["e4m3_agree"] = float((labels["e4m3"] == d_or8).mean())
    out["e4m3_agree_vs_exact"] = float((labels["e4m3"] == d_or).mean())
    out["oracle_e4m3_vs_exact"] = float((d_or8 == d_or).mean())
    out["bf16_agree_theta0"] = float((_decide(gpu["bf16"], 0.0) == _decide(z_or, 0.0)).mean())
    out["e4m3_agree_theta0"] = float((_decide(gpu["e4m3"], 0.0) == _decide(z_or8, 0.0)).mean())
    out["bf16_err_gpu_sets"] = normwise_rel(gpu["bf16"], z_orset)
    out["bf16_err_gpu_sets_tuple_max"] = max(normwise_rel(a, b) for a, b in zip(gpu["bf16"], z_orset))
    out["e4m3_err_gpu_sets"] = normwise_rel(gpu["e4m3"], z_orset8)
    out["bf16_err"] = normwise_rel(gpu["bf16"], z_or)
    out["e4m3_err"] = normwise_rel(gpu["e4m3"], z_or8)
    out["bf16_err_tuple_max"] = max(normwise_rel(a, b) for a, b in zip(gpu["bf16"], z_or))
    out["e4m3_err_tuple_max"] = max(normwise_rel(a, b) for a, b in zip(gpu["e4m3"], z_or8))
    ov, ex = [], 0
    for t in sample:
        a, b = int(off[t]), int(off[t + 1])
        n = O.n_keep(b - a, r)
        rows = [[rank[l, g, a:b] for g in range(cfg.hkv)] for l in range(cfg.layers)]
        sg = [[scores[l, g, a:b] for g in range(cfg.hkv)] for l in range(cfg.layers)]
        o, e = _retained_overlap(rows, sg, res[int(t)]["scores"], n)
        ov.append(o)
        ex += e
    out["retained_overlap_mean"] = float(np.mean(ov))
    out["retained_overlap_min"] = float(np.min(ov))
    out["retained_exchanges"] = int(ex)
    kv.close()
    model.close()
    return out


def test_config2_agreement_and_error_vs_unmodified_oracle():
    """The benchmark's 8-layer BF16 workload (4096 tuples, r = 0.5): 256 seeded tuples."""
    from paper_2602_04430_b300 import multigpu
    out = _run("c2_bf16", "c2", multigpu.rank_seed(1000, 0), 4242, 77, 0.5, N_C2, 9)
    print("config 2 vs the unmodified oracle:", out)
    assert out["bf16_err_gpu_sets"] <= 2e-2, out
    assert out["e4m3_err_gpu_sets"] <= 5e-2, out
    assert out["e4m3_err"] <= 5e-2, out
    assert out["bf16_agree"] >= 0.995, out
    assert out["e4m3_agree"] >= 0.99, out
    assert out["retained_overlap_mean"] >= 0.99, out


def test_config3_agreement_and_error_vs_unmodified_oracle():
    """The 16-layer precision workload (lognormal median 1024, clipped
    128..4096; one shard of 2048 tuples, r = 0.25): 32 seeded tuples (the
    float64 oracle takes ~40 s per tuple and core).  With 32 tuples the
    agreement bars (99.5 % BF16, 99 % E4M3) allow no disagreement.  Over the
    GPU's retained sets the BF16 and E4M3 logits meet their bounds; against the
    oracle's own ranking the error (exchanged near-tie slots through 16 layers)
    is reported."""
    out = _run("c3_bf16", "c3", 3300, 3301, 3302, 0.25, N_C3, 11, n_tuples=2048, max_pos=4096 + 64,
               shard=2048)
    print("config 3 vs the unmodified oracle:", out)
    assert out["bf16_err_gpu_sets"] <= 2e-2, out
    assert out["e4m3_err_gpu_sets"] <= 5e-2, out
    assert out["bf16_agree"] >= 0.995, out
    assert out["e4m3_agree"] >= 0.99, out
    assert out["retained_overlap_mean"] >= 0.99, out
