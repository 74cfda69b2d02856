"""The autotuner's schedule cache (host logic, no GPU): shape keys bucket the
pair count and the longest document by powers of two and separate models,
cache element types and operators; the first batch of a bucket is tuned and
stored, a later batch of the same bucket (also from a fresh process's view of
the file) takes the stored schedule without tuning."""
import types

import numpy as np
import torch

from paper_2602_04430_b300 import schedule_cache as SC
from paper_2602_04430_b300 import stretto, synth


def _fakes(lengths, kv_dtype=stretto.ST_BF16, r=0.5, P=32, kind="filter"):
    cfg = synth.MODELS["c2_bf16"]
    model = types.SimpleNamespace(cfg=cfg)
    off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    kv = types.SimpleNamespace(offsets=off, kv_dtype=kv_dtype, r=r)
    op = types.SimpleNamespace(op=synth.make_prompt(P, cfg.vocab, seed=1, r=r, kind=kind,
                                                    label_ids=(1, 0) if kind == "filter" else (2, 3, 4)))
    return model, kv, [op]


def test_shape_keys_bucket_and_separate():
    m, kv, ops = _fakes([100, 900, 1000])
    k1 = SC.shape_key(m, kv, ops, [1000])
    assert SC.shape_key(m, kv, ops, [600]) == k1            # same power-of-two bucket (1024)
    assert SC.shape_key(m, kv, ops, [1025]) != k1
    m2, kv2, ops2 = _fakes([100, 900, 1030])                 # longest 1030 -> bucket 2048
    assert SC.shape_key(m2, kv2, ops2, [1000]) != k1
    _, kv3, _ = _fakes([100, 900, 1000], kv_dtype=stretto.ST_E4M3)
    assert SC.shape_key(m, kv3, ops, [1000]) != k1
    _, _, ops4 = _fakes([100, 900, 1000], P=48)
    assert SC.shape_key(m, kv, ops4, [1000]) != k1
    _, _, ops5 = _fakes([100, 900, 1000], kind="classify")
    assert SC.shape_key(m, kv, ops5, [1000]) != k1


def test_first_batch_tunes_and_later_batches_reuse(tmp_path, monkeypatch):
    calls = {"tune": 0, "set": []}
    best = {"eval_rows": 131072, "attn_nb": 1, "longest_first": 1, "split_keys": 0, "ms": 12.5}

    def fake_autotune(model, kv, ops, tuple_ids, **kw):
        calls["tune"] += 1
        return dict(best), [dict(best)]

    def fake_set(model, **kw):
        calls["set"].append(kw)

    monkeypatch.setattr(stretto, "autotune", fake_autotune)
    monkeypatch.setattr(stretto, "set_schedule", fake_set)
    m, kv, ops = _fakes([100, 900, 1000])
    path = str(tmp_path / "schedules.json")
    cache = SC.ScheduleCache(path)
    choice, hit = SC.autotune_cached(m, kv, ops, [torch.zeros(1000, dtype=torch.int32)], cache)
    assert not hit and calls["tune"] == 1 and choice["eval_rows"] == 131072
    # a fresh view of the file: the same bucket is a hit, applied without tuning
    cache2 = SC.ScheduleCache(path)
    choice2, hit2 = SC.autotune_cached(m, kv, ops, [torch.zeros(700, dtype=torch.int32)], cache2)
    assert hit2 and calls["tune"] == 1
    assert calls["set"] == [{"eval_rows": 131072, "attn_nb": 1, "longest_first": 1, "split_keys": 0}]
    # another bucket tunes again
    SC.autotune_cached(m, kv, ops, [torch.zeros(3000, dtype=torch.int32)], cache2)
    assert calls["tune"] == 2 and len(SC.ScheduleCache(path).entries) == 2
