"""Autotuned evaluation schedules kept on disk, keyed by shape bucket.

``st_autotune_eval`` times candidate schedules on the real batch (one warm-up
and three timed runs each), which costs seconds; a query executor that sees
batches of the same shape again reuses the choice.  The key is the shape
bucket of a batched evaluation: the model's dimensions, the retained cache's
element type and ratio, every operator's prompt length, retention ratio, kind
and label count, and the pair count and longest document rounded up to powers
of two.  The file is plain JSON: {key: {eval_rows, attn_nb, longest_first,
split_keys, ms}}.  Host logic only; the schedule itself is applied with
``st_set_schedule``.
"""
from __future__ import annotations

import json
import math
import os
from typing import Dict, Optional, Sequence, Tuple

from . import stretto

FIELDS = ("eval_rows", "attn_nb", "longest_first", "split_keys")


def _pow2(n: int) -> int:
    return 1 if n <= 1 else 1 << math.ceil(math.log2(n))


def shape_key(model, kv, ops: Sequence, tuple_counts: Sequence[int]) -> str:
    """The shape bucket of evaluating ``ops`` (stretto.Operator) over
    ``tuple_counts[k]`` tuples each, on ``kv`` (stretto.KVCache)."""
    c = model.cfg
    lengths = kv.offsets[1:] - kv.offsets[:-1]
    longest = int(lengths.max()) if len(lengths) else 0
    parts = [f"model={c.layers}x{c.d}/{c.hq}q{c.hkv}kv{c.hd}/ffn{c.ffn}/v{c.vocab}/{c.dtype}",
             f"kv={getattr(kv, 'kv_dtype', None)}@{getattr(kv, 'r', None)}"]
    for o in ops:
        op = o.op
        parts.append(f"op={op.kind}/P{len(op.prompt)}/r{op.r}/L{len(op.label_ids)}")
    parts.append(f"pairs<={_pow2(int(sum(tuple_counts)))}")
    parts.append(f"len<={_pow2(longest)}")
    return "|".join(parts)


class ScheduleCache:
    """A JSON file of schedules by shape key (created on first save)."""

    def __init__(self, path: str):
        self.path = path
        self.entries: Dict[str, dict] = {}
        if os.path.exists(path):
            with open(path) as f:
                self.entries = json.load(f)

    def get(self, key: str) -> Optional[dict]:
        return self.entries.get(key)

    def put(self, key: str, choice: dict):
        self.entries[key] = {k: choice[k] for k in FIELDS + ("ms",) if k in choice}

    def save(self):
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.entries, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def autotune_cached(model, kv, ops, tuple_ids, cache: ScheduleCache, **kw) -> Tuple[dict, bool]:
    """Set the schedule for this batch: the cached choice for its shape bucket
    if there is one, else the autotuner's (``stretto.autotune`` on the batch,
    which also writes the outputs), stored in the cache.  Returns (choice,
    hit)."""
    key = shape_key(model, kv, ops, [int(t.numel()) for t in tuple_ids])
    hit = cache.get(key)
    if hit is not None:
        stretto.set_schedule(model, **{k: hit[k] for k in FIELDS})
        return hit, True
    best, _ = stretto.autotune(model, kv, ops, tuple_ids, **kw)
    cache.put(key, best)
    cache.save()
    return best, False
