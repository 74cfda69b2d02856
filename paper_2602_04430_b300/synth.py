"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module draws random numbers and lays them out; it performs none of the
method's arithmetic (no normalisation, attention, scoring, retention or label
head).  Every array it returns is an *input*: model weights drawn i.i.d. from
N(0, 0.02^2), tables of documents (token ids with a length mix), operator
prompts and label ids.

Model weights follow a Llama-style decoder (the operators of Sec. 5 run an LLM
over each tuple's document); the paper's checkpoints are not available, so the
weights are random-init from a seed.  All matrices are stored ``[out][in]``
(row n holds the weights of output feature n), in this fixed draw order:
``embed [V][d]``, then per layer ``wq [Hq*hd][d]``, ``wk [Hkv*hd][d]``,
``wv [Hkv*hd][d]``, ``wo [d][Hq*hd]``, ``wg [F][d]``, ``wu [F][d]``,
``wd [d][F]``, then ``w_lm [V][d]``.  RMSNorm gains are fixed to 1 (no
parameters), there are no biases and the LM head is untied.

For a BF16 model the float32 draws are rounded once to bfloat16 (round to
nearest even); both the CUDA path and the oracle then see exactly those values.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

__all__ = [
    "ModelConfig", "TableConfig", "Operator", "MODELS", "TABLES",
    "make_weights", "make_table", "make_prompt", "to_bf16_f32",
    "zipf_ids", "lognormal_lengths",
]


@dataclasses.dataclass(frozen=True)
class ModelConfig:
    """Decoder shape.  ``dtype`` is the weight / activation type of the CUDA path."""
    layers: int
    d: int
    hq: int
    hkv: int
    hd: int
    ffn: int
    vocab: int
    rope_theta: float = 10000.0
    eps: float = 1e-5
    dtype: str = "bf16"          # "f32" or "bf16"
    name: str = ""

    @property
    def group(self) -> int:
        return self.hq // self.hkv

    def n_params(self) -> int:
        per_layer = (self.hq * self.hd * self.d + 2 * self.hkv * self.hd * self.d
                     + self.d * self.hq * self.hd + 3 * self.d * self.ffn)
        return self.layers * per_layer + 2 * self.vocab * self.d


@dataclasses.dataclass(frozen=True)
class TableConfig:
    """A synthetic table of tuples, one document (token sequence) per tuple."""
    n_tuples: int
    length: str                  # "fixed" | "lognormal" | "zipf"
    len_a: float                 # fixed length, lognormal median, or zipf exponent
    len_sigma: float = 0.0       # lognormal sigma
    len_min: int = 1
    len_max: int = 1
    ids: str = "uniform"         # "uniform" | "zipf"
    ids_s: float = 1.1


@dataclasses.dataclass(frozen=True)
class Operator:
    """A KV-cache semantic operator: prompt ids appended after the document,
    label token ids whose logits are read at the last prompt position, the
    retention fraction r of the KV profile, and the decision thresholds."""
    prompt: tuple
    label_ids: tuple
    r: float = 1.0
    theta_pos: float = 0.0
    theta_neg: float = 0.0
    kind: str = "filter"         # "filter" (binary accept/reject/unsure) | "classify"
    bias: Optional[tuple] = None  # per-label additive bias (classify)


# The five workloads: model shapes and tables of the benchmark configurations.
MODELS: Dict[str, ModelConfig] = {
    "tiny_f32": ModelConfig(layers=2, d=128, hq=4, hkv=4, hd=32, ffn=512, vocab=1024,
                            dtype="f32", name="tiny_f32"),
    "c2_bf16": ModelConfig(layers=8, d=1024, hq=16, hkv=4, hd=64, ffn=2816, vocab=32000,
                           dtype="bf16", name="c2_bf16"),
    "c3_bf16": ModelConfig(layers=16, d=2048, hq=32, hkv=8, hd=64, ffn=5632, vocab=32000,
                           dtype="bf16", name="c3_bf16"),
}

TABLES: Dict[str, TableConfig] = {
    "tiny": TableConfig(n_tuples=64, length="fixed", len_a=256, len_min=256, len_max=256,
                        ids="uniform"),
    "c2": TableConfig(n_tuples=4096, length="lognormal", len_a=512, len_sigma=0.6,
                      len_min=64, len_max=2048, ids="zipf", ids_s=1.1),
    "c3": TableConfig(n_tuples=16384, length="lognormal", len_a=1024, len_sigma=0.6,
                      len_min=128, len_max=4096, ids="zipf", ids_s=1.1),
    "c4": TableConfig(n_tuples=32768, length="zipf", len_a=1.1, len_min=32, len_max=8192,
                      ids="zipf", ids_s=1.1),
}


def to_bf16_f32(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    rounding = 0x7FFF + ((u >> 16) & 1)
    u = ((u + rounding) >> 16) << 16
    out = u.astype(np.uint32).view(np.float32)
    # NaN never occurs in N(0, 0.02) draws; keep them NaN all the same.
    nan = np.isnan(a)
    if nan.any():
        out = out.copy()
        out[nan] = np.nan
    return out


def make_weights(cfg: ModelConfig, seed: int = 1234, std: float = 0.02) -> Dict[str, object]:
    """Draw all weights of ``cfg`` from one PCG64 stream, in the documented order.

    Returns ``{"embed": [V][d], "layers": [dict(wq, wk, wv, wo, wg, wu, wd)], "w_lm": [V][d]}``
    as float32 arrays (already rounded to bf16 values for a bf16 model).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    rnd = (lambda shape: to_bf16_f32(rng.standard_normal(shape, dtype=np.float32) * np.float32(std))
           if cfg.dtype == "bf16" else
           (rng.standard_normal(shape, dtype=np.float32) * np.float32(std)))
    d, hq, hkv, hd, f = cfg.d, cfg.hq, cfg.hkv, cfg.hd, cfg.ffn
    out = {"embed": rnd((cfg.vocab, d)), "layers": []}
    for _ in range(cfg.layers):
        out["layers"].append({
            "wq": rnd((hq * hd, d)), "wk": rnd((hkv * hd, d)), "wv": rnd((hkv * hd, d)),
            "wo": rnd((d, hq * hd)), "wg": rnd((f, d)), "wu": rnd((f, d)), "wd": rnd((d, f)),
        })
    out["w_lm"] = rnd((cfg.vocab, d))
    return out


def make_weights_device(cfg: ModelConfig, seed: int = 1234, std: float = 0.02) -> Dict[str, object]:
    """The same layout and distribution as ``make_weights`` (N(0, std^2), bf16 values for
    a bf16 model) drawn on the GPU with torch's seeded CUDA generator: a different
    stream of numbers, for throughput runs of large models where host generation
    would dominate the set-up time."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    dt = torch.bfloat16 if cfg.dtype == "bf16" else torch.float32
    rnd = lambda shape: (torch.randn(shape, generator=g, device="cuda", dtype=torch.float32) * std).to(dt)
    d, hq, hkv, hd, f = cfg.d, cfg.hq, cfg.hkv, cfg.hd, cfg.ffn
    out = {"embed": rnd((cfg.vocab, d)), "layers": []}
    for _ in range(cfg.layers):
        out["layers"].append({
            "wq": rnd((hq * hd, d)), "wk": rnd((hkv * hd, d)), "wv": rnd((hkv * hd, d)),
            "wo": rnd((d, hq * hd)), "wg": rnd((f, d)), "wu": rnd((f, d)), "wd": rnd((d, f)),
        })
    out["w_lm"] = rnd((cfg.vocab, d))
    return out


def make_proxy_weights(d_in: int, h1: int = 512, h2: int = 128, seed: int = 777) -> Dict[str, np.ndarray]:
    """Initial parameters of the proxy MLP: W ~ N(0, 1/fan_in), b = 0 (float32)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {}
    for name, (o, i) in (("1", (h1, d_in)), ("2", (h2, h1)), ("3", (2, h2))):
        out["w" + name] = (rng.standard_normal((o, i), dtype=np.float32) / np.float32(np.sqrt(i)))
        out["b" + name] = np.zeros(o, dtype=np.float32)
    return out


def minibatches(n: int, batch: int, epochs: int, seed: int = 778):
    """Shuffled mini-batch index arrays (the proxy's training order is an input)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(epochs):
        perm = rng.permutation(n).astype(np.int32)
        for i in range(0, n - batch + 1, batch):
            out.append(perm[i:i + batch])
    return out


def lognormal_lengths(rng: np.random.Generator, n: int, median: float, sigma: float,
                      lo: int, hi: int) -> np.ndarray:
    x = rng.lognormal(mean=math.log(median), sigma=sigma, size=n)
    return np.clip(np.rint(x), lo, hi).astype(np.int64)


def _bounded_zipf(rng: np.random.Generator, n: int, s: float, lo: int, hi: int) -> np.ndarray:
    """Draw integers k in [lo, hi] with P(k) proportional to k^-s (inverse CDF)."""
    k = np.arange(lo, hi + 1, dtype=np.float64)
    p = k ** (-s)
    cdf = np.cumsum(p)
    cdf /= cdf[-1]
    u = rng.random(n)
    return (lo + np.searchsorted(cdf, u, side="right")).clip(lo, hi).astype(np.int64)


def zipf_ids(rng: np.random.Generator, n: int, s: float, vocab: int) -> np.ndarray:
    """Token ids with Zipf(s) frequencies over ranks 1..V; id = rank - 1."""
    return (_bounded_zipf(rng, n, s, 1, vocab) - 1).astype(np.int32)


def make_table(tcfg: TableConfig, vocab: int, seed: int = 99,
               n_tuples: Optional[int] = None) -> Dict[str, np.ndarray]:
    """Return ``{"tokens": int32[sum L], "offsets": int64[T+1], "lengths": int64[T]}``.

    ``n_tuples`` overrides the table size (the first tuples of the same stream are
    identical whatever the size, so a prefix of a big table is a small table).
    """
    T = tcfg.n_tuples if n_tuples is None else int(n_tuples)
    rng_len = np.random.Generator(np.random.PCG64(seed))
    rng_ids = np.random.Generator(np.random.PCG64(seed + 1))
    if tcfg.length == "fixed":
        lengths = np.full(T, int(tcfg.len_a), dtype=np.int64)
    elif tcfg.length == "lognormal":
        # draw for the full table, then cut, so prefixes agree across sizes
        full = lognormal_lengths(rng_len, max(T, tcfg.n_tuples), tcfg.len_a, tcfg.len_sigma,
                                 tcfg.len_min, tcfg.len_max)
        lengths = full[:T]
    elif tcfg.length == "zipf":
        full = _bounded_zipf(rng_len, max(T, tcfg.n_tuples), tcfg.len_a, tcfg.len_min,
                             tcfg.len_max)
        lengths = full[:T]
    else:
        raise ValueError(tcfg.length)
    offsets = np.zeros(T + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    total = int(offsets[-1])
    if tcfg.ids == "uniform":
        tokens = rng_ids.integers(0, vocab, size=total, dtype=np.int64).astype(np.int32)
    else:
        tokens = zipf_ids(rng_ids, total, tcfg.ids_s, vocab)
    return {"tokens": tokens, "offsets": offsets, "lengths": lengths}


def make_table_from_lengths(lengths, vocab: int, seed: int = 7, ids: str = "uniform",
                            ids_s: float = 1.1) -> Dict[str, np.ndarray]:
    """A table with explicit document lengths (edge cases, ragged tails)."""
    lengths = np.asarray(lengths, dtype=np.int64)
    offsets = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    rng = np.random.Generator(np.random.PCG64(seed))
    total = int(offsets[-1])
    if ids == "uniform":
        tokens = rng.integers(0, vocab, size=total, dtype=np.int64).astype(np.int32)
    else:
        tokens = zipf_ids(rng, total, ids_s, vocab)
    return {"tokens": tokens, "offsets": offsets, "lengths": lengths}


def make_prompt(P: int, vocab: int, seed: int = 5, label_ids=(1, 0), r: float = 1.0,
                theta_pos: float = 0.0, theta_neg: float = 0.0, kind: str = "filter",
                bias=None) -> Operator:
    """An operator with a uniformly drawn ``P``-token prompt."""
    rng = np.random.Generator(np.random.PCG64(seed))
    prompt = tuple(int(x) for x in rng.integers(0, vocab, size=P))
    return Operator(prompt=prompt, label_ids=tuple(int(x) for x in label_ids), r=float(r),
                    theta_pos=float(theta_pos), theta_neg=float(theta_neg), kind=kind,
                    bias=None if bias is None else tuple(float(b) for b in bias))


def sample_tuples(T: int, k: int, seed: int = 3) -> List[int]:
    """k distinct tuple indices of a T-tuple table, always including the first and last."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = min(k, T)
    pick = set([0, T - 1])
    while len(pick) < k:
        pick.add(int(rng.integers(0, T)))
    return sorted(pick)
