"""Thin ctypes binding of libstretto (include/stretto.h).

Argument marshalling only: torch tensors provide device memory and the current
CUDA stream; every step of the operator runs in the library's CUDA kernels.
The library must have been built in-tree (``paper_2602_04430_b300.build``);
there is no fallback of any kind when it is missing.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional, Sequence

import numpy as np

from . import synth

HERE = os.path.dirname(os.path.abspath(__file__))
# STRETTO_CHECK=1 selects the checked build (index and offset checks, -DST_CHECK)
LIB_PATH = os.path.join(HERE, "libstretto_check.so" if os.environ.get("STRETTO_CHECK") == "1"
                        else "libstretto.so")

ST_OK, ST_EINVAL, ST_ENOMEM, ST_ECUDA, ST_ETIMEOUT, ST_ENAN, ST_EUNSUPPORTED, ST_ERANGE, ST_ECHECK = range(9)
ST_SCORE_EA_LITE, ST_SCORE_EA_FULL = 0, 1
ST_F32, ST_BF16, ST_E4M3 = 0, 1, 2
ST_WS_BUILD, ST_WS_EVAL, ST_WS_ANY = 0, 1, 2
ST_OP_FILTER, ST_OP_CLASSIFY = 0, 1
ST_REJECT, ST_ACCEPT, ST_UNSURE = 0, 1, 2
(ST_VIEW_K, ST_VIEW_V, ST_VIEW_SCORES, ST_VIEW_POOLED, ST_VIEW_RANK, ST_VIEW_KR, ST_VIEW_VR,
 ST_VIEW_SCALES, ST_VIEW_OFFP, ST_VIEW_NKEEP) = range(10)
PROF_FAMILIES = ("gemm", "attention", "retain", "other")
ST_PROXY_PARAMS, ST_PROXY_GRADS, ST_PROXY_ADAM_M, ST_PROXY_ADAM_V = range(4)
PROXY_ORDER = ("w1", "b1", "w2", "b2", "w3", "b3")


class StrettoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libstretto error {code}: {msg}")
        self.code = code


class ModelCfg(ctypes.Structure):
    _fields_ = [("layers", ctypes.c_int32), ("d", ctypes.c_int32), ("hq", ctypes.c_int32),
                ("hkv", ctypes.c_int32), ("hd", ctypes.c_int32), ("ffn", ctypes.c_int32),
                ("vocab", ctypes.c_int32), ("dtype", ctypes.c_int32), ("max_pos", ctypes.c_int32),
                ("rope_theta", ctypes.c_float), ("eps", ctypes.c_float)]


class OpDesc(ctypes.Structure):
    _fields_ = [("prompt", ctypes.POINTER(ctypes.c_int32)), ("P", ctypes.c_int32),
                ("label_ids", ctypes.POINTER(ctypes.c_int32)), ("n_labels", ctypes.c_int32),
                ("kind", ctypes.c_int32), ("r", ctypes.c_double), ("theta_pos", ctypes.c_float),
                ("theta_neg", ctypes.c_float), ("bias", ctypes.POINTER(ctypes.c_float))]


_LIB = None
VP = ctypes.c_void_p


class TuneChoice(ctypes.Structure):
    """st_tune_choice: an operator-evaluation schedule and its measured time."""
    _fields_ = [("eval_rows", ctypes.c_int64), ("attn_nb", ctypes.c_int32),
                ("longest_first", ctypes.c_int32), ("split_keys", ctypes.c_int32), ("ms", ctypes.c_float)]

    def as_dict(self):
        return {"eval_rows": int(self.eval_rows), "attn_nb": int(self.attn_nb),
                "longest_first": int(self.longest_first), "split_keys": int(self.split_keys),
                "ms": float(self.ms)}


class StageDesc(ctypes.Structure):
    """st_stage: one cascade stage (context, cache, operator handles)."""
    _fields_ = [("ctx", ctypes.c_void_p), ("kv", ctypes.c_void_p), ("op", ctypes.c_void_p)]


def lib() -> ctypes.CDLL:
    """Load libstretto.so (raises ImportError if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2602_04430_b300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    i32, i64, sz, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_double
    sigs = {
        "st_create": (i32, [ctypes.POINTER(ModelCfg), ctypes.POINTER(VP), VP, ctypes.POINTER(VP)]),
        "st_destroy": (None, [VP]),
        "st_last_error": (ctypes.c_char_p, [VP]),
        "st_version": (ctypes.c_char_p, []),
        "st_reserve": (i32, [VP, i64, i64]),
        "st_workspace_size": (sz, [VP, i32, i64]),
        "st_set_workspace": (i32, [VP, i32, VP, sz]),
        "st_workspace_held": (sz, [VP, i32]),
        "st_kv_alloc": (i32, [VP, ctypes.POINTER(i64), i32, ctypes.POINTER(VP)]),
        "st_kv_free": (None, [VP]),
        "st_kv_profile_alloc": (i32, [VP, VP, dbl, ctypes.POINTER(VP)]),
        "st_kv_build": (i32, [VP, VP, VP, VP]),
        "st_kv_retain": (i32, [VP, VP, dbl, i32, VP]),
        "st_kv_indices": (i32, [VP, VP, dbl, VP, VP, VP]),
        "st_kv_status": (i32, [VP, VP, VP]),
        "st_status": (i32, [VP, VP]),
        "st_kv_view": (i32, [VP, i32, ctypes.POINTER(VP), ctypes.POINTER(sz)]),
        "st_kv_read": (i32, [VP, i32, VP, sz, VP]),
        "st_op_create": (i32, [VP, ctypes.POINTER(OpDesc), ctypes.POINTER(VP)]),
        "st_op_free": (None, [VP]),
        "st_op_eval": (i32, [VP, VP, VP, VP, i32, VP, VP, VP]),
        "st_op_eval_noalloc": (i32, [VP, VP, VP, VP, i32, VP, VP, VP]),
        "st_op_eval_multi": (i32, [VP, VP, i32, ctypes.POINTER(VP), ctypes.POINTER(VP),
                                   ctypes.POINTER(i32), ctypes.POINTER(VP), ctypes.POINTER(VP), VP]),
        "st_graph_create": (i32, [VP, VP, i32, ctypes.POINTER(VP), ctypes.POINTER(VP),
                                  ctypes.POINTER(i32), ctypes.POINTER(VP), ctypes.POINTER(VP),
                                  ctypes.POINTER(VP)]),
        "st_graph_launch": (i32, [VP, VP]),
        "st_graph_launches": (i64, [VP]),
        "st_graph_free": (None, [VP]),
        "st_autotune_eval": (i32, [VP, VP, i32, ctypes.POINTER(VP), ctypes.POINTER(VP),
                                   ctypes.POINTER(i32), ctypes.POINTER(VP), ctypes.POINTER(VP), VP,
                                   ctypes.POINTER(TuneChoice), ctypes.POINTER(TuneChoice), i32,
                                   ctypes.POINTER(i32)]),
        "st_set_schedule": (i32, [VP, ctypes.POINTER(TuneChoice)]),
        "st_selftest_wait": (i32, [VP, i64, VP]),
        "st_map_eval": (i32, [VP, VP, VP, VP, i32, i32, VP, VP, VP]),
        "st_set_scoring": (i32, [VP, i32, i32]),
        "st_set_gemm_pairs": (i32, [i32]),
        "st_kv_profile_bytes": (i32, [VP, ctypes.POINTER(ctypes.c_size_t)]),
        "st_kv_read_at": (i32, [VP, i32, ctypes.c_size_t, VP, ctypes.c_size_t, VP]),
        "st_kv_export": (i32, [VP, VP, VP, ctypes.c_size_t, VP]),
        "st_kv_import": (i32, [VP, VP, VP, ctypes.c_size_t, VP]),
        "st_kv_score_query": (i32, [VP, VP, VP, VP]),
        "st_cascade_run": (i32, [i32, ctypes.POINTER(StageDesc), VP, i32, VP, VP, ctypes.POINTER(i32),
                                 ctypes.POINTER(ctypes.c_float), VP]),
        "st_run_host": (i32, [VP, VP, VP, i32, VP, VP, VP, VP]),
        "st_proxy_cascade": (i32, [VP, VP, VP, ctypes.c_float, i32, ctypes.POINTER(StageDesc), VP, i32, VP, VP,
                                   ctypes.POINTER(i32), VP]),
        "st_gemm": (i32, [VP, VP, VP, i32, i32, i32, VP, VP]),
        "st_proxy_create": (i32, [VP, i32, i32, i32, ctypes.POINTER(VP), ctypes.POINTER(VP)]),
        "st_proxy_free": (None, [VP]),
        "st_proxy_train_step": (i32, [VP, VP, VP, VP, VP, i32, ctypes.c_float, VP, VP]),
        "st_proxy_eval": (i32, [VP, VP, VP, VP, i32, VP, VP, VP]),
        "st_cascade_compact": (i32, [VP, VP, VP, i32, ctypes.c_float, VP, VP, VP]),
        "st_cascade_merge": (i32, [VP, VP, i32, VP, VP, VP, VP, VP]),
        "st_proxy_steps": (i64, [VP]),
        "st_proxy_set_precision": (i32, [VP, i32]),
        "st_proxy_restore": (i32, [VP, VP, VP, VP, sz, i64, VP]),
        "st_proxy_read": (i32, [VP, i32, VP, sz, VP]),
        "st_prof_enable": (i32, [VP, i32]),
        "st_prof_read": (i32, [VP, ctypes.POINTER(dbl)]),
        "st_prof_reset": (i32, [VP]),
        "st_launch_count": (i64, [VP]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return VP(s.cuda_stream)


def _ptr(t) -> VP:
    return VP(t.data_ptr())


class Model:
    """A decoder with its weights resident on the device (an ``st_ctx``)."""

    def __init__(self, cfg: synth.ModelConfig, weights: Dict[str, object], max_pos: int = 16640,
                 device: str = "cuda"):
        import torch
        self.cfg = cfg
        self.L = lib()
        dt = torch.bfloat16 if cfg.dtype == "bf16" else torch.float32
        self.torch_dtype = dt
        arrays = [weights["embed"]]
        for lw in weights["layers"]:
            arrays += [lw[k] for k in ("wq", "wk", "wv", "wo", "wg", "wu", "wd")]
        arrays.append(weights["w_lm"])
        dev = [(a if isinstance(a, torch.Tensor) else
                torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))).to(device).to(dt).contiguous()
               for a in arrays]
        ptrs = (VP * len(dev))(*[t.data_ptr() for t in dev])
        c = ModelCfg(cfg.layers, cfg.d, cfg.hq, cfg.hkv, cfg.hd, cfg.ffn, cfg.vocab,
                     ST_BF16 if cfg.dtype == "bf16" else ST_F32, max_pos, cfg.rope_theta, cfg.eps)
        self._cfg = c
        h = VP()
        rc = self.L.st_create(ctypes.byref(c), ptrs, _stream(), ctypes.byref(h))
        if rc != ST_OK:
            raise StrettoError(rc, self.L.st_last_error(None).decode())
        self.h = h
        del dev

    def check(self, rc: int):
        if rc != ST_OK:
            raise StrettoError(rc, self.L.st_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.st_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, build_rows: int = 0, eval_rows: int = 0):
        self.check(self.L.st_reserve(self.h, int(build_rows), int(eval_rows)))

    def workspace_size(self, which: int, rows: int) -> int:
        """Bytes of device workspace one chunk of ``rows`` rows needs (ST_WS_BUILD / ST_WS_EVAL)."""
        return int(self.L.st_workspace_size(self.h, int(which), int(rows)))

    def workspace_held(self, which: int = ST_WS_ANY) -> int:
        """Device bytes of workspace the library currently owns for this context."""
        return int(self.L.st_workspace_held(self.h, int(which)))

    def set_workspace(self, which: int, buf=None):
        """Carve that workspace out of the caller's device tensor ``buf`` (kept alive
        here until replaced), or go back to library-owned workspace with None."""
        if not hasattr(self, "_ws_keep"):
            self._ws_keep = {}
        if buf is None:
            self.check(self.L.st_set_workspace(self.h, int(which), None, 0))
            self._ws_keep.pop(int(which), None)
            return
        nbytes = buf.numel() * buf.element_size()
        self.check(self.L.st_set_workspace(self.h, int(which), _ptr(buf), nbytes))
        self._ws_keep[int(which)] = buf

    def selftest_wait(self, limit_cycles: int = 1000000, stream=None):
        """Run the bounded-wait failure self-test (its time-out shows in status())."""
        self.check(self.L.st_selftest_wait(self.h, int(limit_cycles), _stream(stream)))

    def status(self, stream=None):
        self.check(self.L.st_status(self.h, _stream(stream)))

    def set_scoring(self, mode: int, horizon: int = 64):
        """Retention score of later ``KVCache.build`` calls (``st_set_scoring``)."""
        self.check(self.L.st_set_scoring(self.h, int(mode), int(horizon)))

    def kv_alloc(self, offsets: np.ndarray) -> "KVCache":
        return KVCache(self, offsets)

    def operator(self, op: synth.Operator) -> "Operator":
        return Operator(self, op)

    def gemm(self, A, W, C, stream=None):
        M, K = A.shape
        N = W.shape[0]
        self.check(self.L.st_gemm(self.h, _ptr(A), _ptr(W), M, N, K, _ptr(C), _stream(stream)))

    # ---- profiling
    def prof_enable(self, on: bool = True):
        self.check(self.L.st_prof_enable(self.h, 1 if on else 0))

    def prof_reset(self):
        self.check(self.L.st_prof_reset(self.h))

    def prof_read(self) -> Dict[str, Dict[str, float]]:
        buf = (ctypes.c_double * 16)()
        self.check(self.L.st_prof_read(self.h, buf))
        out = {}
        for i, name in enumerate(PROF_FAMILIES):
            out[name] = {"launches": buf[4 * i], "ms": buf[4 * i + 1], "flops": buf[4 * i + 2],
                         "bytes": buf[4 * i + 3]}
        return out

    def launch_count(self) -> int:
        return int(self.L.st_launch_count(self.h))


class KVCache:
    """The caches of one table (an ``st_kv``)."""

    def __init__(self, model: Model, offsets: np.ndarray, _handle=None, _source=None):
        self.model = model
        self.L = model.L
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        self.offsets = off
        self.T = len(off) - 1
        self._source = _source       # a profile keeps its source cache alive
        if _handle is not None:
            self.h = _handle
            return
        h = VP()
        model.check(self.L.st_kv_alloc(model.h, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                       self.T, ctypes.byref(h)))
        self.h = h

    def profile(self, r_max: float = 1.0) -> "KVCache":
        """A second retained profile of this cache (``st_kv_profile_alloc``): shares
        the full cache, holds its own retained cache for any r <= r_max."""
        h = VP()
        self.model.check(self.L.st_kv_profile_alloc(self.model.h, self.h, float(r_max), ctypes.byref(h)))
        return KVCache(self.model, self.offsets, _handle=h, _source=self)

    def close(self):
        if getattr(self, "h", None):
            self.L.st_kv_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build(self, tokens, stream=None):
        self.model.check(self.L.st_kv_build(self.model.h, self.h, _ptr(tokens), _stream(stream)))

    def retain(self, r: float, kv_dtype: Optional[int] = None, stream=None):
        if kv_dtype is None:
            kv_dtype = ST_BF16 if self.model.cfg.dtype == "bf16" else ST_F32
        self.model.check(self.L.st_kv_retain(self.model.h, self.h, float(r), int(kv_dtype),
                                             _stream(stream)))
        self.kv_dtype, self.r = int(kv_dtype), float(r)

    def status(self, stream=None):
        self.model.check(self.L.st_kv_status(self.model.h, self.h, _stream(stream)))

    def indices(self, r: float, stream=None):
        """The retained slot indices at fraction r (st_kv_indices): returns
        (idx int32 [layers, hkv, total], off int64 [T+1]) on the device; tuple t's
        indices, in rank order, are idx[l, g, off[t]:off[t+1]]."""
        import torch
        cfg = self.model.cfg
        off = torch.empty(self.T + 1, dtype=torch.int64, device="cuda")
        self.model.check(self.L.st_kv_indices(self.model.h, self.h, float(r), None, _ptr(off), _stream(stream)))
        total = int(off[-1].item())
        idx = torch.empty((cfg.layers, cfg.hkv, max(total, 1)), dtype=torch.int32, device="cuda")
        self.model.check(self.L.st_kv_indices(self.model.h, self.h, float(r), _ptr(idx), _ptr(off),
                                              _stream(stream)))
        return idx[:, :, :total], off

    def export_profile(self, stream=None) -> np.ndarray:
        """The current retained profile as a host byte array (``st_kv_export``)."""
        n = ctypes.c_size_t()
        self.model.check(self.L.st_kv_profile_bytes(self.h, ctypes.byref(n)))
        buf = np.empty(n.value, dtype=np.uint8)
        self.model.check(self.L.st_kv_export(self.model.h, self.h, buf.ctypes.data_as(VP), n.value,
                                             _stream(stream)))
        return buf

    def import_profile(self, blob: np.ndarray, stream=None):
        """Make a blob from ``export_profile`` this cache's retained profile (``st_kv_import``)."""
        blob = np.ascontiguousarray(blob, dtype=np.uint8)
        self.model.check(self.L.st_kv_import(self.model.h, self.h, blob.ctypes.data_as(VP), blob.nbytes,
                                             _stream(stream)))

    def save_profile(self, path: str):
        self.export_profile().tofile(path)

    def load_profile(self, path: str):
        self.import_profile(np.fromfile(path, dtype=np.uint8))

    def score_query(self, op: "Operator", stream=None):
        """Replace the scores by ``op``'s query-specific ones (``st_kv_score_query``;
        needs a retained profile at r = 1 in the model dtype)."""
        self.model.check(self.L.st_kv_score_query(self.model.h, self.h, op.h, _stream(stream)))

    def view_bytes(self, which: int) -> int:
        p, n = VP(), ctypes.c_size_t()
        self.model.check(self.L.st_kv_view(self.h, which, ctypes.byref(p), ctypes.byref(n)))
        return int(n.value)

    def read(self, which: int, dtype, shape, stream=None):
        """Copy a cache view into a new torch tensor of the given dtype and shape."""
        import torch
        out = torch.empty(shape, dtype=dtype, device="cuda")
        nbytes = out.numel() * out.element_size()
        self.model.check(self.L.st_kv_read(self.h, which, _ptr(out), nbytes, _stream(stream)))
        return out

    def read_at(self, which: int, dtype, shape, offset_elems: int, stream=None):
        """Copy a contiguous piece of a view, starting at element ``offset_elems``."""
        import torch
        out = torch.empty(shape, dtype=dtype, device="cuda")
        es = out.element_size()
        self.model.check(self.L.st_kv_read_at(self.h, which, int(offset_elems) * es, _ptr(out),
                                              out.numel() * es, _stream(stream)))
        return out


class Operator:
    """An operator's prompt / labels / thresholds uploaded once (an ``st_operator``)."""

    def __init__(self, model: Model, op: synth.Operator):
        self.model = model
        self.L = model.L
        self.op = op
        P = len(op.prompt)
        nl = len(op.label_ids)
        self._prompt = (ctypes.c_int32 * P)(*op.prompt)
        self._labels = (ctypes.c_int32 * nl)(*op.label_ids)
        self._bias = (ctypes.c_float * nl)(*(op.bias if op.bias is not None else [0.0] * nl))
        d = OpDesc(ctypes.cast(self._prompt, ctypes.POINTER(ctypes.c_int32)), P,
                   ctypes.cast(self._labels, ctypes.POINTER(ctypes.c_int32)), nl,
                   ST_OP_CLASSIFY if op.kind == "classify" else ST_OP_FILTER, float(op.r),
                   float(op.theta_pos), float(op.theta_neg),
                   ctypes.cast(self._bias, ctypes.POINTER(ctypes.c_float)))
        h = VP()
        model.check(self.L.st_op_create(model.h, ctypes.byref(d), ctypes.byref(h)))
        self.h = h
        self.n_labels = nl

    def close(self):
        if getattr(self, "h", None):
            self.L.st_op_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def eval(self, kv: KVCache, tuple_ids, logits=None, labels=None, stream=None):
        """Run the operator on the device tuple ids; returns (logits, labels) device tensors."""
        import torch
        n = int(tuple_ids.numel())
        if logits is None:
            logits = torch.empty((n, self.n_labels), dtype=torch.float32, device="cuda")
        if labels is None:
            labels = torch.empty((n,), dtype=torch.int32, device="cuda")
        self.model.check(self.L.st_op_eval(self.model.h, kv.h, self.h, _ptr(tuple_ids), n,
                                           _ptr(logits), _ptr(labels), _stream(stream)))
        return logits, labels

    def map(self, kv: KVCache, tuple_ids, n_gen: int, with_logits: bool = False, stream=None):
        """Greedy decode of n_gen tokens per tuple (``st_map_eval``); returns the
        [n][n_gen] token tensor (and the [n][n_gen][vocab] logits if asked)."""
        import torch
        n = int(tuple_ids.numel())
        tokens = torch.empty((n, n_gen), dtype=torch.int32, device="cuda")
        logits = (torch.empty((n, n_gen, self.model.cfg.vocab), dtype=torch.float32, device="cuda")
                  if with_logits else None)
        self.model.check(self.L.st_map_eval(self.model.h, kv.h, self.h, _ptr(tuple_ids), n, int(n_gen),
                                            _ptr(tokens), _ptr(logits) if logits is not None else None,
                                            _stream(stream)))
        return (tokens, logits) if with_logits else tokens

    def eval_noalloc(self, kv: KVCache, tuple_ids, logits, labels, stream=None):
        """Same as ``eval`` through the entry that allocates no device memory (its
        activations live in the library's fixed-size static scratch array)."""
        n = int(tuple_ids.numel())
        self.model.check(self.L.st_op_eval_noalloc(self.model.h, kv.h, self.h, _ptr(tuple_ids), n,
                                                   _ptr(logits), _ptr(labels), _stream(stream)))
        return logits, labels

    def run_host(self, kv: KVCache, tokens_host, logits_host, labels_host, kv_dtype: int,
                 stream=None):
        """Whole path from host buffers (pinned torch CPU tensors)."""
        self.model.check(self.L.st_run_host(self.model.h, kv.h, self.h, int(kv_dtype),
                                            _ptr(tokens_host), _ptr(logits_host),
                                            _ptr(labels_host), _stream(stream)))


class Proxy:
    """The learned proxy MLP (an ``st_proxy``) and the cascade routing kernels."""

    def __init__(self, model: Model, params: Dict[str, np.ndarray]):
        self.model = model
        self.L = model.L
        self.h1, self.d = params["w1"].shape
        self.h2 = params["w2"].shape[0]
        self._init = [np.ascontiguousarray(params[k], dtype=np.float32) for k in PROXY_ORDER]
        arr = (VP * 6)(*[a.ctypes.data for a in self._init])
        h = VP()
        model.check(self.L.st_proxy_create(model.h, self.d, self.h1, self.h2, arr, ctypes.byref(h)))
        self.h = h
        self.sizes = [a.size for a in self._init]
        self.shapes = [a.shape for a in self._init]

    def close(self):
        if getattr(self, "h", None):
            self.L.st_proxy_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def train_step(self, x, y, batch, lr: float, loss=None, stream=None):
        self.model.check(self.L.st_proxy_train_step(
            self.model.h, self.h, _ptr(x), _ptr(y), _ptr(batch), int(batch.numel()),
            float(lr), _ptr(loss) if loss is not None else None, _stream(stream)))

    def eval(self, x, rows=None, n=None, conf=None, label=None, stream=None):
        import torch
        n = int(rows.numel()) if rows is not None else (int(x.shape[0]) if n is None else n)
        conf = torch.empty(n, dtype=torch.float32, device="cuda") if conf is None else conf
        label = torch.empty(n, dtype=torch.int32, device="cuda") if label is None else label
        self.model.check(self.L.st_proxy_eval(self.model.h, self.h, _ptr(x),
                                              _ptr(rows) if rows is not None else None, n,
                                              _ptr(conf), _ptr(label), _stream(stream)))
        return conf, label

    def set_precision(self, dtype: int):
        """ST_F32 (float32 contractions) or ST_BF16 (tensor-core BF16 contractions)."""
        self.model.check(self.L.st_proxy_set_precision(self.h, int(dtype)))

    def steps(self) -> int:
        """Adam steps taken (st_proxy_steps)."""
        return int(self.L.st_proxy_steps(self.h))

    def state(self):
        """The training state for a checkpoint: flat device copies of the
        parameters and Adam moments, and the step count."""
        import torch
        n = sum(self.sizes)
        out = {}
        for name, which in (("params", ST_PROXY_PARAMS), ("m", ST_PROXY_ADAM_M), ("v", ST_PROXY_ADAM_V)):
            out[name] = torch.empty(n, dtype=torch.float32, device="cuda")
            self.model.check(self.L.st_proxy_read(self.h, which, _ptr(out[name]), n * 4, _stream()))
        out["steps"] = self.steps()
        return out

    def restore(self, state, stream=None):
        """Resume from ``state()`` of a proxy of the same shape (st_proxy_restore).
        Each of params / m / v must be a contiguous float32 CUDA tensor of
        n_params elements; the library refuses any other size."""
        import torch
        n = sum(self.sizes)
        for k in ("params", "m", "v"):
            t = state[k]
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise ValueError(f"proxy state '{k}' must be a contiguous float32 CUDA tensor")
            if t.numel() != n:
                raise ValueError(f"proxy state '{k}' holds {t.numel()} values, this proxy has {n}")
        nbytes = state["params"].numel() * 4
        self.model.check(self.L.st_proxy_restore(self.h, _ptr(state["params"]), _ptr(state["m"]),
                                                  _ptr(state["v"]), nbytes, int(state["steps"]),
                                                  _stream(stream)))

    def read(self, which: int) -> Dict[str, np.ndarray]:
        import torch
        out = torch.empty(sum(self.sizes), dtype=torch.float32, device="cuda")
        self.model.check(self.L.st_proxy_read(self.h, which, _ptr(out), out.numel() * 4,
                                              _stream()))
        flat = out.cpu().numpy()
        res, o = {}, 0
        for k, sz, shp in zip(PROXY_ORDER, self.sizes, self.shapes):
            res[k] = flat[o:o + sz].reshape(shp)
            o += sz
        return res


def cascade_compact(model: Model, conf, tau: float, ids=None, out=None, count=None, stream=None):
    import torch
    n = int(conf.numel())
    out = torch.empty(max(n, 1), dtype=torch.int32, device="cuda") if out is None else out
    count = torch.zeros(1, dtype=torch.int32, device="cuda") if count is None else count
    model.check(model.L.st_cascade_compact(model.h, _ptr(conf), _ptr(ids) if ids is not None else None,
                                           n, float(tau), _ptr(out), _ptr(count), _stream(stream)))
    return out, count


def cascade_merge(model: Model, proxy_label, unsure_pos, count, full_label, out=None, stream=None):
    import torch
    n = int(proxy_label.numel())
    out = torch.empty(n, dtype=torch.int32, device="cuda") if out is None else out
    model.check(model.L.st_cascade_merge(model.h, _ptr(proxy_label), n, _ptr(unsure_pos),
                                         _ptr(count), _ptr(full_label), _ptr(out), _stream(stream)))
    return out


def eval_multi(model: Model, kv: KVCache, ops, tuple_ids, logits=None, labels=None, stream=None):
    """Several operators, each over its own device tuple ids, in one batched pass
    (``st_op_eval_multi``); returns the lists of (logits, labels) device tensors."""
    args, logits, labels = _multi_args(ops, tuple_ids, logits, labels)
    model.check(model.L.st_op_eval_multi(model.h, kv.h, *args, _stream(stream)))
    return logits, labels


def _multi_args(ops, tuple_ids, logits, labels):
    import torch
    k = len(ops)
    ns = [int(t.numel()) for t in tuple_ids]
    if logits is None:
        logits = [torch.empty((n, o.n_labels), dtype=torch.float32, device="cuda") for n, o in zip(ns, ops)]
    if labels is None:
        labels = [torch.empty((n,), dtype=torch.int32, device="cuda") for n in ns]
    arr = lambda xs: (VP * k)(*[_ptr(x) for x in xs])
    return (k, (VP * k)(*[o.h for o in ops]), arr(tuple_ids), (ctypes.c_int32 * k)(*ns), arr(logits),
            arr(labels)), logits, labels


class Graph:
    """A batched evaluation recorded as a CUDA graph (``st_graph``).  Keeps the
    tuple-id and output tensors it was created with (``logits``, ``labels``)."""

    def __init__(self, model: Model, kv: KVCache, ops, tuple_ids, logits=None, labels=None):
        self.model, self.L = model, model.L
        args, self.logits, self.labels = _multi_args(ops, tuple_ids, logits, labels)
        self._keep = (ops, tuple_ids, kv)
        h = VP()
        model.check(self.L.st_graph_create(model.h, kv.h, *args, ctypes.byref(h)))
        self.h = h

    def launch(self, stream=None):
        self.model.check(self.L.st_graph_launch(self.h, _stream(stream)))

    def launches(self) -> int:
        return int(self.L.st_graph_launches(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.L.st_graph_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(model: Model, kv: KVCache, ops, tuple_ids, logits=None, labels=None, stream=None):
    """Time candidate evaluation schedules on this batch (``st_autotune_eval``);
    returns (best, tried) as dicts.  The best schedule stays set in the model."""
    args, logits, labels = _multi_args(ops, tuple_ids, logits, labels)
    best = TuneChoice()
    tried = (TuneChoice * 32)()
    nt = ctypes.c_int32()
    model.check(model.L.st_autotune_eval(model.h, kv.h, *args, _stream(stream), ctypes.byref(best), tried,
                                         32, ctypes.byref(nt)))
    return best.as_dict(), [tried[i].as_dict() for i in range(nt.value)]


def set_schedule(model: Model, eval_rows: int = 0, attn_nb: int = 1, longest_first: int = 1,
                 split_keys: int = 0):
    sc = TuneChoice(int(eval_rows), int(attn_nb), int(longest_first), int(split_keys), 0.0)
    model.check(model.L.st_set_schedule(model.h, ctypes.byref(sc)))


def cascade_run(stages, tuple_ids, labels=None, stage=None, stream=None):
    """Multi-stage cascade over device tuple ids; stages = [(model, kv, operator)].
    Returns (labels, deciding stage, tuples sent to each stage, ms per stage)."""
    import torch
    n = int(tuple_ids.numel())
    k = len(stages)
    labels = torch.empty(n, dtype=torch.int32, device="cuda") if labels is None else labels
    stage = torch.empty(n, dtype=torch.int32, device="cuda") if stage is None else stage
    arr = (StageDesc * k)(*[StageDesc(m.h, kv.h, op.h) for m, kv, op in stages])
    counts = (ctypes.c_int32 * k)()
    ms = (ctypes.c_float * k)()
    m0 = stages[0][0]
    m0.check(m0.L.st_cascade_run(k, arr, _ptr(tuple_ids), n, _ptr(labels), _ptr(stage), counts, ms,
                                 _stream(stream)))
    return labels, stage, list(counts), list(ms)


def proxy_cascade(proxy: "Proxy", x, tau: float, stages, tuple_ids, labels=None, stage=None, stream=None):
    """The learned-proxy cascade in one call (``st_proxy_cascade``): the proxy on
    rows ``tuple_ids`` of the pooled states ``x``, confident tuples (conf >= tau)
    decided by it, the rest through the operator ``stages`` = [(model, kv,
    operator)].  Returns (labels, deciding stage: 0 proxy / k+1 operator stage k,
    tuples the proxy saw then tuples sent to each stage)."""
    import torch
    n = int(tuple_ids.numel())
    k = len(stages)
    labels = torch.empty(max(n, 1), dtype=torch.int32, device="cuda") if labels is None else labels
    stage = torch.empty(max(n, 1), dtype=torch.int32, device="cuda") if stage is None else stage
    arr = (StageDesc * k)(*[StageDesc(m.h, kv.h, op.h) for m, kv, op in stages])
    counts = (ctypes.c_int32 * (k + 1))()
    m = proxy.model
    m.check(m.L.st_proxy_cascade(m.h, proxy.h, _ptr(x), float(tau), k, arr, _ptr(tuple_ids), n, _ptr(labels),
                                 _ptr(stage), counts, _stream(stream)))
    return labels, stage, list(counts)


def set_gemm_pairs(on: bool):
    """Process-wide GEMM kernel choice (``st_set_gemm_pairs``)."""
    lib().st_set_gemm_pairs(1 if on else 0)


def version() -> str:
    return lib().st_version().decode()
