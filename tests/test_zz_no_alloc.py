"""The operator entry that allocates no device memory, against the regular entry.

Callers that cannot let the library call cudaMalloc / cudaFree (an executor
that must not synchronise the device, or a process whose GPU memory belongs to
another framework's caching allocator) use st_op_eval_noalloc, whose
activations live in the library's static scratch array.  Checked here, on a
fresh context that has never evaluated an operator (bf16 and float32 models):

* it allocates nothing: across repeated calls the device's free memory, torch's
  allocator and the context's own workspaces stay exactly as they were, and the
  context's evaluation workspace stays empty (the first call on a device may
  still load the library's kernels and its scratch array's module, so the
  measurement starts after it);
* it computes what st_op_eval computes: the same kernels in the same order on
  one chunk, so logits and labels are bit-identical, on calls in a row (each
  finds the previous call's data in the shared array);
* a batch larger than the array is refused with a clear error.

This file is collected last.
"""
import gc

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LENGTHS = [1, 64, 65, 300, 700, 2048]


def _fresh(kind):
    import torch
    from paper_2602_04430_b300 import build, stretto, synth
    build.build()
    cfg = synth.MODELS[kind]
    w = synth.make_weights(cfg, seed=31)
    table = synth.make_table_from_lengths(LENGTHS, cfg.vocab, seed=32, ids="zipf")
    model = stretto.Model(cfg, w, max_pos=4096)
    kv = model.kv_alloc(table["offsets"])
    kv.build(torch.from_numpy(table["tokens"]).cuda())
    kv.retain(0.5)
    op = synth.make_prompt(32, cfg.vocab, seed=33, label_ids=(1, 0), r=0.5)
    return model, kv, model.operator(op), stretto, torch


@pytest.mark.parametrize("kind", ["c2_bf16", "tiny_f32"])
def test_noalloc_allocates_nothing_and_matches_the_regular_entry(kind):
    model, kv, opr, stretto, torch = _fresh(kind)
    assert model.workspace_held(stretto.ST_WS_EVAL) == 0
    held = model.workspace_held(stretto.ST_WS_ANY)
    orders = [[0, 1, 2, 3, 4, 5], [5, 3, 1, 0, 2, 4, 4], [0, 1, 2, 3, 4, 5]]
    ids = [torch.tensor(o, dtype=torch.int32, device="cuda") for o in orders]
    z = [torch.full((len(o), 2), float("nan"), dtype=torch.float32, device="cuda") for o in orders]
    lab = [torch.full((len(o),), -1, dtype=torch.int32, device="cuda") for o in orders]
    # first call: may load kernels / the scratch array's module on this device
    opr.eval_noalloc(kv, ids[0], z[0], lab[0])
    torch.cuda.synchronize()
    model.status()
    gc.collect()
    gc.disable()          # no finaliser of another test's objects may free memory meanwhile
    try:
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        alloc0 = torch.cuda.memory_allocated()
        for i in (1, 2):
            opr.eval_noalloc(kv, ids[i], z[i], lab[i])
            torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        alloc1 = torch.cuda.memory_allocated()
    finally:
        gc.enable()
    model.status()
    assert free1 == free0, (free0, free1)
    assert alloc1 == alloc0
    assert model.workspace_held(stretto.ST_WS_EVAL) == 0
    assert model.workspace_held(stretto.ST_WS_ANY) == held
    # only now the regular entry, which grows the context's evaluation workspace
    for i, o in enumerate(orders):
        ref_z, ref_l = opr.eval(kv, ids[i])
        torch.cuda.synchronize()
        np.testing.assert_array_equal(z[i].cpu().numpy(), ref_z.cpu().numpy())
        np.testing.assert_array_equal(lab[i].cpu().numpy(), ref_l.cpu().numpy())
    assert model.workspace_held(stretto.ST_WS_EVAL) > 0
    assert np.isfinite(z[1].cpu().numpy()).all()
    kv.close()
    model.close()


def test_noalloc_refuses_batches_beyond_the_scratch():
    model, kv, opr, stretto, torch = _fresh("c2_bf16")
    n = 4096   # 4096 tuples x 32 prompt rows need far more than the static scratch
    ids = torch.zeros(n, dtype=torch.int32, device="cuda")
    z = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    lab = torch.empty((n,), dtype=torch.int32, device="cuda")
    with pytest.raises(stretto.StrettoError) as e:
        opr.eval_noalloc(kv, ids, z, lab)
    assert e.value.code == stretto.ST_EINVAL
    assert "static scratch" in str(e.value)
    assert model.workspace_held(stretto.ST_WS_EVAL) == 0
    kv.close()
    model.close()
