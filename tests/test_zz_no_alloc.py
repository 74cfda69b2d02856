"""The operator entry that allocates no device memory, against the regular entry.

Callers that cannot let the library call cudaMalloc / cudaFree (an executor
that must not synchronise the device, or a process whose GPU memory belongs to
another framework's caching allocator) use st_op_eval_noalloc, whose
activations live in the library's static scratch array.  Its logits and labels
must match st_op_eval's on the same caches, on two calls in a row (the second
call finds the first call's data in the shared array), and a batch larger than
the array must be refused with a clear error.  This file is collected last.
"""
import numpy as np
import pytest

from tests.util import normwise_rel

pytestmark = pytest.mark.gpu

LENGTHS = [1, 64, 65, 300, 700, 2048]


@pytest.fixture(scope="module")
def setup():
    import torch
    from paper_2602_04430_b300 import build, stretto, synth
    build.build()
    cfg = synth.MODELS["c2_bf16"]
    w = synth.make_weights(cfg, seed=31)
    table = synth.make_table_from_lengths(LENGTHS, cfg.vocab, seed=32, ids="zipf")
    model = stretto.Model(cfg, w, max_pos=4096)
    kv = model.kv_alloc(table["offsets"])
    kv.build(torch.from_numpy(table["tokens"]).cuda())
    kv.retain(0.5)
    op = synth.make_prompt(32, cfg.vocab, seed=33, label_ids=(1, 0), r=0.5)
    opr = model.operator(op)
    return dict(model=model, kv=kv, opr=opr, stretto=stretto, torch=torch)


@pytest.mark.parametrize("order", [[0, 1, 2, 3, 4, 5], [5, 3, 1, 0, 2, 4, 4]])
def test_noalloc_matches_regular_entry_twice(setup, order):
    torch, opr, kv = setup["torch"], setup["opr"], setup["kv"]
    ids = torch.tensor(order, dtype=torch.int32, device="cuda")
    ref_z, ref_l = opr.eval(kv, ids)
    torch.cuda.synchronize()
    ref_z, ref_l = ref_z.cpu().numpy(), ref_l.cpu().numpy()
    for call in range(2):
        z = torch.full((len(order), 2), float("nan"), dtype=torch.float32, device="cuda")
        lab = torch.full((len(order),), -1, dtype=torch.int32, device="cuda")
        opr.eval_noalloc(kv, ids, z, lab)
        torch.cuda.synchronize()
        setup["model"].status()
        z, lab = z.cpu().numpy(), lab.cpu().numpy()
        assert np.isfinite(z).all()
        assert normwise_rel(z, ref_z) <= 2e-2, call
        np.testing.assert_array_equal(lab, ref_l)


def test_noalloc_refuses_batches_beyond_the_scratch(setup):
    torch, opr, kv, stretto = setup["torch"], setup["opr"], setup["kv"], setup["stretto"]
    n = 4096   # 4096 tuples x 32 prompt rows need far more than the static scratch
    ids = torch.zeros(n, dtype=torch.int32, device="cuda")
    z = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    lab = torch.empty((n,), dtype=torch.int32, device="cuda")
    with pytest.raises(stretto.StrettoError) as e:
        opr.eval_noalloc(kv, ids, z, lab)
    assert e.value.code == stretto.ST_EINVAL
    assert "static scratch" in str(e.value)
