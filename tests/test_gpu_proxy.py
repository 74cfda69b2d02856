"""The learned proxy on the GPU against the FP64 oracle: gradients of one step,
parameters after several Adam steps, confidences and labels, and the cascade's
routing (compaction and merge, bit-exact on the kernel's own confidences)."""
import numpy as np
import pytest

from tests.util import normwise_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    from paper_2602_04430_b300 import build, stretto, synth
    build.build()
    cfg = synth.ModelConfig(layers=1, d=256, hq=4, hkv=2, hd=64, ffn=256, vocab=512, dtype="bf16")
    model = stretto.Model(cfg, synth.make_weights(cfg, seed=1), max_pos=256)
    d_in = 1024
    params = synth.make_proxy_weights(d_in, 512, 128, seed=5)
    r = np.random.Generator(np.random.PCG64(6))
    x = r.standard_normal((2048, d_in)).astype(np.float32)
    y = (x[:, :8].sum(axis=1) + 0.5 * r.standard_normal(2048) > 0).astype(np.int32)
    return dict(model=model, params=params, x=x, y=y, torch=torch, stretto=stretto, synth=synth)


def test_gradients_of_one_step(setup):
    from oracle import proxy as PX
    torch, stretto = setup["torch"], setup["stretto"]
    px = stretto.Proxy(setup["model"], setup["params"])
    x, y = setup["x"], setup["y"]
    batch = np.arange(3, 3 + 384, dtype=np.int32)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    px.train_step(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(),
                  torch.from_numpy(batch).cuda(), lr=0.0, loss=loss)
    torch.cuda.synchronize()
    g = px.read(stretto.ST_PROXY_GRADS)
    ref_loss, ref = PX.loss_and_grads({k: v.astype(np.float64) for k, v in setup["params"].items()},
                                      x[batch], y[batch])
    assert abs(loss.item() - ref_loss) <= 1e-5 * abs(ref_loss)
    for k in ref:
        assert normwise_rel(g[k], ref[k]) <= 1e-4, k


def test_adam_steps_match_oracle(setup):
    from oracle import proxy as PX
    torch, stretto, synth = setup["torch"], setup["stretto"], setup["synth"]
    px = stretto.Proxy(setup["model"], setup["params"])
    x, y = setup["x"], setup["y"]
    batches = synth.minibatches(len(x), 256, 2, seed=9)[:12]
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    for b in batches:
        px.train_step(xd, yd, torch.from_numpy(b).cuda(), lr=1e-3)
    torch.cuda.synchronize()
    got = px.read(stretto.ST_PROXY_PARAMS)
    ref, losses = PX.train(setup["params"], x, y, batches, lr=1e-3)
    # Adam divides by sqrt(v): where a gradient sits at the float32 rounding level
    # its normalised update can differ by O(lr) from the FP64 one, so the updates
    # are compared in the L2 norm, plus a bound on the fraction of such elements.
    for k in ref:
        delta_ref = ref[k] - setup["params"][k]
        delta_got = got[k].astype(np.float64) - setup["params"][k]
        l2 = np.linalg.norm(delta_got - delta_ref) / np.linalg.norm(delta_ref)
        assert l2 <= 1e-3, (k, l2)
        far = np.abs(delta_got - delta_ref) > 1e-3 * np.abs(delta_ref).max()
        assert far.mean() <= 1e-3, (k, far.mean())
    # eval: confidences and labels of the trained network
    conf, lab = px.eval(xd)
    torch.cuda.synchronize()
    rconf, rlab = PX.confidence_and_label(ref, x)
    conf, lab = conf.cpu().numpy(), lab.cpu().numpy()
    assert normwise_rel(conf, rconf) <= 1e-4
    clear = np.abs(rconf - 0.5) > 1e-4
    np.testing.assert_array_equal(lab[clear], rlab[clear])


@pytest.mark.parametrize("tau", [0.0, 0.6, 0.9, 1.01])
def test_cascade_routing_bit_exact(setup, tau):
    from oracle import proxy as PX
    torch, stretto = setup["torch"], setup["stretto"]
    model = setup["model"]
    r = np.random.Generator(np.random.PCG64(11))
    n = 3000
    conf = (0.5 + 0.5 * r.random(n)).astype(np.float32)
    plab = r.integers(0, 2, n).astype(np.int32)
    ids = r.permutation(10 * n)[:n].astype(np.int32)
    cd, pl = torch.from_numpy(conf).cuda(), torch.from_numpy(plab).cuda()
    pos, cnt = stretto.cascade_compact(model, cd, tau)
    tid, cnt2 = stretto.cascade_compact(model, cd, tau, ids=torch.from_numpy(ids).cuda())
    torch.cuda.synchronize()
    k = int(cnt.item())
    ref_pos = np.nonzero(conf < np.float32(tau))[0]
    assert k == len(ref_pos) == int(cnt2.item())
    np.testing.assert_array_equal(pos.cpu().numpy()[:k], ref_pos)
    np.testing.assert_array_equal(tid.cpu().numpy()[:k], ids[ref_pos])
    full = r.integers(0, 2, n).astype(np.int32)
    full_unsure = torch.from_numpy(full[ref_pos] if k else np.zeros(1, np.int32)).cuda()
    merged = stretto.cascade_merge(model, pl, pos, cnt, full_unsure)
    torch.cuda.synchronize()
    ref, unsure = PX.cascade(plab, conf, np.float32(tau), full)
    np.testing.assert_array_equal(merged.cpu().numpy(), ref)


def test_training_resumes_from_a_checkpoint(setup):
    """st_proxy_steps / st_proxy_restore: a fresh proxy restored from another's
    state (parameters, Adam moments, step count) after 5 steps continues
    exactly: the next 3 steps give both the same parameters bit for bit."""
    torch, stretto, synth = setup["torch"], setup["stretto"], setup["synth"]
    x, y = setup["x"], setup["y"]
    batches = synth.minibatches(len(x), 256, 1, seed=11)[:8]
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    a = stretto.Proxy(setup["model"], setup["params"])
    for b in batches[:5]:
        a.train_step(xd, yd, torch.from_numpy(b).cuda(), lr=1e-3)
    state = a.state()
    assert state["steps"] == 5
    c = stretto.Proxy(setup["model"], setup["params"])
    assert c.steps() == 0
    c.restore(state)
    assert c.steps() == 5
    for b in batches[5:]:
        bd = torch.from_numpy(b).cuda()
        a.train_step(xd, yd, bd, lr=1e-3)
        c.train_step(xd, yd, bd, lr=1e-3)
    torch.cuda.synchronize()
    pa, pc = a.read(stretto.ST_PROXY_PARAMS), c.read(stretto.ST_PROXY_PARAMS)
    for k in pa:
        assert np.array_equal(pa[k], pc[k]), k
    assert a.steps() == c.steps() == 8


def test_restore_refuses_a_state_of_another_shape(setup):
    """A checkpoint of a proxy with another hidden width (or a truncated buffer)
    is refused before anything is read: by the binding's checks, and by the
    library's own size check when the C entry is called directly."""
    import ctypes
    torch, stretto, synth = setup["torch"], setup["stretto"], setup["synth"]
    a = stretto.Proxy(setup["model"], setup["params"])
    d = a.d
    other = stretto.Proxy(setup["model"], synth.make_proxy_weights(d, 64, 32, seed=5))
    with pytest.raises(ValueError):
        a.restore(other.state())
    st = a.state()
    short = dict(st, params=st["params"][:-1].contiguous())
    with pytest.raises(ValueError):
        a.restore(short)
    # the C entry itself: a byte count that is not n_params * 4
    n = st["params"].numel() * 4
    rc = a.L.st_proxy_restore(a.h, stretto._ptr(st["params"]), stretto._ptr(st["m"]), stretto._ptr(st["v"]),
                              ctypes.c_size_t(n - 4), 3, stretto._stream())
    assert rc == stretto.ST_EINVAL
    assert a.steps() == 0
    a.restore(st)
    torch.cuda.synchronize()


def test_bf16_contractions_match_the_oracle(setup):
    """st_proxy_set_precision(ST_BF16): the tensor-core BF16 contractions
    against the oracle's BF16 reading (each product's operands rounded to
    bfloat16, exact accumulation): loss and gradients of one step, then
    parameters after 12 Adam steps and the confidences they give.  A rounded
    operand is a decision taken in float32 on both sides, but its input comes
    from a float32 (GPU) or float64 (oracle) accumulation, so a few roundings
    land on neighbouring bfloat16 values: the bound is a few units of
    bfloat16's 2^-8, well under the distance to the float32 network."""
    from oracle import proxy as PX
    torch, stretto, synth = setup["torch"], setup["stretto"], setup["synth"]
    x, y = setup["x"], setup["y"]
    p64 = {k: v.astype(np.float64) for k, v in setup["params"].items()}
    px = stretto.Proxy(setup["model"], setup["params"])
    px.set_precision(stretto.ST_BF16)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    batch = np.arange(3, 3 + 384, dtype=np.int32)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    px.train_step(xd, yd, torch.from_numpy(batch).cuda(), lr=0.0, loss=loss)
    torch.cuda.synchronize()
    g = px.read(stretto.ST_PROXY_GRADS)
    ref_loss, ref = PX.loss_and_grads(p64, x[batch], y[batch], bf=True)
    _, ref32 = PX.loss_and_grads(p64, x[batch], y[batch])
    assert abs(loss.item() - ref_loss) <= 1e-4 * abs(ref_loss)
    for k in ref:
        err = normwise_rel(g[k], ref[k])
        assert err <= 4e-3, (k, err)
        if k.startswith("w"):
            assert err < 0.5 * normwise_rel(ref32[k], ref[k]) or err <= 1e-4, k
    # Adam steps, then confidences.  Adam divides each gradient by its own
    # running magnitude, so where a gradient is near zero the few bfloat16
    # roundings that land differently can flip its sign and move that weight by
    # up to ~lr per step: the bound is per element, 2 lr per step.
    px2 = stretto.Proxy(setup["model"], setup["params"])
    px2.set_precision(stretto.ST_BF16)
    lr = 1e-3
    batches = synth.minibatches(len(x), 256, 2, seed=19)[:12]
    for b in batches:
        px2.train_step(xd, yd, torch.from_numpy(b).cuda(), lr=lr)
    torch.cuda.synchronize()
    ours = px2.read(stretto.ST_PROXY_PARAMS)
    ref_p, _ = PX.train(p64, x, y, batches, lr=lr, bf=True)
    for k in ref_p:
        assert np.abs(ours[k] - ref_p[k]).max() <= 2 * lr * len(batches), k
        assert normwise_rel(ours[k], ref_p[k]) <= 5e-2, k
    conf, lab = px2.eval(xd[:512])
    c_ref, l_ref = PX.confidence_and_label(ref_p, x[:512], bf=True)
    assert np.abs(conf.cpu().numpy() - c_ref).max() <= 2e-2
    assert (lab.cpu().numpy() == l_ref).mean() >= 0.98
    with pytest.raises(stretto.StrettoError):
        px2.set_precision(stretto.ST_E4M3)
