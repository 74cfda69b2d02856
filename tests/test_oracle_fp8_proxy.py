"""Pins of the oracle's FP8 E4M3 codec, block quantiser, proxy MLP, Adam and cascade (CPU only)."""
import math
import os

import numpy as np
import pytest
import torch

from oracle import fp8 as F
from oracle import proxy as PX

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_decode_all_256_codes_matches_torch():
    codes = torch.arange(256, dtype=torch.int32).to(torch.uint8)
    ref = codes.view(torch.float8_e4m3fn).to(torch.float64).numpy()
    ours = np.array([F.e4m3_decode(c) for c in range(256)])
    np.testing.assert_array_equal(np.isnan(ours), np.isnan(ref))
    m = ~np.isnan(ref)
    np.testing.assert_array_equal(ours[m], ref[m])
    np.testing.assert_array_equal(np.signbit(ours[m]), np.signbit(ref[m]))


def test_spec_points_golden():
    """Values fixed by the OCP 8-bit floating point specification (E4M3)."""
    path = os.path.join(GOLDEN, "e4m3_spec_points.txt")
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        code, val = line.split()
        v = F.e4m3_decode(int(code, 16))
        if val == "nan":
            assert np.isnan(v)
        else:
            assert v == float(val), (code, v, val)


def test_round_trip_every_finite_code():
    for c in range(256):
        v = F.e4m3_decode(c)
        if np.isnan(v):
            continue
        got = int(F.e4m3_encode(np.array([v]))[0])
        assert got == c, (hex(c), v, hex(got))


def test_encode_matches_torch_rn_even_including_ties():
    grid = np.array([F.e4m3_decode(c) for c in range(0x7F)])
    mids = (grid[1:] + grid[:-1]) / 2.0                      # exact ties (float32-representable)
    r = np.random.Generator(np.random.PCG64(1))
    vals = np.concatenate([mids, -mids, r.uniform(-448, 448, 20000), r.standard_normal(5000) * 1e-2,
                           r.standard_normal(5000) * 1e-3]).astype(np.float32)
    ref = torch.from_numpy(vals).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    ours = F.e4m3_encode(vals)
    np.testing.assert_array_equal(ours, ref)


def test_saturation():
    assert int(F.e4m3_encode(np.array([1000.0]))[0]) == 0x7E
    assert int(F.e4m3_encode(np.array([-1e9]))[0]) == 0xFE
    assert int(F.e4m3_encode(np.array([448.0]))[0]) == 0x7E
    assert int(F.e4m3_encode(np.array([464.0]))[0]) == 0x7E   # beyond the grid: saturates


@pytest.mark.parametrize("arith", ["f64", "f32"])
def test_block_quantiser_error_bound(arith):
    r = np.random.Generator(np.random.PCG64(2))
    x = r.standard_normal((150, 64)) * np.exp(r.standard_normal((150, 1)))
    x[64:128] = 0.0                                   # an all-zero block: scale 1, exact
    codes, scales, deq = F.quantize_blocks(x, arith)
    assert scales.shape == (3,)
    assert float(scales[1]) == 1.0
    np.testing.assert_array_equal(deq[64:128], 0.0)
    for b in (0, 2):
        blk = x[b * 64:(b + 1) * 64]
        s = float(scales[b])
        np.testing.assert_allclose(s, np.abs(blk).max() / 448.0, rtol=1e-6)
        err = np.abs(blk - deq[b * 64:(b + 1) * 64])
        bound = np.maximum(np.abs(blk) * 2.0 ** -4, s * 2.0 ** -10) * (1 + 1e-6)
        assert np.all(err <= bound)
        assert np.abs(deq[b * 64:(b + 1) * 64]).max() == pytest.approx(np.abs(blk).max(), rel=1e-6)


def _proxy_params(seed=0, din=12, h1=8, h2=6):
    r = np.random.Generator(np.random.PCG64(seed))
    return {"w1": r.standard_normal((h1, din)) / np.sqrt(din), "b1": 0.1 * r.standard_normal(h1),
            "w2": r.standard_normal((h2, h1)) / np.sqrt(h1), "b2": 0.1 * r.standard_normal(h2),
            "w3": r.standard_normal((2, h2)) / np.sqrt(h2), "b3": 0.1 * r.standard_normal(2)}


def _torch_mlp(p, x):
    t = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in p.items()}
    h = torch.nn.functional.gelu(torch.from_numpy(x) @ t["w1"].T + t["b1"])
    h = torch.nn.functional.gelu(h @ t["w2"].T + t["b2"])
    return h @ t["w3"].T + t["b3"], t


def test_proxy_grads_match_autograd_and_finite_differences():
    p = _proxy_params()
    r = np.random.Generator(np.random.PCG64(3))
    x = r.standard_normal((10, 12))
    y = r.integers(0, 2, 10)
    loss, g = PX.loss_and_grads(p, x, y)
    z, t = _torch_mlp(p, x)
    tl = torch.nn.functional.cross_entropy(z, torch.from_numpy(y))
    tl.backward()
    assert abs(loss - tl.item()) < 1e-13
    for k in p:
        np.testing.assert_allclose(g[k], t[k].grad.numpy(), rtol=1e-10, atol=1e-13)
    # central finite differences on a few coordinates
    for k in ("w1", "b2", "w3"):
        flat = p[k].reshape(-1)
        for i in (0, flat.size // 2, flat.size - 1):
            h = 1e-6
            pp = {kk: vv.copy() for kk, vv in p.items()}
            pm = {kk: vv.copy() for kk, vv in p.items()}
            pp[k].reshape(-1)[i] += h
            pm[k].reshape(-1)[i] -= h
            fd = (PX.loss_and_grads(pp, x, y)[0] - PX.loss_and_grads(pm, x, y)[0]) / (2 * h)
            assert abs(fd - g[k].reshape(-1)[i]) <= 1e-7 * max(1.0, abs(fd))


def test_adam_matches_torch():
    p = _proxy_params(4)
    r = np.random.Generator(np.random.PCG64(5))
    x = r.standard_normal((32, 12))
    y = r.integers(0, 2, 32)
    batches = [np.arange(i, i + 8) for i in range(0, 32, 8)] * 3
    ours, losses = PX.train(p, x, y, batches, lr=1e-2)
    t = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in p.items()}
    opt = torch.optim.Adam(list(t.values()), lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for bi in batches:
        opt.zero_grad()
        h = torch.nn.functional.gelu(torch.from_numpy(x[bi]) @ t["w1"].T + t["b1"])
        h = torch.nn.functional.gelu(h @ t["w2"].T + t["b2"])
        z = h @ t["w3"].T + t["b3"]
        torch.nn.functional.cross_entropy(z, torch.from_numpy(y[bi])).backward()
        opt.step()
    for k in p:
        np.testing.assert_allclose(ours[k], t[k].detach().numpy(), rtol=1e-9, atol=1e-12)
    assert losses[-1] < losses[0]


def test_gelu_matches_torch():
    x = np.linspace(-8, 8, 1001)
    np.testing.assert_allclose(PX.gelu(x), torch.nn.functional.gelu(torch.from_numpy(x)).numpy(),
                               rtol=1e-13, atol=1e-16)


def test_cascade_worked_example_golden():
    """The soft-pick example of Sec. 4.1 (continuous relaxation paragraph)."""
    path = os.path.join(GOLDEN, "cascade_soft_pick_example.txt")
    rows = {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            key, *vals = line.split()
            rows[key] = [float(v) for v in vals]
    acc, rej, uns, _ = PX.cascade_soft(rows["picks"], rows["accepts"], rows["rejects"])
    exp = rows["expected_accept_reject_unsure"]
    np.testing.assert_allclose([acc, rej, uns], exp, atol=1e-15)
    # after the partially picked first operator alone
    a1, r1, u1, _ = PX.cascade_soft(rows["picks"][:1], rows["accepts"][:1], rows["rejects"][:1])
    np.testing.assert_allclose([a1, r1, u1], rows["expected_after_first"], atol=1e-15)


def test_hard_cascade_and_cost():
    # picks in {0,1}: a tuple rejected by stage 1 never reaches stage 2, and costs only stage 1
    a, r, u, c = PX.cascade_soft([1, 1], [0, 1], [1, 0], costs=[1.0, 10.0])
    assert (a, r, u, c) == (0.0, 1.0, 0.0, 1.0)
    a, r, u, c = PX.cascade_soft([1, 1], [0, 1], [0, 0], costs=[1.0, 10.0])
    assert (a, r, u, c) == (1.0, 0.0, 0.0, 11.0)
    a, r, u, c = PX.cascade_soft([0, 1], [1, 0], [0, 1], costs=[1.0, 10.0])   # stage 1 not selected
    assert (a, r, u, c) == (0.0, 1.0, 0.0, 10.0)
    lab, uns = PX.cascade(np.array([1, 0, 1]), np.array([0.9, 0.5, 0.7]), 0.6, np.array([0, 1, 0]))
    assert lab.tolist() == [1, 1, 1] and uns.tolist() == [False, True, False]


def test_bf16_rounding_matches_torch_cast():
    r = np.random.Generator(np.random.PCG64(11))
    x = np.concatenate([r.standard_normal(20000) * 10.0 ** r.integers(-30, 30, 20000),
                        np.array([0.0, -0.0, 1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 3.0e38, -1e-40])])
    x = x.astype(np.float32)
    # exact half-way cases: the 16 discarded bits are 0x8000, both parities of the kept bit
    u = (r.integers(0, 2 ** 15, 2000, dtype=np.uint32) << 17) | np.uint32(0x3F800000) | np.uint32(0x8000)
    u2 = u | np.uint32(0x10000)
    ties = np.concatenate([u.view(np.float32), u2.view(np.float32)])
    for v in (x, ties):
        ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
        np.testing.assert_array_equal(PX.bf16(v), ref)


def test_bf16_contractions_match_torch_with_rounded_operands():
    """The BF16 forward / backward against a torch float64 run that casts each
    product's operands through torch.bfloat16, and against the exact network
    within bfloat16's resolution; a dropped rounding point changes the result."""
    p = _proxy_params(6, din=40, h1=24, h2=16)
    r = np.random.Generator(np.random.PCG64(7))
    x = r.standard_normal((12, 40))
    y = r.integers(0, 2, 12)
    rb = lambda a: a.to(torch.bfloat16).to(torch.float64)
    t = {k: torch.tensor(v, dtype=torch.float64) for k, v in p.items()}
    xt = torch.from_numpy(x)
    a1 = rb(xt) @ rb(t["w1"]).T + t["b1"]
    h1 = torch.nn.functional.gelu(a1)
    a2 = rb(h1) @ rb(t["w2"]).T + t["b2"]
    h2 = torch.nn.functional.gelu(a2)
    z = rb(h2) @ rb(t["w3"]).T + t["b3"]
    zo, _ = PX.forward(p, x, bf=True)
    np.testing.assert_allclose(zo, z.numpy(), rtol=1e-13, atol=1e-14)
    # backward: the same chain rule, operands of every product through bfloat16
    pr = torch.softmax(z, 1)
    dz = pr.clone()
    dz[torch.arange(12), torch.from_numpy(y)] -= 1.0
    dz /= 12
    ref = {"w3": rb(dz).T @ rb(h2), "b3": dz.sum(0)}
    gelu_d = lambda a: 0.5 * (1 + torch.erf(a / math.sqrt(2))) + a * torch.exp(-0.5 * a * a) / math.sqrt(2 * math.pi)
    da2 = (rb(dz) @ rb(t["w3"])) * gelu_d(a2)
    ref.update({"w2": rb(da2).T @ rb(h1), "b2": da2.sum(0)})
    da1 = (rb(da2) @ rb(t["w2"])) * gelu_d(a1)
    ref.update({"w1": rb(da1).T @ rb(xt), "b1": da1.sum(0)})
    _, g = PX.loss_and_grads(p, x, y, bf=True)
    for k in ref:
        np.testing.assert_allclose(g[k], ref[k].numpy(), rtol=1e-12, atol=1e-15)
    # within bfloat16 resolution of the exact network, and not equal to it
    _, g64 = PX.loss_and_grads(p, x, y)
    for k in ("w1", "w2", "w3"):
        rel = np.abs(g[k] - g64[k]).max() / np.abs(g64[k]).max()
        assert 1e-5 < rel < 3e-2, (k, rel)


def test_shared_e4m3_profile_blocks_are_the_profiles():
    """An E4M3 profile retained at r_p and read by an operator of r < r_p: the
    blocks and scales are the profile's, the operator reads the first
    n_keep(L, r) rows.  Pinned against quantize_blocks itself on the profile's
    rank-ordered set: equal to quantising the operator's own set when its size
    is a multiple of 64 (blocks coincide), and differing from it only in the
    last, partial block otherwise."""
    from oracle import fp8 as F8
    from oracle import operator as O
    from paper_2602_04430_b300 import synth
    cfg = synth.ModelConfig(layers=1, d=64, hq=2, hkv=1, hd=16, ffn=96, vocab=97, dtype="f32", name="prof")
    w = synth.make_weights(cfg, seed=41, std=0.3)
    doc = np.random.default_rng(42).integers(0, cfg.vocab, 256)
    c = O.kv_build(cfg, w, doc)
    full = O.rank_order(c.scores[0][0])
    # same ratio: identical to the plain E4M3 path
    a = O.retained_kv(c, 0.5, kv_fp8=True, fp8_profile_r=0.5)
    b = O.retained_kv(c, 0.5, kv_fp8=True)
    np.testing.assert_array_equal(a[0][0][0], b[0][0][0])
    # n = 128 of a 256-slot profile: whole blocks, equal to quantising the prefix
    k128 = O.retained_kv(c, 0.5, kv_fp8=True, fp8_profile_r=1.0)[0][0][0]
    np.testing.assert_array_equal(k128, F8.quantize_blocks(c.k[0][0][full[:128]])[2])
    # n = n_keep(256, 0.4) (not a multiple of 64): the profile's blocks, cut;
    # a large key in the partial block beyond n sets that block's scale
    n = O.n_keep(256, 0.4)
    assert n % 64 != 0
    c.k[0][0][full[n]] = 50.0 * c.k[0][0][full[n]]
    kp = O.retained_kv(c, 0.4, kv_fp8=True, fp8_profile_r=1.0)[0][0][0]
    prof = F8.quantize_blocks(c.k[0][0][full])[2]
    np.testing.assert_array_equal(kp, prof[:n])
    own = F8.quantize_blocks(c.k[0][0][full[:n]])[2]
    cut = 64 * (n // 64)
    np.testing.assert_array_equal(kp[:cut], own[:cut])
    assert not np.array_equal(kp[cut:], own[cut:])    # the partial block's scale differs
