"""The CTA-pair GEMM (2-SM MMA, 256 x 256 tiles) against the single-CTA GEMM
and a float64 product: plain-store GEMMs on ragged shapes (M not a multiple
of the 256-row pair tile, one pair tile only partly inside M), and the whole
build + retain + evaluate path, whose projections use every fused epilogue
(QKV + RoPE scatter, residual + RMSNorm statistics, SwiGLU).  Both kernels
run the same K steps in the same order, so their results must agree bit for
bit."""
import pytest

from tests.util import normwise_rel

pytestmark = pytest.mark.gpu


@pytest.fixture()
def pairs_restored():
    from paper_2602_04430_b300 import stretto
    yield stretto
    stretto.set_gemm_pairs(True)


@pytest.mark.parametrize("M,N,K", [(129, 256, 64), (255, 1536, 1024), (257, 1024, 2816),
                                   (1000, 5632, 1024), (4173, 1024, 1024), (65536, 256, 128)])
def test_pair_gemm_equals_single(pairs_restored, M, N, K):
    import torch
    from paper_2602_04430_b300 import build, synth
    stretto = pairs_restored
    build.build()
    cfg = synth.MODELS["c2_bf16"]
    model = stretto.Model(cfg, synth.make_weights(cfg, seed=301), max_pos=2200)
    g = torch.Generator(device="cuda").manual_seed(M + 3 * N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    W = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    out = {}
    for on in (True, False):
        stretto.set_gemm_pairs(on)
        C = torch.full((M, N), float("nan"), device="cuda", dtype=torch.float32)
        model.gemm(A, W, C)
        torch.cuda.synchronize()
        model.status()
        out[on] = C
    assert torch.equal(out[True], out[False])
    ref = A.double() @ W.double().T
    assert normwise_rel(out[True].cpu().numpy(), ref.cpu().numpy()) <= 1e-5


def test_full_path_identical_with_pairs(pairs_restored):
    import torch
    from paper_2602_04430_b300 import build, synth
    stretto = pairs_restored
    build.build()
    cfg = synth.MODELS["c2_bf16"]
    table = synth.make_table(synth.TABLES["c2"], cfg.vocab, seed=302, n_tuples=96)
    model = stretto.Model(cfg, synth.make_weights(cfg, seed=303), max_pos=2200)
    kv = model.kv_alloc(table["offsets"])
    tok = torch.from_numpy(table["tokens"]).cuda()
    op = model.operator(synth.make_prompt(32, cfg.vocab, seed=304, r=0.5))
    ids = torch.arange(kv.T, dtype=torch.int32, device="cuda")
    R = int(table["offsets"][-1])
    res = {}
    for on in (True, False):
        stretto.set_gemm_pairs(on)
        kv.build(tok)
        kv.retain(0.5)
        lg, lb = op.eval(kv, ids)
        torch.cuda.synchronize()
        model.status()
        Kc = kv.read(stretto.ST_VIEW_K, torch.bfloat16, (cfg.layers, cfg.hkv, R, cfg.hd)).clone()
        S = kv.read(stretto.ST_VIEW_SCORES, torch.float32, (cfg.layers, cfg.hkv, R)).clone()
        P = kv.read(stretto.ST_VIEW_POOLED, torch.float32, (kv.T, cfg.d)).clone()
        res[on] = (Kc, S, P, lg.clone(), lb.clone())
    for a, b in zip(res[True], res[False]):
        assert torch.equal(a, b)
