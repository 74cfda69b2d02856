"""The checked build (libstretto_check.so, -DST_CHECK): every ragged offset
and index the kernels follow is checked before use (retention segments, the
attention's work records, the label head's rows, the cascade's scatter
positions, the index gather).  On valid inputs no check fires and the results
are bit-identical to the regular build's; each library runs in its own
process (STRETTO_CHECK selects it).  And the always-on check of the public
merge entry: a position outside [0, n) is skipped and reported."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASE = r'''
import json, sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
from paper_2602_04430_b300 import stretto, synth
cfg = synth.ModelConfig(layers=2, d=256, hq=8, hkv=2, hd=64, ffn=512, vocab=512, dtype="bf16", name="chk")
w = synth.make_weights(cfg, seed=31)
lengths = [1, 2, 63, 64, 65, 127, 129, 300, 700, 1500]
table = synth.make_table_from_lengths(lengths, cfg.vocab, seed=32)
model = stretto.Model(cfg, w, max_pos=1600)
kv = model.kv_alloc(table["offsets"])
kv.build(torch.from_numpy(table["tokens"]).cuda())
T = kv.T
ids = torch.tensor([9, 0, 3, 3, 7, 1, 8, 2, 6, 5, 4], dtype=torch.int32, device="cuda")
out = {}
for name, code in (("bf16", stretto.ST_BF16), ("e4m3", stretto.ST_E4M3)):
    kv.retain(0.5, code)
    for r in (0.5, 0.25):
        op = model.operator(synth.make_prompt(24, cfg.vocab, seed=33, r=r))
        lg, lb = op.eval(kv, ids)
        out[f"{name}_{r}_logits"] = lg.cpu().numpy().tolist()
        out[f"{name}_{r}_labels"] = lb.cpu().numpy().tolist()
kv.retain(0.5, stretto.ST_BF16)
toks = model.operator(synth.make_prompt(16, cfg.vocab, seed=34, r=0.5)).map(kv, ids[:4], 3)
out["map"] = toks.cpu().numpy().tolist()
idx, idx_off = kv.indices(0.25)
out["indices"] = idx.cpu().numpy().tolist()
torch.cuda.synchronize()
model.status()
kv.status()
print("RESULT " + json.dumps(out))
'''


def _run(check: bool):
    env = dict(os.environ)
    env["STRETTO_CHECK"] = "1" if check else "0"
    code = "ROOT = %r\n" % ROOT + CASE
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT ")][-1]
    return json.loads(line[7:])


def test_checked_build_is_clean_and_bit_identical():
    from paper_2602_04430_b300 import build
    build.build()
    build.build(check=True)
    a, b = _run(False), _run(True)
    assert set(a) == set(b)
    for k in a:
        np.testing.assert_array_equal(np.asarray(a[k]), np.asarray(b[k]), err_msg=k)


def test_merge_skips_and_reports_positions_outside_the_table():
    import torch
    from paper_2602_04430_b300 import build, stretto, synth
    build.build()
    cfg = synth.MODELS["tiny_f32"]
    model = stretto.Model(cfg, synth.make_weights(cfg, seed=1), max_pos=512)
    model.status()
    n = 6
    proxy_lab = torch.tensor([1, 1, 0, 0, 1, 0], dtype=torch.int32, device="cuda")
    pos = torch.tensor([2, 6, 4], dtype=torch.int32, device="cuda")        # 6 is outside [0, 6)
    count = torch.tensor([3], dtype=torch.int32, device="cuda")
    full = torch.tensor([7, 8, 9], dtype=torch.int32, device="cuda")
    out = stretto.cascade_merge(model, proxy_lab, pos, count, full)
    torch.cuda.synchronize()
    with pytest.raises(stretto.StrettoError) as e:
        model.status()
    assert e.value.code == stretto.ST_ERANGE
    model.status()
    assert out.cpu().tolist() == [1, 1, 7, 0, 9, 0]
    assert n == out.numel()
