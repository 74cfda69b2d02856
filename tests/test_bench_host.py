"""Host-side pieces of the benchmark that decide what the JSON line claims:
the compulsory attention bytes behind the roofline fraction (a hand-worked
case) and the clock record parsed from nvidia-smi samples (throttle reasons,
median clock, peak power), fed a fake sample file."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_attention_bytes_hand_case():
    import bench
    from paper_2602_04430_b300 import synth
    cfg = synth.ModelConfig(layers=2, d=16, hq=4, hkv=2, hd=4, ffn=32, vocab=64)
    nkeep = [2, 5, 32, 33]           # retained counts (sum 72; one 64-slot block each)
    # per layer and kv head the retained K and V, 2 bytes a value: 2 * 2 * 2 * 4 * 2 * 72
    kv_bf16 = 4608
    # per prompt row (4 tuples x P = 2) and layer: Q and O (hq * hd each) plus the
    # row's own K and V (hkv * hd each), 2 bytes a value: 2 * 8 * 2 * 4 * (8 + 4)
    prompt = 1536
    assert bench.attention_bytes(cfg, nkeep, 2, 2) == kv_bf16 + prompt
    # E4M3: one byte a value, plus a float32 K and V scale per 64-slot block
    scales = 2 * 4 * 2 * 2 * 4
    assert bench.attention_bytes(cfg, nkeep, 1, 2) == kv_bf16 // 2 + scales + prompt


def test_clock_record_reports_throttle_reasons():
    import bench
    cs = bench.ClockSampler(0)
    rows = [
        "0, 1350, 2032, 1080.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1300, 2032, 1095.0, 0x0000000000000008, Active, Not Active, Not Active, Active",
        "0, 1400, 2032, 900.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    cs.f.write("\n".join(rows) + "\n")
    s = cs.summary()
    assert s["sm_mhz"] == 1350.0 and s["sm_max_mhz"] == 2032.0
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert s["samples"] == 3 and s["power_w_max"] == pytest.approx(1095.0)


def test_clock_record_without_samples():
    import bench
    cs = bench.ClockSampler(0)
    assert cs.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
