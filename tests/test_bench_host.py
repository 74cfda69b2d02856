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
    assert bench.attention_bytes(cfg, nkeep, 2) == kv_bf16
    # E4M3: one byte a value, plus a float32 K and V scale per 64-slot block
    scales = 2 * 4 * 2 * 2 * 4
    assert bench.attention_bytes(cfg, nkeep, 1) == kv_bf16 // 2 + scales
    # reported apart: per prompt row (4 tuples x P = 2) and layer, Q and O (hq * hd
    # each) plus the row's own K and V (hkv * hd each), 2 bytes a value
    assert bench.prompt_attention_bytes(cfg, 8) == 2 * 8 * 2 * 4 * (8 + 4)


def test_band_decision_and_cascade_labels_hand_case():
    import numpy as np
    import bench
    # theta = 1, delta = 0.5: accept above 1.5, reject below 0.5, unsure between (ties unsure)
    m8 = np.array([2.0, 1.5, 1.0, 0.5, 0.0, 1.2], dtype=np.float32)
    np.testing.assert_array_equal(bench.decide_band_f32(m8, 1.5, 0.5), [1, 2, 2, 2, 0, 2])
    conf = np.array([0.99, 0.6, 0.95, 0.5, 0.7, 0.55], dtype=np.float32)
    plab = np.array([1, 0, 0, 1, 1, 0])
    plain = np.array([1, 1, 1, 0, 0, 1])
    lab, to8, to16 = bench.cascade_labels(conf, plab, m8, plain, 1.0, 0.9, 0.5)
    # conf >= 0.9: the proxy (tuples 0, 2); else E4M3 (tuples 1, 3, 4, 5): decided 4 (reject),
    # inside the band 1, 3, 5 -> plain
    np.testing.assert_array_equal(lab, [1, 1, 0, 0, 0, 1])
    np.testing.assert_array_equal(to8, [False, True, False, True, True, True])
    np.testing.assert_array_equal(to16, [False, True, False, True, False, True])


def test_operating_point_is_the_cheapest_that_reaches_the_target():
    import numpy as np
    import bench
    rng = np.random.Generator(np.random.PCG64(0))
    n = 2000
    plain = rng.integers(0, 2, n)
    m8 = np.where(plain == 1, 1.0, -1.0) + rng.normal(0, 0.4, n)      # theta 0: some FP8 flips near 0
    m8 = m8.astype(np.float32)
    conf = rng.uniform(0.5, 1.0, n).astype(np.float32)
    # the proxy is right exactly when it is confident above 0.8
    plab = np.where(conf >= 0.8, plain, 1 - plain)
    cost = {"proxy": 0.01, "e4m3": 1.0, "bf16": 1.2}
    pt = bench.choose_operating_point(conf, plab, m8, plain, 0.0, cost, 0.99)
    assert not pt["plain_only"]
    lab, to8, to16 = bench.cascade_labels(conf, plab, m8, plain, 0.0, pt["tau"], pt["delta"])
    assert (lab == plain).mean() >= 0.99
    assert pt["cost"] == pytest.approx(0.01 + to8.mean() * 1.0 + to16.mean() * 1.2)
    # every confident tuple can go to the proxy: the fallback is the unconfident part
    assert pt["fallback"] <= (conf < 0.8).mean() + 0.02
    # when the E4M3 stage is dearer than BF16 and the proxy is always wrong, plain BF16 alone wins
    pt2 = bench.choose_operating_point(conf, 1 - plain, m8, plain, 0.0, {"proxy": 0.01, "e4m3": 2.0, "bf16": 1.0},
                                       0.99)
    assert pt2["plain_only"] and pt2["cost"] == 1.0


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
