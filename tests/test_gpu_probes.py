"""The throughput probes of bench.py (context for the roofline denominators)
measure plausible rates on the device: positive, ordered as the hardware's
pipes are (FP32 FMA above the special-function unit, which is above FP64 on
this part) and below a generous bound of the unit counts at 3 GHz."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

pytestmark = pytest.mark.gpu


def test_probes_are_positive_and_ordered():
    import torch

    import bench
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    r = {k: bench.peak_probe(k) for k in ("ffma", "dfma", "sfu", "alu", "copy")}
    assert all(v > 0 for v in r.values())
    assert r["ffma"] < sms * 128 * 3.0e9
    assert r["sfu"] < sms * 16 * 3.0e9
    assert r["ffma"] > r["sfu"] > r["dfma"]
    assert 1e11 < r["copy"] < 2e13
