"""Host-only checks of the benchmark's roofline arithmetic (no GPU): the
algorithmic counts per pixel that `achieved` divides by, the FP32 ALU peak
derived from unit counts and clock, and the DRAM-traffic pin, which must
follow the kernel it was captured on."""
import importlib
import sys

import pytest


@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ".")
    return importlib.import_module("bench")


def test_algorithmic_counts(bench):
    nk, ks, nrbf = 48, 7, 63
    # forward: filter bank + adjoint (2 N_k k^2 FMAs each), phi as written (63 FMAs
    # per response), the prox (~12)
    assert bench.FLOPS_PER_PX_STAGE == 2 * (2 * nk * ks * ks) + 2 * nk * nrbf + 12 == 15468
    # backward: five k x k contractions (z, b, the adjoint of c, dL/dk's two
    # correlations), three 63-term RBF sums (phi, phi', dL/dw), ~20 pointwise
    assert bench.BWD_FLOPS_PER_PX_STAGE == 5 * 2 * nk * ks * ks + 3 * 2 * nk * nrbf + 20
    # quality: 2 window means (121 FMA) + 3 second moments (121 mul + FMA) + the rest
    assert bench.QUALITY_FLOPS_PER_PX == 2 * 2 * 121 + 3 * 3 * 121 + 21 + 3 + 18 + 4 + 3 == 1622


def test_fp32_peak(bench):
    # 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2070 MHz
    assert bench._fp32_peak_tflops(2070.0, 152) == pytest.approx(152 * 128 * 2 * 2.070e9 / 1e12)


def test_traffic_pin_follows_the_captured_kernel(bench, monkeypatch):
    pin = bench._TRAFFIC
    monkeypatch.setattr(bench, "_kernel_sources_hash", lambda: pin["sources_sha256_16"])
    assert bench._measured_traffic(pin["kernel"]) == pin["bytes_per_launch"]
    assert bench._measured_traffic(pin["kernel"] + " (another)") is None
    # changed kernel sources: no traffic figure until it is captured again
    monkeypatch.setattr(bench, "_kernel_sources_hash", lambda: "0" * 16)
    assert bench._measured_traffic(pin["kernel"]) is None
    # at least one full plane read, below all three planes read and written
    assert 1 << 20 < pin["bytes_per_launch"] < 4 * (1 << 20)
