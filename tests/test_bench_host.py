"""Host-only checks of the benchmark's roofline arithmetic (no GPU): the
algorithmic counts per pixel that `achieved` divides by, the FP32 ALU peak
derived from unit counts and clock, and the DRAM-traffic pin, which must
follow the kernel it was captured on."""
import importlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def test_split_roofline_of_the_tensor_core_stage(bench):
    """Mixed precision: T_min = max(conv flops / tensor peak, (phi + prox) flops /
    FP32 peak), the binding term reported with frac = T_min / T."""
    class Wl:
        flops_per_px_stage = bench.FLOPS_PER_PX_STAGE
        flops = 1e9 * bench.FLOPS_PER_PX_STAGE     # 1e9 pixel-stages
        traffic, kernel, launches = None, "tc", 8
    assert bench.CONV_FLOPS_PER_PX_STAGE + bench.ALU_FLOPS_PER_PX_STAGE == bench.FLOPS_PER_PX_STAGE
    peaks = {"bf16_tflops_sustained": 1700.0}
    ms = 200.0
    r = bench._split_roofline(Wl, "tf32", ms, peaks, "measured", 80.0, 152, 2070.0)
    t_alu = 1e9 * 6060 / 80e12
    t_tc = 1e9 * 9408 / (1700e12 * 1.1 / 2.25)
    assert r["bound"] == "alu" and t_alu > t_tc
    assert r["frac"] == pytest.approx(t_alu / (ms / 1e3))
    assert r["achieved"] / r["peak"] == pytest.approx(r["frac"])
    assert r["terms"]["tensor"]["frac"] == pytest.approx(t_tc / (ms / 1e3))
    # BF16 doubles the tensor peak: the ALU term binds all the more
    r2 = bench._split_roofline(Wl, "bf16", ms, peaks, "measured", 80.0, 152, 2070.0)
    assert r2["terms"]["tensor"]["peak"] == pytest.approx(1700.0)


def test_split_roofline_of_the_mixed_training_step(bench):
    """Training with a tensor-core forward: only the forward's filter bank and
    adjoint go on the tensor term; phi, the prox and the whole FP32 backward on
    the ALU term, which binds."""
    class Wl:
        flops_per_px_stage = bench.FLOPS_PER_PX_STAGE + bench.BWD_FLOPS_PER_PX_STAGE
        flops = 1e8 * flops_per_px_stage
        conv_flops_per_px_stage = bench.CONV_FLOPS_PER_PX_STAGE
        alu_flops_per_px_stage = bench.ALU_FLOPS_PER_PX_STAGE + bench.BWD_FLOPS_PER_PX_STAGE
        traffic, kernel, launches = None, "tc + bwd", 30
    assert (Wl.conv_flops_per_px_stage + Wl.alu_flops_per_px_stage == Wl.flops_per_px_stage)
    ms = 10.0
    r = bench._split_roofline(Wl, "tf32", ms, {"bf16_tflops_sustained": 1700.0}, "measured",
                              80.0, 152, 2070.0)
    t_alu = 1e8 * Wl.alu_flops_per_px_stage / 80e12
    assert r["bound"] == "alu"
    assert r["frac"] == pytest.approx(t_alu / (ms / 1e3))
    assert r["terms"]["tensor"]["flops"] == pytest.approx(1e8 * bench.CONV_FLOPS_PER_PX_STAGE)
    assert "FP32 backward" in r["achieved_basis"]


def test_reference_arm_config_equals_the_default_workload_config(bench):
    # the driver compares the two arms' config: the reference line must name
    # the same workload keys as the GPU arm's default line
    assert bench.CONFIG["data_term"] == "idiv" and bench.CONFIG["H"] == bench.H == 512


def test_bench_names_resolve():
    """Every name a bench.py function reads from outside its scopes is a module
    global or a builtin (a workload constructor that names an undefined variable
    fails only when that workload runs on a GPU)."""
    import builtins
    import symtable
    src = open(os.path.join(ROOT, "bench.py")).read()
    top = symtable.symtable(src, "bench.py", "exec")
    module_names = {s.get_name() for s in top.get_symbols() if s.is_assigned() or s.is_imported()}
    known = module_names | set(dir(builtins))
    bad = []

    def walk(t, path):
        for child in t.get_children():
            p = f"{path}.{child.get_name()}"
            if child.get_type() == "function":
                for sym in child.get_symbols():
                    if sym.is_global() and sym.is_referenced() and sym.get_name() not in known:
                        bad.append((p, sym.get_name()))
            walk(child, p)

    walk(top, "bench")
    assert not bad, bad
