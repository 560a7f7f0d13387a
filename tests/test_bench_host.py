"""Host-side arithmetic of bench.py's roofline reporting (CPU only)."""
import bench


def test_alu_roofline_fractions():
    # 40.27 TFLOP/s achieved on 152 SMs: half the FP32 FMA rate at 2070 MHz
    peak = 152 * 128 * 2 * 2070e6 / 1e12
    flops = 0.5 * peak * 1e12 * 2e-3          # over 2 ms
    r = bench.alu_roofline(flops, 2.0, 152, {"sm_mhz": 1035.0}, traffic=1.0e6, flop_basis="x")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["traffic"] == 1.0e6 and r["flop_basis"] == "x"
    assert abs(r["peak"] - peak) < 1e-9 and abs(r["frac"] - 0.5) < 1e-12
    assert r["sampled_sm_mhz"] == 1035.0 and abs(r["frac_at_sampled_clock"] - 1.0) < 1e-12
    load = bench.MEASURED.get("clocks_under_load", {}).get("sm_mhz_median")
    if load:
        assert abs(r["frac_at_gemm_load_clock"] - 0.5 * 2070.0 / load) < 1e-12


def test_alu_roofline_without_clock_samples():
    r = bench.alu_roofline(1e12, 1.0, 152, {"sm_mhz": None, "reasons": ["nvidia-smi unavailable"]})
    assert "frac_at_sampled_clock" not in r and abs(r["achieved"] - 1000.0) < 1e-9
