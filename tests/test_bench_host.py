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


def test_tensor_roofline_algorithmic_and_executed():
    peak = bench.MEASURED["bf16_tflops"]
    alg = 0.25 * peak * 1e12 * 1e-3           # a quarter of the peak over 1 ms
    r = bench.tensor_roofline(alg, 3 * alg, 1.0, {"sm_mhz": 2070.0}, traffic=2.0e6, ncu_active=0.5)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s" and r["traffic"] == 2.0e6
    assert abs(r["frac"] - 0.25) < 1e-12 and abs(r["frac_executed"] - 0.75) < 1e-12
    assert r["sampled_sm_mhz"] == 2070.0 and r["ncu_tensor_pipe_active"] == 0.5
    sus = bench.MEASURED.get("bf16_tflops_sustained")
    if sus:
        assert abs(r["frac_of_sustained_peak"] - r["achieved"] / sus) < 1e-12


def test_dftgemm_flop_counts():
    # the pruned 128 x 128 DFT as real products: 4 per complex product, two stages
    assert bench.DG_ALG_FLOP_PER_IMAGE == 4 * 2 * 128 * 64 * 64 + 4 * 2 * 128 * 128 * 64 == 12582912
    assert bench.DG_FLOP_PER_IMAGE == 3 * bench.DG_ALG_FLOP_PER_IMAGE
