"""Host-side helpers of bench.py: the clock/throttle summary and the byte accounting
behind the roofline fields (no GPU)."""
import bench


def test_clock_summary_counts_only_active_reasons():
    text = "\n".join([
        "0, 2070, 2070, 850.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 900.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ])
    out = bench.Clocks.summarise(text)
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert out["samples"] == 3
    quiet = bench.Clocks.summarise(text.replace(", Active", ", Not Active"))
    assert quiet["reasons"] == []


def test_cg_byte_accounting():
    # k1: gauge + p + t; k2: gauge + t + r (2x) + x (2x, FP32 for 16-bit formats) + p; k3: r + p (2x)
    assert bench.CG_BYTES["f16_12"] == {"k1": 96 + 2 * 52, "k2": 96 + 4 * 52 + 2 * 96, "k3": 3 * 52}
    assert bench.CG_BYTES["i16_12"] == bench.CG_BYTES["f16_12"]
    assert bench.CG_BYTES["f32_12"] == {"k1": 192 + 2 * 96, "k2": 192 + 6 * 96, "k3": 3 * 96}
    assert bench.CG_BYTES["f64"]["k2"] == 576 + 6 * 192
    assert bench.DSLASH_BYTES["f64"] == 960 and bench.DSLASH_BYTES["f16_12"] == 200
