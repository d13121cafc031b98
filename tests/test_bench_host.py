"""Host logic of bench.py that needs no GPU: the roofline objects built from
the library's per-kind timing stats, and the steady-state pole counts the
CPU baseline extrapolates to."""
import bench


def test_dominant_kernel_and_rooflines():
    peaks = {"bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
    # kind: (launches, ms, algorithmic flops) over 5 steps
    stats = {0: (100, 400.0, 6.8e13), 1: (100, 300.0, 2.55e13),
             2: (500, 9000.0, 9.0e15), 3: (500, 5500.0, 2.9e14)}
    dom, roofs = bench.kernel_rooflines(stats, 5, peaks, "measured")
    assert dom == 2
    r = roofs[2]
    assert r["bound"] == "alu" and r["peak"] == bench.FP64_NOMINAL_TFLOPS
    assert abs(r["achieved"] - 9.0e15 / 9.0 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 1.25) < 1e-12
    assert abs(r["ms_per_step"] - 1800.0) < 1e-9
    t = roofs[0]
    assert t["bound"] == "tensor" and t["peak"] == 1700.0
    assert abs(t["achieved"] - 170.0) < 1e-9 and abs(t["issued_tflops"] - 1020.0) < 1e-9
    # with a measured FP64 GEMM rate, the FP64 kinds are measured against it
    dom, roofs = bench.kernel_rooflines(stats, 5, peaks, "measured", fp64_peak=1.1)
    assert roofs[2]["peak"] == 1.1 and abs(roofs[2]["frac"] - roofs[2]["achieved"] / 1.1) < 1e-12
    assert "measured" in roofs[2]["peak_source"]
    # nothing timed: zero rates, no division by zero
    dom0, roofs0 = bench.kernel_rooflines({k: (0, 0.0, 0.0) for k in range(4)}, 1, peaks, "m")
    assert all(roofs0[k]["achieved"] == 0.0 for k in range(4))


def test_steady_state_pole_counts():
    from paper_2106_03508_gb300.synth import CONFIGS
    for nmom in (1, 3):
        s, o, v = bench._oracle_setup("c1", nmom)
        N = CONFIGS["c1"]["nmo"]
        assert o + v == (nmom + 2) * N
        assert o == CONFIGS["c1"]["nocc"] + (nmom + 1) // 2 * N


def test_oracle_sample_scales_both_sectors():
    """The CPU-baseline sample times a share of both outer summed indices plus
    one Fock cycle and extrapolates to one iteration: on the small c1 system
    the estimate exceeds the sample's own wall time and the description names
    both sectors."""
    t_iter, wall, desc = bench.oracle_sample("c1", 1, fock_cycles=3, frac=0.25)
    assert t_iter > 0 and wall > 0
    assert "occupied" in desc and "virtual" in desc and "x 3 cycles" in desc
