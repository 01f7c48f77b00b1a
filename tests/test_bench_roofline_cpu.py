"""Host-side arithmetic of the benchmark's roofline record (no GPU): which
bound a kernel class is reported against and how its ceiling is derived."""
import bench


def _k(ms, flops, byts, launches=10):
    return {"ms": ms, "flops": flops, "bytes": byts, "launches": launches}


def test_tensor_class_uses_the_3xtf32_ceiling():
    peaks = {"hbm_gbs": 6794.1, "bf16_tflops_sustained": 1701.3, "sm_max_mhz": 2070.0}
    kern = {"gemm_tcgen05": _k(1000.0, 5.0e13, 1.0e12), "copy": _k(10.0, 0.0, 1.0e10)}
    rl, name = bench.roofline(kern, "f32", peaks, "measured")
    assert name == "gemm_tcgen05" and rl["bound"] == "tensor"
    assert abs(rl["peak"] - 1701.3 * 1.1 / 2.25 / 3.0) < 1e-9
    assert abs(rl["achieved"] - 50.0) < 1e-9  # 5e13 flops in 1 s
    assert abs(rl["frac"] - 50.0 / rl["peak"]) < 1e-12
    assert rl["traffic"] is None


def test_memory_bound_class_uses_measured_hbm():
    peaks = {"hbm_gbs": 6794.1, "bf16_tflops_sustained": 1701.3, "sm_max_mhz": 2070.0}
    kern = {"copy": _k(100.0, 0.0, 3.0e11)}
    rl, _ = bench.roofline(kern, "f32", peaks, "measured")
    assert rl["bound"] == "hbm" and abs(rl["achieved"] - 3000.0) < 1e-6
    assert abs(rl["frac"] - 3000.0 / 6794.1) < 1e-12


def test_fallback_peaks_cover_every_branch():
    peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}
    for name in ("gemm_tcgen05", "pivoted_cholesky"):
        rl, _ = bench.roofline({name: _k(10.0, 1.0e12, 1.0e9)}, "f32", peaks, "fallback")
        assert rl["frac"] > 0.0


def test_class_table_covers_every_class_with_its_bound():
    peaks = {"hbm_gbs": 6794.1, "bf16_tflops_sustained": 1701.3, "sm_max_mhz": 2070.0}
    kern = {"gemm_tcgen05": _k(500.0, 2.0e13, 1.0e12), "copy": _k(100.0, 0.0, 3.0e11),
            "pivoted_cholesky": _k(300.0, 1.0e12, 5.0e11), "permute": _k(0.0, 0.0, 1.0)}
    t = bench.class_table(kern, "f32", peaks, "measured")
    assert set(t) == {"gemm_tcgen05", "copy", "pivoted_cholesky"}  # zero-time classes are left out
    assert abs(sum(v["share"] for v in t.values()) - 1.0) < 1e-12
    assert t["gemm_tcgen05"]["bound"] == "tensor" and t["copy"]["bound"] == "hbm"
    assert t["pivoted_cholesky"]["bound"] == "alu"
    assert abs(t["copy"]["achieved"] - 3000.0) < 1e-3
    assert list(t)[0] == "gemm_tcgen05"  # largest device time first


def test_threaded_oracle_operator_and_converged_cg():
    """The CPU baseline's threaded product equals the oracle's sparse product,
    and the converged run reaches the requested residual."""
    import numpy as np

    import synthetic
    from oracle import operator as op

    n = 8
    g = synthetic.gaussian_random_field(n, 1)
    f = synthetic.uniform_rhs(n, 100)
    A = op.assemble(n, g)
    x = np.random.default_rng(0).standard_normal(n ** 3)
    Aop = bench.threaded_operator(A, 3)
    np.testing.assert_allclose(Aop @ x, A @ x, rtol=0, atol=0)
    conv = bench.cpu_converged(n, g, f, 1e-10, threads=2)
    assert conv["converged"] and conv["rel_residual"] <= 1e-10 and conv["iters"] > 5
    rec = bench.cpu_baseline_record(n, conv, 1e-10)
    assert rec["kind"] == "oracle" and rec["threads"] == 2 and "converged" in rec["sample"]
    assert bench.cpu_chunk(Aop, f, 7) > 0.0
