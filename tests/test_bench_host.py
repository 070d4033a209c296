"""Host-side logic of bench.py (no GPU): the roofline arithmetic, the clock
sampler's window filter and reasons, the CPU sample, and the DRAM traffic
recorded from ncu against the algorithmic bytes of each kernel."""
import math

import numpy as np
import pytest
import torch

import bench

M, NB, NF = 393216, 38, 257


def test_qhat_bytes_per_point():
    # nf frequencies x 2 nb real rows; bf16x3 keeps hi + lo BF16 (4 bytes)
    assert bench.qhat_bytes_per_point(NB, NF, "bf16x3") == NF * 2 * NB * 4
    assert bench.qhat_bytes_per_point(NB, NF, "bf16") == NF * 2 * NB * 2
    assert bench.qhat_bytes_per_point(NB, NF, "fp64") == NF * 2 * NB * 8


@pytest.mark.parametrize("phase,extra", [("fft", "x"), ("modes", "phi"), ("mean", "x")])
def test_kernel_roofline_credits_only_algorithmic_bytes(phase, extra):
    # the FFT and the mean are credited with X read once, the modes with Phi
    # written; the Qhat written and read back is overhead, reported apart
    peaks = {"hbm_gbs": 6000.0}
    ms = 10.0
    r = bench.kernel_roofline(phase, ms, M, NB, NF, NB, peaks, "bf16x3")
    q = NF * 2 * NB * 4 * M
    x = bench.NT * M * 4
    phi = NF * NB * M * 8
    want = {"x": x, "phi": phi}[extra]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["bytes_per_launch"] == want
    assert r["achieved"] == pytest.approx(want / (ms * 1e-3) / 1e9, abs=0.051)   # rounded to 0.1 GB/s
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0, abs=1e-4)
    if phase != "mean":
        assert r["overhead_bytes"] == q


def test_tensor_gram_roofline_is_on_tensor_flops():
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops_sustained": 1500.0}
    r = bench.kernel_roofline("gram", 5.0, M, NB, NF, NB, peaks, "bf16x3")
    flops = 3 * 8.0 * NF * NB * NB * M
    assert r["bound"] == "tensor" and r["peak"] == 1500.0
    assert r["achieved"] == pytest.approx(flops / 5e-3 / 1e12, rel=1e-3)
    assert r["overhead_bytes"] == NF * 2 * NB * 4 * M
    r1 = bench.kernel_roofline("gram", 5.0, M, NB, NF, NB, peaks, "bf16")
    assert r1["achieved"] == pytest.approx(r["achieved"] / 3, rel=1e-3)


def test_kernel_roofline_alu_forms():
    peaks = {"hbm_gbs": 6000.0}
    r = bench.kernel_roofline("gram", 50.0, M, NB, NF, NB, peaks, "fp32")
    flops = 4.0 * NF * NB * (NB + 1) * M
    assert r["bound"] == "alu" and r["achieved"] == pytest.approx(flops / 50e-3 / 1e12, rel=1e-3)
    r = bench.kernel_roofline("eig", 1.6, M, NB, NF, NB, peaks, "bf16x3")
    assert r["bound"] == "alu" and r["peak"] == bench.FP64_PEAK and r["traffic"] is None


def test_step_roofline():
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops_sustained": 1500.0}
    r = bench.step_roofline(30.0, M, NB, NF, NB, peaks, "bf16x3")
    B = bench.NT * M * 4 + NF * NB * M * 8
    assert r["bytes"] == B
    assert r["t_hbm_ms"] == pytest.approx(B / 6000e9 * 1e3, rel=1e-3)
    t_gemm = 3 * (8.0 * NF * NB * NB * M + 8.0 * NF * NB * NB * M) / 1500e12 * 1e3
    assert r["t_gemm_ms"] == pytest.approx(t_gemm, rel=1e-3)
    assert r["t_fft_ms"] == pytest.approx(2.5 * bench.NFFT * math.log2(bench.NFFT) * NB * M
                                          / (bench.FP32_PEAK * 1e12) * 1e3, rel=1e-3)
    assert r["frac"] == pytest.approx(max(r["t_hbm_ms"], r["t_gemm_ms"], r["t_fft_ms"]) / 30.0, abs=1e-4)


@pytest.mark.parametrize("phase", ["fft", "gram", "modes"])
def test_recorded_traffic_matches_the_bytes_moved(phase):
    # DRAM read + write from the ncu captures, scaled to the full grid, within
    # 5 % of the bytes this pipeline moves (algorithmic + Qhat overhead): no
    # kernel re-reads what it has read once
    r = bench.kernel_roofline(phase, 1.0, M, NB, NF, NB, {"hbm_gbs": 6000.0}, "bf16x3")
    if r["traffic"] is None:
        pytest.skip("no capture of the current kernel version")
    moved = r.get("bytes_per_launch", 0) + r["overhead_bytes"]
    assert abs(r["traffic"] / moved - 1.0) <= 0.05


class _FakeSampler(bench.ClockSampler):
    """The sampler's reduction over rows as nvidia-smi prints them."""

    def __init__(self, rows):
        super().__init__(0)
        self.rows = rows

        class _P:
            def terminate(self):
                pass

            def wait(self, timeout=None):
                return 0

        class _T:
            def join(self, timeout=None):
                pass

        self.proc, self.thread = _P(), _T()


def _row(sm, power_cap=False, thermal=False):
    a = "Active" if power_cap else "Not Active"
    t = "Active" if thermal else "Not Active"
    return ["0", str(sm), "2070", "900.0", "0x0", "Not Active", "Not Active", t, a]


def test_clock_sampler_filters_to_the_timed_region():
    rows = [(0.5, _row(1000, thermal=True)), (1.0, _row(2070)), (1.5, _row(2055, power_cap=True)),
            (2.0, _row(2070)), (3.5, _row(900, thermal=True))]
    s = _FakeSampler(rows).stop(0.9, 2.1)
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"] and s["window"] == "timed region"
    s = _FakeSampler(rows).stop(5.0, 6.0)            # nothing inside: every sample, and said so
    assert s["samples"] == 5 and "sw_thermal_slowdown" in s["reasons"] and s["window"].startswith("whole run")


def test_sample_columns_spread_and_deterministic():
    X = torch.arange(12 * 1000, dtype=torch.float32).reshape(12, 1000)
    cols, idx = bench.sample_columns(X, 7)
    assert cols.shape == (12, 7) and idx[0] == 0 and idx[-1] == 999
    assert np.all(np.diff(idx) > 0)
    np.testing.assert_array_equal(cols, X[:, torch.as_tensor(idx)].double().numpy())
    c2, i2 = bench.sample_columns(X, 7)
    np.testing.assert_array_equal(i2, idx)
