"""Host-side arithmetic of bench.py (no GPU): the executed tensor FLOPs its
roofline divides by a launch's time, counted here independently as the MMAs
the tensor kernels issue, the FP32 form's algorithmic FLOP count, and the
bookkeeping that drops an ncu record once the kernel source has changed."""
import importlib.util
import math
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _Workload:
    def __init__(self, grid_n, T=1000, A=256, K=5, n_pol=2):
        self.grid_n, self.T, self.A, self.K, self.n_pol = list(grid_n), T, A, K, n_pol


MMA_FLOP = 2 * 128 * 128 * 16          # one tcgen05 MMA of 128 x 128 x 16


def _mmas_per_channel_sample(n, terms):
    """MMAs the tensor kernels issue for one channel and sample: a stage is 8
    k-blocks of `terms` MMAs (6 k-blocks for side 96's 48-point DFTs).  Pair
    kernel at sides 128 and 96: two CTAs (pixel-class columns), each a row
    stage and two column stages; side 64: one CTA, a row and a column stage;
    other sides: two stages per pixel class."""
    kb = 6 if n == 96 else 8
    if n in (128, 96):
        return 2 * 3 * kb * terms
    if n == 64:
        return 2 * kb * terms
    return (n // 64) ** 2 * 2 * kb * terms


@pytest.mark.parametrize("grid_n", [[128] * 64, [96] * 64, [64] * 64, [64] * 64 + [96] * 64 + [128] * 64, [256] * 3])
@pytest.mark.parametrize("form,terms", [("tc_split_fp16", 3), ("tc_split_bf16", 3), ("tc_fp16", 1)])
def test_tensor_roofline_counts_the_kernels_mmas(bench, grid_n, form, terms):
    wl = _Workload(grid_n)
    r = bench.tensor_roofline(wl, form, 1.0, {"bf16_tflops": 1000.0, "bf16_tflops_sustained": 500.0})
    want = sum(_mmas_per_channel_sample(n, terms) for n in grid_n) * wl.T * MMA_FLOP
    assert r["executed_flops_per_launch"] == pytest.approx(want, rel=1e-12)
    # FLOP over 1 ms against the peaks given
    assert r["achieved"] == pytest.approx(want / 1e-3 / 1e12, rel=1e-12)
    assert r["frac"] == pytest.approx(r["achieved"] / 1000.0, rel=1e-12)
    assert r["frac_of_sustained"] == pytest.approx(r["achieved"] / 500.0, rel=1e-12)


def test_lwa_executed_flops_match_the_recorded_figure(bench):
    # 64 channels x 1000 samples x 144 MMAs: the figure the profiles quote (4.83e12)
    r = bench.tensor_roofline(_Workload([128] * 64), "tc_split_fp16", 3.346, {"bf16_tflops": 1911.3})
    assert r["executed_flops_per_launch"] == 64 * 1000 * 144 * MMA_FLOP == 4831838208000
    assert r["frac"] == pytest.approx(4831838208000 / 3.346e-3 / 1e12 / 1911.3, rel=1e-12)


def test_fp32_flops_per_spectrum_closed_form(bench):
    # gridding 8 A K^2 + row-pruned radix-2 FFTs 5 N log2 N (N/2 + N) + products 8 N^2
    assert bench.fp32_flops_per_spectrum(1, 1, 2) == 8 + 5 * 2 * 1 * 3 + 32
    A, K, N = 256, 5, 128
    assert bench.fp32_flops_per_spectrum(A, K, N) == pytest.approx(
        8 * A * K * K + 5 * N * math.log2(N) * 1.5 * N + 8 * N * N, rel=1e-15)


def test_ncu_records_are_dropped_when_the_kernel_source_changes(bench):
    h = bench.kernel_source_hash("tc_split_fp16")
    assert h == bench.kernel_source_hash("tc_split_fp16") and len(h) == 16
    assert h != bench.kernel_source_hash("fp32")
    table = {("lwa", "tc_split_fp16"): (1.0e8, h), ("lwa", "fp32"): (2.0e8, "0" * 16)}
    assert bench.ncu_record(table, "lwa", "tc_split_fp16") == 1.0e8
    assert bench.ncu_record(table, "lwa", "fp32") is None          # recorded on other source
    assert bench.ncu_record(table, "dense", "fp32") is None        # never recorded
