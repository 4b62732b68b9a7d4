"""The bench's roofline objects on the CPU, from fake profiling timers.

bench.kernel_rooflines derives one object per instrumented kernel (k_ace_basis and
k_ace_adjoint against the FP32 ALU peak, k_eam_force against HBM) from the step's
CUDA-event phase totals, the ACE pair/atom counters and the EAM prefix total; the
bench reports the one with the most time as `roofline`.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class FakeCtx:
    def __init__(self, walked, total):
        self.walked, self.total = walked, total

    def neighbor_total(self, which):
        return {0: self.total, 2: self.walked}[which]


PEAKS = {"fp32_tflops": 74.5, "fp32_sm_mhz": 2000.0, "tf32_mma_tflops": 303.0, "tf32_sm_mhz": 2000.0, "sms": 152,
         "fp32_derived_tflops": 80.5}


def prof(basis_ms, adj_ms, force_ms, calls=10, pairs=3.0e8, atoms=2.4e6, mma=0):
    return {"phases": {"ace_basis": (basis_ms, calls), "ace_adjoint": (adj_ms, calls),
                       "eam_force": (force_ms, calls)},
            "ace_pairs": pairs, "ace_atoms": atoms, "ace_mma": mma}


def test_objects_follow_the_flop_and_byte_counts():
    n = 4_000_000
    r = bench.kernel_rooflines(FakeCtx(215_000_000, 342_000_000), prof(12.0, 11.0, 10.0), n, 6785.9, "test", PEAKS)
    b = r["k_ace_basis"]
    flops = bench.BASIS_FLOP_PER_PAIR * 3.0e8 + bench.BASIS_FLOP_PER_ATOM * 2.4e6
    assert b["achieved"] == pytest.approx(flops / 12.0e-3 / 1e12)
    assert b["frac"] == pytest.approx(b["achieved"] / PEAKS["fp32_tflops"])
    assert b["ms_per_launch"] == pytest.approx(1.2) and b["bound"] == "alu"
    a = r["k_ace_adjoint"]
    assert a["achieved"] == pytest.approx((bench.ADJ_FLOP_PER_PAIR * 3.0e8 + bench.ADJ_FLOP_PER_ATOM * 2.4e6)
                                          / 11.0e-3 / 1e12)
    e = r["k_eam_force"]
    want = bench.EAM_FORCE_BYTES_PER_ENTRY * 215_000_000 + bench.EAM_FORCE_BYTES_PER_ATOM * n
    assert e["algorithmic_bytes_per_launch"] == want
    assert e["achieved"] == pytest.approx(want / 1.0e-3 / 1e9)
    assert e["frac"] == pytest.approx(e["achieved"] / 6785.9) and e["bound"] == "hbm"
    assert e["row_entries_walked"] == 215_000_000 and e["row_entries_total"] == 342_000_000


@pytest.mark.parametrize("times,dominant", [((12.0, 11.0, 10.0), "k_ace_basis"),
                                            ((9.0, 11.0, 10.0), "k_ace_adjoint"),
                                            ((9.0, 8.0, 10.0), "k_eam_force")])
def test_the_dominant_kernel_is_the_one_with_the_most_time(times, dominant):
    r = bench.kernel_rooflines(FakeCtx(1, 2), prof(*times), 100, 6785.9, "test", PEAKS)
    assert bench.dominant_kernel(r) == dominant


def test_no_time_gives_zero_not_an_error():
    r = bench.kernel_rooflines(FakeCtx(0, 0), prof(0.0, 0.0, 0.0, calls=0), 100, 6785.9, "test", PEAKS)
    assert all(v["achieved"] == 0.0 for v in r.values())


def test_tensor_pipe_use_of_the_basis_kernel():
    """The basis kernel's tensor object counts 2*16*8*8 flops per issued MMA tile against
    the measured TF32 MMA peak; it is absent when no tile was counted (FP64)."""
    r = bench.kernel_rooflines(FakeCtx(1, 2), prof(12.0, 11.0, 10.0, mma=3.0e8), 100, 6785.9, "test", PEAKS)
    t = r["k_ace_basis"]["tensor"]
    assert t["achieved"] == pytest.approx(2048 * 3.0e8 / 12.0e-3 / 1e12)
    assert t["frac"] == pytest.approx(t["achieved"] / 303.0) and t["mma_tiles_per_launch"] == 3.0e7
    r0 = bench.kernel_rooflines(FakeCtx(1, 2), prof(12.0, 11.0, 10.0), 100, 6785.9, "test", PEAKS)
    assert "tensor" not in r0["k_ace_basis"]


def test_curve_interpolation_at_equal_cost_and_error():
    """The selector/CSP comparison reads one detector's curve at the other's precise fraction
    (or error) by linear interpolation along the curve; outside its range there is no value."""
    k = "force_err_rms_meV_A_label_positive"
    pts = [{"precise_fraction": p, k: e} for p, e in ((0.04, 5.0), (0.06, 3.0), (0.08, 1.0))]
    assert bench.curve_at(pts, "precise_fraction", 0.05, k) == pytest.approx(4.0)
    assert bench.curve_at(pts, k, 2.0, "precise_fraction") == pytest.approx(0.07)
    assert bench.curve_at(pts, "precise_fraction", 0.10, k) is None
