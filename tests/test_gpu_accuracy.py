"""Short versions of the long-run accuracy studies (paper_2211_02435_b300.accuracy):
FP32 stays within the FP32 tolerance of FP64 over tens of steps, pull and
AA agree bitwise, and the FP16 / BF16 forms stay within their rounding
bounds of FP64 on the Fourier-mode flow with the central-moment method."""
import pytest

from paper_2211_02435_b300 import accuracy as A
from paper_2211_02435_b300 import build as B

pytestmark = pytest.mark.gpu


def test_fp32_vs_fp64_short():
    B.build()
    res = A.fp32_vs_fp64(n=32, steps=40, every=20)
    assert res["pull_aa_bitwise_equal_at_end"]
    for row in res["rows"]:
        assert row["u_rel_linf"] < 1e-5


def test_half_storage_short():
    B.build()
    res = A.half_storage(n=32, steps=200, every=100)
    last = res["rows"][-1]
    assert last["f32"]["u_rel_linf"] < 1e-5
    # per-step rounding 2^-11 (FP16) / 2^-8 (BF16) of |df|, relaxed over 200 steps
    assert last["f16_delta"]["u_rel_linf"] < 2e-2
    assert last["bf16_delta"]["u_rel_linf"] < 1.5e-1
