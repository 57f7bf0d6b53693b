"""Short versions of the long-run accuracy studies (paper_2211_02435_b300.accuracy):
FP32 stays within the FP32 tolerance of FP64 over tens of steps, pull and
AA agree bitwise, and the FP16 / BF16 forms stay within their rounding
bounds of FP64 on the Fourier-mode flow with the central-moment method."""
import numpy as np
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


def test_tgv_plateau_short():
    """The Table 3 experiment on a 64 x 64 x 1 lattice, where the vortex
    decays 16 times faster (kappa = 2 pi / 64), for 16 000 steps: the
    analytic E/E0 ends near 1e-41, so every form ends on its round-off
    plateau.  Zero-centered storage with delta-equilibria sits orders of
    magnitude below absolute storage (Sec. 5.1), and the absolute
    equilibrium on zero-centered storage keeps R-CM and R-K far below
    absolute storage."""
    B.build()
    res = A.tgv_plateau(n=64, steps=16_000, every=4_000)
    end = {k: v[-1] for k, v in res["runs"].items()}
    assert res["analytic"][-1] < 1e-38
    for k, v in res["runs"].items():
        assert v[0] == 1.0 and all(np.isfinite(v)), k
        assert v[-1] > 10 * res["analytic"][-1], k  # a plateau, not the analytic decay
    for m in ("SRT", "R-WO-MRT", "R-O-MRT", "R-CM"):
        assert end[f"{m}/absolute"] > 100 * end[f"{m}/zc_dfeq"], (m, end)
    for m in ("R-CM", "R-K"):
        assert end[f"{m}/absolute"] > 100 * end[f"{m}/zc_feq"], (m, end)
    # the deviation arithmetic of the absolute equilibrium does no worse
    # than Eq. 2.6 as written
    for m in ("R-WO-MRT", "R-O-MRT", "R-CM", "R-K"):
        assert end[f"{m}/zc_feq_deviation"] <= 10 * end[f"{m}/zc_feq"], (m, end)


def _table3():
    """Table 3 values from tests/golden/table3_tgv_plateaus.txt."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table3_tgv_plateaus.txt")
    cols = ("absolute", "zc_feq", "zc_dfeq")
    out = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        name, *vals = line.split()
        for c, v in zip(cols, vals):
            if v != "-":
                out[f"{name}/{c}"] = float(v)
    return out


# Printed cells of Table 3 that this library does not reproduce to 1.5
# decades, with the measured reason.  With every rate 1 each regularised
# method collides to the same equilibrium, so on absolute storage every
# method sits on the same floor (the FP64 quantisation of the stored f ~ w
# sets it, ~8e-27 here for all methods); the paper's spread of that column
# (1.7e-29 .. 1.9e-26) comes from the order of its generated arithmetic,
# which it does not print.  For the same reason R-WO-MRT with the absolute
# equilibrium on zero-centered storage lands on R-CM's level (4.0e-33)
# rather than 4.4e-31: with rates 1 the weighted basis never enters the
# regularised arithmetic.  These cells are held to 3 decades, and to the
# method-independent floor that explains them.
TABLE3_OFF = {"R-WO-MRT/absolute": 3.0, "R-CM/absolute": 3.0, "R-WO-MRT/zc_feq": 3.0}


@pytest.mark.slow
def test_tgv_plateau_table3_orders_of_magnitude():
    """The full Table 3 case (L = 256, 200 000 steps) for every method and
    storage form the paper prints: each of the 10 printed plateaus within
    1.5 decades of ours, except the three cells of TABLE3_OFF, held to 3
    decades and to the explanation given there (the absolute-storage floor is
    the same for every method; R-WO-MRT with f^eq equals R-CM with f^eq).
    The paper's ordering holds in every row: zero-centered storage with
    delta-equilibria lowest, absolute storage highest."""
    B.build()
    paper = _table3()
    assert len(paper) == 10
    res = A.tgv_plateau(n=256, steps=200_000, every=50_000,
                        methods=["SRT", "R-WO-MRT", "R-CM", "R-K"],
                        forms=["absolute", "zc_feq", "zc_dfeq"])
    ours = {k: v[-1] for k, v in res["runs"].items()}
    for key, ref in paper.items():
        band = TABLE3_OFF.get(key, 1.5)
        assert key in ours, key
        assert abs(np.log10(ours[key] / ref)) < band, (key, ours[key], ref)
    floor = ours["SRT/absolute"]
    for m in ("R-WO-MRT", "R-CM", "R-K"):
        assert abs(np.log10(ours[f"{m}/absolute"] / floor)) < 0.5, (m, ours)
    assert abs(np.log10(ours["R-WO-MRT/zc_feq"] / ours["R-CM/zc_feq"])) < 0.5, ours
    for m in ("SRT", "R-WO-MRT", "R-CM"):
        assert ours[f"{m}/absolute"] > 100 * ours[f"{m}/zc_dfeq"], (m, ours)
