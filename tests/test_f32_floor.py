"""The FP32 floor of the force error, which sets the mixed-form tolerance.

tests/f32_model.py evaluates the pair terms from the fixed-point positions with
every operation rounded to a given type.  In FP64 it is the oracle (pins the
model's formula); in FP32 it is the smallest error any FP32 evaluation of the
terms can have.  The mixed-form tolerances (tests/tolerances.py) must sit above
that floor, and not far above it.
"""
import numpy as np
import pytest

from f32_model import forces_model, quantize
from helpers import rel_inf, rel_l2
from paper_1905_02521_gb300 import workloads as W
from tolerances import F32_INF, F32_L2


@pytest.fixture(scope="module")
def configs(oracle):
    s, pot = W.mgo_system(3, 300.0)
    xs = [s["pos"][0]]
    sim = oracle.Sim(s["pos"], s["vel"], s["types"], pot, s["box"], s["T"], s["gamma"], 1.0, seed=12345)
    sim.step(40, record=False)
    xs.append(sim.state()[0].reshape(-1, 3))
    return s, pot, xs


def test_model_in_fp64_is_the_oracle(oracle, configs):
    s, pot, xs = configs
    for x in xs:
        _, xq = quantize(x, s["box"])
        F = forces_model(xq, s["types"], s["box"], pot, dtype=np.float64)
        fo, _, _ = oracle.pair_forces(xq, s["types"], s["box"], pot)
        assert rel_inf(F, fo) < 1e-12


def test_mixed_tolerances_sit_above_the_fp32_floor(oracle, configs):
    s, pot, xs = configs
    for x in xs:
        F = forces_model(x, s["types"], s["box"], pot, dtype=np.float32)
        fo, _, _ = oracle.pair_forces(x, s["types"], s["box"], pot)
        l2, inf = rel_l2(F, fo), rel_inf(F, fo)
        print("FP32 floor: relative L2 %.2e, max / RMS %.2e" % (l2, inf))
        assert 2e-6 < l2 < F32_L2 / 1.5
        assert F32_INF / 4 < inf < F32_INF / 1.8
