"""Tolerances of the GPU parity tests, in one place.

FP64 form: 1e-12 norm-wise (max |diff| / RMS).

FP32 (mixed) form, forces compared with the oracle on the GPU's own
configuration: the criterion is the relative L2 error of the force vector,
||F - F_oracle|| / ||F_oracle|| <= 1e-5 ("1e-5 relative").  A second guard
bounds the largest component error relative to the RMS force at 4e-5: single
FP32 pair terms of ~10 eV/A cancel to net forces of ~0.5 eV/A in the crystal,
and a correctly rounded FP32 evaluation of the pair terms (tests/f32_model.py)
already reaches 1.7e-5 in that norm on 216-ion MgO configurations; the guard
sits 2.3x above that floor (tests/test_f32_floor.py pins both numbers).
"""
F64_TOL = 1e-12
F32_L2 = 1e-5
F32_INF = 4e-5
