"""Host-side checks of FP32 facts the superposition kernel relies on, in the
same IEEE round-to-nearest single precision the GPU uses.

* The pass walk divides slot numbers by the slot stride K1 (1 <= K1 <= 257)
  as floor((n + 1/2) * RN(1/K1)) for n <= 1024 instead of an integer
  division: exact, because the product's relative error (below 2^-23) stays
  under the 1 / (2 K1) that separates n / K1 + 1 / (2 K1) from the next
  integer.
* The fixed-point scale 2^sh and its inverse (-100 <= sh <= 30) are built from
  their exponent field; they are the normal powers of two.
"""
import numpy as np


def test_reciprocal_floor_division_is_exact():
    n = np.arange(0, 1025, dtype=np.int64)
    half = np.float32(0.5)
    for k1 in range(1, 258):
        rk = np.float32(1.0) / np.float32(k1)  # correctly rounded, as __frcp_rn
        q = np.floor((n.astype(np.float32) + half) * rk).astype(np.int64)
        assert np.array_equal(q, n // k1), k1


def test_exponent_built_powers_of_two():
    for sh in range(-100, 31):
        up = np.array([(sh + 127) << 23], dtype=np.int32).view(np.float32)[0]
        down = np.array([(127 - sh) << 23], dtype=np.int32).view(np.float32)[0]
        assert up == np.float32(np.ldexp(1.0, sh))
        assert down == np.float32(np.ldexp(1.0, -sh))
