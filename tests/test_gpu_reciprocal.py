"""The FP64 pivot reciprocal of the block factorization (Newton's method
from a single-precision seed) against the IEEE quotient 1/d: within one unit
in the last place over a wide range of magnitudes and both signs, exact at
powers of two, and the plain quotient outside the seed's exponent range."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_pivot_reciprocal_within_one_ulp(cuda):
    import torch
    import paper_2510_13333_b300 as P
    rng = np.random.default_rng(0)
    d = rng.standard_normal(1 << 20) * 10.0 ** rng.uniform(-40, 40, 1 << 20)
    d = np.concatenate([d, 2.0 ** np.arange(-60, 61), -(2.0 ** np.arange(-60, 61)),
                        [1e-300, -1e-300, 3e-200, 1e200, 1.9999999999999998, 1.0000000000000002]])
    got = P.scopf_pivot_reciprocal(torch.tensor(d, device="cuda")).cpu().numpy()
    ref = 1.0 / d
    ulp = np.abs(got - ref) / np.spacing(np.abs(ref))
    assert ulp.max() <= 1.0, (ulp.max(), d[np.argmax(ulp)])
    pw = np.abs(np.log2(np.abs(d)) - np.round(np.log2(np.abs(d)))) == 0
    assert np.array_equal(got[pw], ref[pw])
