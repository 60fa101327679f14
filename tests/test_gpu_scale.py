"""The scale-up workload: the synthetic 2000-bus network (mean degree 2.7,
360 generators) with 128 contingencies (100 line, 28 generator, uneven
switch sets), mixed-precision batched factorization with the FP64 fallback.
A full NCL solve is certified by the oracle at the returned point."""
import pytest

from tests import helpers as H
from tests.test_gpu_fullsize import certify

pytestmark = pytest.mark.gpu


def test_scale_up_solution_certified_by_oracle(cuda):
    import paper_2510_13333_b300 as P
    inst = H.instance(4)
    lib = P.SCOPF(inst, precision=P.PREC_MIXED)
    s = lib.sizes
    assert s.n_blocks == 129 and s.n_border == 720
    r = lib.ncl_solve()
    assert r["call_status"] == 0, r
    out = certify(inst, lib, r)
    print(f"2000-bus x 128: objective {r['objective']:.9f}, {r['inner_iters']} IPM iterations, "
          f"{r['fp64_fallbacks']} FP64 fallbacks, certificate {out}")
