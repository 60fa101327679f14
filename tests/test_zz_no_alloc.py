"""The no-allocation dense border solve (scopf_dense_ldlt_solve_noalloc),
for callers that cannot allocate device memory during a call, must give
the same result as the allocating entry point scopf_dense_ldlt_solve.

Kept in a file of its own that pytest collects last, so that a run that
stops at the first failure has already run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _sqd(n1, n2, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n1, n1))
    A = A @ A.T / n1 + np.eye(n1)
    C = rng.standard_normal((n2, n2))
    C = C @ C.T / n2 + 0.1 * np.eye(n2)
    B = rng.standard_normal((n2, n1))
    return np.block([[A, B.T], [B, -C]])


def test_noalloc_matches_allocating_entry_point(cuda):
    import torch
    import paper_2510_13333_b300 as P
    # two calls in a row (different sizes: the second must not see stale
    # contents of the shared scratch), each compared with the regular call
    # the largest order the static scratch takes (768: the panel kernel's
    # shared memory is then close to its opt-in), two ordinary orders, and
    # a 1 x 1 block
    for n1, n2, seed in ((512, 256, 2), (120, 60, 3), (90, 47, 4), (1, 0, 5)):
        K = _sqd(n1, n2, seed) if n2 else np.array([[2.5]])
        n = n1 + n2
        S = torch.tensor(K.T.copy(), device="cuda")
        b = torch.tensor(np.random.default_rng(seed).standard_normal(n), device="cuda")
        x_ref, in_ref = P.scopf_dense_ldlt_solve(S, b)
        x, inertia, status = P.scopf_dense_ldlt_solve_noalloc(S, b)
        torch.cuda.synchronize()
        assert status == 0
        assert inertia == in_ref
        err = (x - x_ref).abs().max().item() / x_ref.abs().max().item()
        assert err <= 1e-10, err


def test_noalloc_rejects_oversize(cuda):
    import torch
    import paper_2510_13333_b300 as P
    n = 769
    S = torch.eye(n, dtype=torch.float64, device="cuda")
    b = torch.ones(n, dtype=torch.float64, device="cuda")
    _, _, status = P.scopf_dense_ldlt_solve_noalloc(S, b)
    assert status == P.ScopfError("x", -1).status == -1
