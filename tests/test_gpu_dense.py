"""GPU dense LDL^T of the border (Schur complement) block against the
LAPACK solution and the eigenvalue inertia, on symmetric quasi-definite
matrices shaped like the first-stage coupling block (ragged sizes included)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def sqd(n1, n2, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n1, n1))
    A = A @ A.T / n1 + np.eye(n1)
    C = rng.standard_normal((n2, n2))
    C = C @ C.T / n2 + 0.1 * np.eye(n2)
    B = rng.standard_normal((n2, n1))
    return np.block([[A, B.T], [B, -C]])


@pytest.mark.parametrize("n1,n2", [(1, 0), (20, 17), (120, 60), (400, 320)])
def test_dense_ldlt_solve(cuda, n1, n2):
    import torch
    import paper_2510_13333_b300 as P
    K = sqd(n1, n2, n1 + n2)
    n = n1 + n2
    b = np.random.default_rng(1).standard_normal(n)
    S = torch.tensor(K.T.copy(), device="cuda")   # column-major
    x, inertia = P.scopf_dense_ldlt_solve(S, torch.tensor(b, device="cuda"))
    x_ref = np.linalg.solve(K, b)
    err = np.abs(x.cpu().numpy() - x_ref).max() / np.abs(x_ref).max()
    assert err <= 1e-10, err
    ev = np.linalg.eigvalsh(K)
    assert inertia == (int((ev > 0).sum()), int((ev < 0).sum()), 0)
