"""The host part of the multi-tau reuse (Sec. 3.3): plsqr_projected_solve must solve the projected
problem (3.6), min_y || [B_k; sqrt(tau) I] y - beta_1 e_1 ||, for a lower-bidiagonal B_k with
alpha on the diagonal and beta below it; its residual history is the minimum of that problem for
each number of columns.  Pinned against a dense least-squares solve of the same problem (no GPU)."""
import numpy as np
import pytest


def _lstsq(alpha, beta, tau, k):
    B = np.zeros((k + 1, k))
    for j in range(k):
        B[j, j] = alpha[j]
        B[j + 1, j] = beta[j + 1]
    A = np.vstack([B, np.sqrt(tau) * np.eye(k)])
    rhs = np.zeros(2 * k + 1)
    rhs[0] = beta[0]
    y, *_ = np.linalg.lstsq(A, rhs, rcond=None)
    return y, np.linalg.norm(A @ y - rhs)


@pytest.mark.parametrize("tau", [0.0, 1e-3, 0.1, 10.0])
@pytest.mark.parametrize("k", [1, 2, 7, 40])
def test_projected_solve_matches_dense_least_squares(tau, k):
    from paper_1308_6634_gb300 import plsqr
    rng = np.random.default_rng(k)
    alpha = rng.uniform(0.2, 2.0, k + 1)
    beta = rng.uniform(0.05, 1.5, k + 1)
    y, rb = plsqr.projected_solve(alpha, beta, tau)
    y_ref, r_ref = _lstsq(alpha, beta, tau, k)
    assert np.linalg.norm(y - y_ref) <= 1e-10 * np.linalg.norm(y_ref)
    for i in range(1, k + 1):
        assert abs(rb[i - 1] - _lstsq(alpha, beta, tau, i)[1]) <= 1e-10 * beta[0]
    assert abs(rb[-1] - r_ref) <= 1e-10 * beta[0]


def test_projected_solve_undamped_is_the_plain_least_squares_solution():
    """tau = 0: y solves min ||B_k y - beta_1 e_1||, and a square-consistent case gives B y = rhs."""
    from paper_1308_6634_gb300 import plsqr
    alpha = np.array([2.0, 1.0, 3.0])
    beta = np.array([4.0, 0.0, 0.5])  # beta_2 = 0: the first column decouples, y_1 = beta_1 / alpha_1
    y, rb = plsqr.projected_solve(alpha, beta, 0.0)
    assert abs(y[0] - 2.0) < 1e-15 and abs(y[1]) < 1e-15
    assert rb[0] < 1e-15 and rb[1] < 1e-15


def test_projected_solve_rejects_bad_input():
    from paper_1308_6634_gb300 import plsqr
    with pytest.raises(ValueError):
        plsqr.projected_solve([1.0], [1.0], 0.0)
    with pytest.raises(RuntimeError):
        plsqr.projected_solve([1.0, 1.0], [1.0, 1.0], -1.0)
