"""The bound behind FP16 storage of the explicit local inverses: rounding
S = A^{-1} (A SPD with unit diagonal, as the scaled local matrices) to IEEE
half precision gives S + dS with every eigenvalue of (S + dS) A within
1 -+ (2^-11 ||S||_inf + n 2^-25) ||A||_inf.  Checked on random matrices of
several conditions, including ones where the bound is nearly tight."""
import numpy as np
import pytest
import scipy.linalg as sla


def _unit_diag_spd(n, cond, rng):
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    w = np.geomspace(1.0, 1.0 / cond, n)
    A = (Q * w) @ Q.T
    d = 1.0 / np.sqrt(np.diag(A))
    return d[:, None] * A * d[None, :]


@pytest.mark.parametrize("n,cond", [(40, 10.0), (120, 1e2), (200, 1e3), (64, 5e3)])
def test_fp16_rounding_of_the_inverse_stays_within_the_bound(n, cond):
    rng = np.random.default_rng(n)
    A = _unit_diag_spd(n, cond, rng)
    S = np.linalg.inv(A)
    S = 0.5 * (S + S.T)
    S16 = S.astype(np.float16).astype(np.float64)
    assert np.all(np.isfinite(S16))
    bound = (np.ldexp(np.abs(S).sum(axis=1).max(), -11) + n * np.ldexp(1.0, -25)) * np.abs(A).sum(axis=1).max()
    lam = sla.eigh(S16, np.linalg.inv(A), eigvals_only=True)  # eig of S16 A, symmetric form
    assert np.all(np.abs(lam - 1.0) <= bound * (1 + 1e-9)), (np.abs(lam - 1).max(), bound)


def test_the_bound_admits_the_well_conditioned_case_and_rejects_a_poor_one():
    rng = np.random.default_rng(7)
    def bound(A):
        S = np.linalg.inv(A)
        return (np.ldexp(np.abs(S).sum(axis=1).max(), -11) + A.shape[0] * np.ldexp(1.0, -25)) * \
            np.abs(A).sum(axis=1).max()
    assert bound(_unit_diag_spd(100, 20.0, rng)) <= 0.25
    assert bound(_unit_diag_spd(100, 1e5, rng)) > 0.25
