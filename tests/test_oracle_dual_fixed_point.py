"""The property the exact early stop of the dual iteration rests on (the dual
APG of the P-metric prox, Sec. III-B): a dual step is a fixed function of
(R, Q), the momentum factor multiplying only the change of Q, so once the
iteration stops changing it never changes again.  Checked on the oracle's
own dual APG in float64: with a prox weight that saturates the dual ball,
the results after n steps stop depending on n, bit for bit, from some small n
on; with a weight that does not, they keep changing (the check has teeth)."""
import numpy as np
import pytest

import oracle
from workloads import gaussian_probe_like, phantom


def _orthonormal(N, ell, seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((N, ell)))
    return q.T.copy()


def _pc(kind, n):
    if kind == "identity":
        return oracle.nystrom.Identity()
    # P = I + U diag(d) U^T with every column but the last active
    return oracle.nystrom.Precond(_orthonormal(n * n, 8, 3), np.linspace(3.0, 1.0, 8), 0.0, False)


def _first_fixed(s, reg, lb, P, n_max):
    """The least n with prox_dual(n) = prox_dual(n + 1) = prox_dual(n + 2)
    bitwise (x and Q), or None."""
    runs = [oracle.prox.prox_dual(s, reg, lb, P, n) for n in range(n_max + 3)]
    for n in range(n_max + 1):
        if all(np.array_equal(runs[n][k], runs[n + d][k]) for d in (1, 2) for k in (0, 1)):
            return n, runs
    return None, runs


@pytest.mark.parametrize("reg", ["tv", "hs"])
@pytest.mark.parametrize("kind", ["identity", "lowrank"])
def test_saturated_dual_iteration_is_stationary(reg, kind):
    n = 24
    s = phantom(n, 6, 3, "mixed") + 0.05 * gaussian_probe_like((n, n), 9)
    P = _pc(kind, n)
    n0, runs = _first_fixed(s, reg, 1e-7, P, 15)
    assert n0 is not None, "the saturated dual iteration did not become stationary within 15 steps"
    # once stationary, any number of further steps gives the same bits
    x40, Q40 = oracle.prox.prox_dual(s, reg, 1e-7, P, 40)
    assert np.array_equal(runs[n0][0], x40) and np.array_equal(runs[n0][1], Q40)


@pytest.mark.parametrize("reg", ["tv", "hs"])
def test_unsaturated_dual_iteration_keeps_moving(reg):
    n = 24
    s = phantom(n, 6, 3, "mixed") + 0.05 * gaussian_probe_like((n, n), 9)
    n0, _ = _first_fixed(s, reg, 0.05, oracle.nystrom.Identity(), 12)
    assert n0 is None
