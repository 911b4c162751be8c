"""Host logic of the hyperparameter loop (paper_2309_05435_gb300.hyper) with
the library calls replaced by a concave quadratic objective on the CPU: the
quasi-Newton ascent reaches the known maximiser from coupled, badly scaled
starting points, scales its steps to max_step, and adds a hyperprior's
gradient."""
import numpy as np
import pytest

from paper_2309_05435_gb300 import hyper


class _FakeLib:
    """grad log p = -A (theta - t_star) for an SPD A with strong coupling."""

    def __init__(self, A, t_star):
        self.A, self.t_star, self.theta, self.calls = A, t_star, None, 0

    def qsel_set_data(self, ctx, y):
        pass

    def qsel_set_theta(self, ctx, theta):
        self.theta = np.asarray(theta, dtype=float)

    def qsel_loglik_grad(self, ctx):
        self.calls += 1
        return -self.A @ (self.theta - self.t_star)


@pytest.fixture
def fake(monkeypatch):
    A = np.array([[40.0, 38.0, 1.0], [38.0, 40.0, 0.5], [1.0, 0.5, 5.0]])   # log kappa / log tau coupled
    lib = _FakeLib(A, np.array([-1.0, 1.5, 1.0]))
    monkeypatch.setattr(hyper, "qsel", lib)
    return lib


def test_reaches_the_maximiser(fake):
    theta, hist = hyper.optimize_theta(None, None, [0.5, -0.5, 3.0], iters=60)
    np.testing.assert_allclose(theta, fake.t_star, atol=1e-6)
    assert len(hist) < 30
    # one gradient per iteration after the three of the initial diagonal
    assert fake.calls == 1 + 3 + len(hist)


def test_steps_are_scaled_to_max_step(fake):
    _, hist = hyper.optimize_theta(None, None, [5.0, -5.0, 9.0], iters=5, max_step=0.25)
    for h in hist:
        assert np.max(np.abs(h["step"])) <= 0.25 + 1e-12


def test_hyperprior_gradient_is_added(fake):
    B = np.diag([2.0, 2.0, 2.0])
    prior_mode = np.array([0.0, 0.0, 0.0])
    theta, _ = hyper.optimize_theta(None, None, [0.0, 0.0, 0.0], iters=80,
                                    prior_grad=lambda t: -B @ (np.asarray(t) - prior_mode))
    # maximiser of -1/2 (t - t*)^T A (t - t*) - 1/2 t^T B t
    expected = np.linalg.solve(fake.A + B, fake.A @ fake.t_star)
    np.testing.assert_allclose(theta, expected, atol=1e-6)
