"""Lloyd's stopping rule in driver.lloyd (Section 1: a fixed count, convergence, or a small
decrease), checked on the host against a fake binding that scripts each iteration's two costs;
no GPU, no kernels."""
import pytest
import torch

from paper_1502_04265_gb300 import driver


class FakeBinding:
    """Records the calls the driver makes and writes scripted (cost_old, cost_new) pairs."""

    def __init__(self, costs):
        self.costs = costs
        self.assigns = 0
        self.updates = 0

    def kmeans_row_norms(self, X, ctx=None):
        return (X * X).sum(1)

    def kmeans_quantize(self, X, dtype, ctx=None):
        return X.clone(), None

    def kmeans_seed_pp(self, X, k, u, w=None, ctx=None):
        return torch.arange(k), X[:k].clone()

    def kmeans_assign(self, X, C, labels=None, **kw):
        self.assigns += 1
        labels.zero_()
        return labels

    def kmeans_update(self, X, labels, C, w=None, C_new=None, cost_old=None, cost_new=None, ctx=None):
        old, new = self.costs[self.updates]
        self.updates += 1
        cost_old.fill_(old)
        cost_new.fill_(new)
        C_new.copy_(C)


COSTS = [(100.0, 60.0), (60.0, 50.0), (50.0, 49.99), (49.99, 49.99), (49.99, 49.99), (49.99, 49.99)]


def run(monkeypatch, iters, tol=None):
    fake = FakeBinding(COSTS)
    monkeypatch.setattr(driver, "B", fake)
    X = torch.arange(40, dtype=torch.float32).reshape(10, 4)
    out = driver.lloyd(X, 3, iters, torch.zeros(3, dtype=torch.float64), return_trace=True, tol=tol)
    return fake, out


def test_fixed_count_runs_every_iteration(monkeypatch):
    fake, out = run(monkeypatch, 6)
    assert fake.assigns == fake.updates == 6 and out["iterations"] == 6
    assert out["trace"].shape == (6, 2)
    assert out["converged_at"] == 3  # the first update that left the cost unchanged


def test_tol_zero_stops_at_convergence(monkeypatch):
    fake, out = run(monkeypatch, 6, tol=0.0)
    assert fake.assigns == 4 and out["iterations"] == 4
    assert out["trace"].shape == (4, 2) and out["converged_at"] == 3


def test_small_relative_decrease_stops_early(monkeypatch):
    # (50 - 49.99) / 50 = 2e-4 <= 1e-3 at the third iteration; 10 / 60 > 1e-3 before it
    fake, out = run(monkeypatch, 6, tol=1e-3)
    assert fake.assigns == 3 and out["iterations"] == 3 and out["converged_at"] is None


def test_iteration_cap_wins_over_tol(monkeypatch):
    fake, out = run(monkeypatch, 2, tol=0.0)
    assert fake.assigns == 2 and out["iterations"] == 2 and out["converged_at"] is None


@pytest.mark.parametrize("tol", [-1e-3, float("nan")])
def test_bad_tol_is_refused(monkeypatch, tol):
    with pytest.raises(ValueError):
        run(monkeypatch, 3, tol=tol)
