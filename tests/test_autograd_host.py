"""Host wiring of MobiusAction (paper_1206_5214_gb300/autograd.py) on the CPU.

The library calls are replaced by a fake with a known action,
S(U, b5, c5) = b5 sum|U|^2 + c5^2 |phi|^2 (with per-slice coefficients
S = sum_s b5(s) sum|U|^2 + sum_s c5(s)^2 |phi|^2), whose force follows torch's
complex convention G = dS/dRe U + i dS/dIm U = 2 b5 U. The test checks what the
Function itself does: the upstream gradient scales both outputs, the outputs
come back in argument order, a gradient nobody asked for is None, every handle
is destroyed (also when the force call fails), and torch.autograd.gradcheck
agrees with the wiring. The force itself is checked on the GPU against the
oracle and against differences of the action.
"""
import numpy as np
import pytest
import torch

import paper_1206_5214_gb300.autograd as ag


class FakeLib:
    def __init__(self):
        self.live = 0
        self.fail = False

    def create(self, dims, Ls, M5, b5, c5, mf):
        self.live += 1
        return {"b5": b5, "c5": c5, "mu": 0.0}

    def set_s(self, h, b5s, c5s):
        h["b5s"], h["c5s"] = np.array(b5s, float), np.array(c5s, float)

    def set_mu(self, h, mu):
        h["mu"] = mu
        self.mu_seen = mu

    def destroy(self, h):
        self.live -= 1

    def load_gauge(self, h, U):
        h["U"] = U.clone()

    def force(self, h, G, phi, tol, inner_prec):
        if self.fail:
            raise RuntimeError("planted failure")
        U = h["U"]
        nU, nphi = float((U.abs() ** 2).sum()), float((phi.abs() ** 2).sum())
        if "b5s" in h:
            b5s, c5s = h["b5s"], h["c5s"]
            if G is not None:
                G.copy_(2.0 * b5s.sum() * U)
            return b5s.sum() * nU + (c5s ** 2).sum() * nphi, np.full(len(b5s), nU), 2.0 * c5s * nphi, 0, 1
        b5, c5 = h["b5"], h["c5"]
        if G is not None:
            G.copy_(2.0 * b5 * U)
        return b5 * nU + c5 * c5 * nphi, nU, 2.0 * c5 * nphi, 0, 1


@pytest.fixture
def fake(monkeypatch):
    f = FakeLib()
    monkeypatch.setattr(ag, "mdwf_create", f.create)
    monkeypatch.setattr(ag, "mdwf_destroy", f.destroy)
    monkeypatch.setattr(ag, "mdwf_load_gauge", f.load_gauge)
    monkeypatch.setattr(ag, "mdwf_force", f.force)
    monkeypatch.setattr(ag, "mdwf_set_s_coefficients", f.set_s)
    monkeypatch.setattr(ag, "mdwf_set_chemical_potential", f.set_mu)
    return f


def _inputs(seed=3):
    g = torch.Generator().manual_seed(seed)
    U = torch.randn(2, 2, 2, 2, 4, 3, 3, dtype=torch.complex128, generator=g)
    phi = torch.randn(4, 8, 4, 3, dtype=torch.complex128, generator=g)
    return U, phi


def test_gradients_scaled_by_upstream(fake):
    U, phi = _inputs()
    U.requires_grad_(True)
    b5c5 = torch.tensor([1.5, 0.5], dtype=torch.float64, requires_grad=True)
    S = ag.mobius_action(U, b5c5, phi, (2, 2, 2, 2), 4, 1.8, 0.01)
    expect = 1.5 * float((U.detach().abs() ** 2).sum()) + 0.25 * float((phi.abs() ** 2).sum())
    assert float(S.detach()) == pytest.approx(expect, rel=1e-14)
    (3.0 * S).backward()
    assert torch.allclose(U.grad, 3.0 * 2.0 * 1.5 * U.detach(), rtol=1e-14, atol=0)
    gb = np.array([float((U.detach().abs() ** 2).sum()), 2 * 0.5 * float((phi.abs() ** 2).sum())]) * 3.0
    assert np.allclose(b5c5.grad.numpy(), gb, rtol=1e-14)
    assert fake.live == 0


def test_only_requested_gradients(fake):
    U, phi = _inputs()
    b5c5 = torch.tensor([1.5, 0.5], dtype=torch.float64, requires_grad=True)
    S = ag.mobius_action(U, b5c5, phi, (2, 2, 2, 2), 4, 1.8, 0.01)
    S.backward()
    assert U.grad is None and b5c5.grad is not None
    assert fake.live == 0


def test_handles_freed_on_failure(fake):
    U, phi = _inputs()
    b5c5 = torch.tensor([1.5, 0.5], dtype=torch.float64)
    fake.fail = True
    with pytest.raises(RuntimeError, match="planted"):
        ag.mobius_action(U, b5c5, phi, (2, 2, 2, 2), 4, 1.8, 0.01)
    assert fake.live == 0


def test_gradcheck_through_the_wiring(fake):
    U, phi = _inputs(7)
    U = (0.3 * U).requires_grad_(True)
    b5c5 = torch.tensor([1.2, 0.4], dtype=torch.float64, requires_grad=True)
    f = lambda U_, bc: ag.mobius_action(U_, bc, phi, (2, 2, 2, 2), 4, 1.8, 0.01)
    assert torch.autograd.gradcheck(f, (U, b5c5), eps=1e-6, atol=1e-6, rtol=1e-6)
    assert fake.live == 0


def test_per_slice_coefficients_and_mu(fake):
    U, phi = _inputs(5)
    U.requires_grad_(True)
    bc = torch.tensor([[1.2, 1.9, 1.4, 2.3], [0.1, 0.8, 0.2, 1.0]], dtype=torch.float64, requires_grad=True)
    S = ag.mobius_action(U, bc, phi, (2, 2, 2, 2), 4, 1.8, 0.01, mu=0.1)
    assert fake.mu_seen == 0.1
    nU, nphi = float((U.detach().abs() ** 2).sum()), float((phi.abs() ** 2).sum())
    assert float(S.detach()) == pytest.approx(6.8 * nU + 1.69 * nphi, rel=1e-13)
    (2.0 * S).backward()
    assert bc.grad.shape == (2, 4)
    expect = 2.0 * np.stack([np.full(4, nU), 2.0 * bc.detach().numpy()[1] * nphi])
    assert np.allclose(bc.grad.numpy(), expect, rtol=1e-13)
    assert torch.allclose(U.grad, 2.0 * 2.0 * 6.8 * U.detach(), rtol=1e-13, atol=0)
    assert fake.live == 0


def test_per_slice_gradcheck(fake):
    U, phi = _inputs(9)
    U = (0.3 * U).requires_grad_(True)
    bc = torch.tensor([[1.2, 1.9, 1.4, 2.3], [0.1, 0.8, 0.2, 1.0]], dtype=torch.float64, requires_grad=True)
    f = lambda U_, b: ag.mobius_action(U_, b, phi, (2, 2, 2, 2), 4, 1.8, 0.01)
    assert torch.autograd.gradcheck(f, (U, bc), eps=1e-6, atol=1e-6, rtol=1e-6)
    assert fake.live == 0


def test_coefficient_shape_refused(fake):
    U, phi = _inputs()
    with pytest.raises(ValueError, match="shape"):
        ag.mobius_action(U, torch.zeros(2, 3, dtype=torch.float64), phi, (2, 2, 2, 2), 4, 1.8, 0.01)
    assert fake.live == 0
