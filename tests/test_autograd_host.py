"""Host logic of the adjoint autograd Function, on the CPU with the library's entry points replaced by fakes
that count handles: every handle made by a forward pass is destroyed whether or not backward runs, a second
backward is refused, and a description of another precision is refused before any handle is made."""
import gc

import numpy as np
import pytest
import torch

from paper_1504_06123_gb300 import autograd as AG
from paper_1504_06123_gb300 import lbve as L


class FakeLib:
    def __init__(self):
        self.made = 0
        self.destroyed = 0
        self.backwards = 0

    def create_adjoint(self, d, rho, every):
        self.made += 1
        return object()

    def step(self, h, n, stream=None):
        pass

    def fields(self, h, mask, dst=None, stream=None):
        return np.arange(5 * 8, dtype=np.float64)      # [u (2 x 8) | sigma (3 x 8)] of an 8-node channel

    def backward(self, h, du, ds, stream=None):
        self.backwards += 1
        return np.ones(4)

    def destroy(self, h):
        self.destroyed += 1


@pytest.fixture
def fake(monkeypatch):
    f = FakeLib()
    monkeypatch.setattr(L, "lbve_create_adjoint", f.create_adjoint)
    monkeypatch.setattr(L, "lbve_step", f.step)
    monkeypatch.setattr(L, "lbve_fields", f.fields)
    monkeypatch.setattr(L, "lbve_backward", f.backward)
    monkeypatch.setattr(L, "lbve_destroy", f.destroy)
    live0 = AG.AdjointRun.live
    yield f
    gc.collect()
    assert AG.AdjointRun.live == live0


def desc(prec=L.LBVE_F64):
    return L.make_desc(nx=2, ny=4, C=8, B=2, precision=L.LBVE_F32 if prec == L.LBVE_S16 else prec, hist_storage=prec)


def theta(requires_grad=True):
    return torch.tensor([0.01, 50.0, 0.1, 1e-5], dtype=torch.float64, requires_grad=requires_grad)


def test_backward_frees_the_handle(fake):
    th = theta()
    u, s = AG.LBVEChannelAdjoint.apply(th, desc(), 10)
    assert fake.made == 1 and fake.destroyed == 0
    (u.sum() + s.sum()).backward()
    assert fake.backwards == 1 and fake.destroyed == 1
    assert np.array_equal(th.grad.numpy(), np.ones(4))


def test_no_grad_forward_frees_the_handle(fake):
    with torch.no_grad():
        u, s = AG.LBVEChannelAdjoint.apply(theta(), desc(), 10)
    del u, s
    gc.collect()
    assert fake.made == 1 and fake.destroyed == 1


def test_unused_outputs_free_the_handle(fake):
    u, s = AG.LBVEChannelAdjoint.apply(theta(), desc(), 10)
    assert fake.destroyed == 0
    del u, s
    gc.collect()
    assert fake.made == 1 and fake.destroyed == 1 and fake.backwards == 0


def test_theta_without_grad_frees_at_once(fake):
    u, s = AG.LBVEChannelAdjoint.apply(theta(requires_grad=False), desc(), 10)
    assert fake.made == 1 and fake.destroyed == 1


def test_second_backward_is_refused(fake):
    u, s = AG.LBVEChannelAdjoint.apply(theta(), desc(), 10)
    loss = u.sum() + s.sum()
    loss.backward(retain_graph=True)
    with pytest.raises(RuntimeError, match="second time"):
        loss.backward()
    assert fake.backwards == 1 and fake.destroyed == 1


def test_other_storage_is_refused(fake):
    with pytest.raises(ValueError, match="FP64 or FP32"):
        AG.LBVEChannelAdjoint.apply(theta(), desc(L.LBVE_S16), 10)
    f = desc()
    f.hist_form = L.LBVE_FORM_F
    with pytest.raises(ValueError, match="form-P"):
        AG.LBVEChannelAdjoint.apply(theta(), f, 10)
    assert fake.made == 0
    AG.LBVEChannelAdjoint.apply(theta(), desc(L.LBVE_F32), 10)     # FP32 storage is differentiated
    assert fake.made == 1
