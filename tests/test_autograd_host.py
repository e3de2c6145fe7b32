"""Host logic of the autograd wrapper on the CPU, with a fake library: the
forward keeps a tape only when the handle's path has one and it fits the HBM
budget, hands the backward the same tape (or none, so that it recomputes),
returns [J][N] jets for J = the mask's row count, and the backward's weight
gradient becomes W.grad."""
import types

import pytest

from paper_2409_14248_gb300 import capi

torch = pytest.importorskip("torch")
from paper_2409_14248_gb300.autograd import _Jets  # noqa: E402


class FakeLibrary:
    def __init__(self, tape_floats):
        self.tape_floats, self.fwd_tape, self.bwd_tape = tape_floats, "unset", "unset"

    def hrkan_tape_floats(self, h, N, mask):
        return self.tape_floats

    def hrkan_forward_jets(self, h, W, x, N, mask, jets, tape):
        self.fwd_tape = tape
        jets.fill_(1.0)

    def hrkan_backward(self, h, W, x, N, mask, tape, g, dW):
        self.bwd_tape = tape
        dW.copy_(g.sum() * torch.ones_like(dW))


@pytest.fixture
def fake(monkeypatch):
    def install(tape_floats):
        lib = FakeLibrary(tape_floats)
        for name in ("hrkan_tape_floats", "hrkan_forward_jets", "hrkan_backward"):
            monkeypatch.setattr(capi, name, getattr(lib, name))
        return lib
    return install


@pytest.mark.parametrize("tape_floats,budget,kept", [
    (1000, 0, True),          # no cap: keep the tape
    (1000, 4000, True),       # exactly fits (4 bytes per float)
    (1000, 3999, False),      # one byte short: recompute
    (0, 0, False),            # the fused path has no tape
])
def test_tape_is_kept_only_when_it_exists_and_fits(fake, tape_floats, budget, kept):
    lib = fake(tape_floats)
    net = types.SimpleNamespace(handle="h", hbm_budget_bytes=budget)
    W = torch.zeros(7, requires_grad=True)
    x = torch.zeros(2, 5)
    jets = _Jets.apply(W, x, net, 0x8F)                 # u, u_x, u_t, u_xx, u_xy: 5 rows
    assert jets.shape == (5, 5)
    (2.0 * jets).sum().backward()
    if kept:
        assert lib.fwd_tape is not None and lib.fwd_tape.numel() == tape_floats
        assert lib.bwd_tape is lib.fwd_tape or lib.bwd_tape.data_ptr() == lib.fwd_tape.data_ptr()
    else:
        assert lib.fwd_tape is None and lib.bwd_tape is None
    assert torch.equal(W.grad, torch.full((7,), 2.0 * 25))
