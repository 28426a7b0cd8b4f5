"""Differentiation form: PBRRenderFn (torch.autograd.Function) calls the
library's hand-written backward.  Gradients of a torch loss through it are
compared with the FP64 oracle's adjoint of the same loss."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2205_14330_gb300 import scenes

pytestmark = pytest.mark.gpu


def test_autograd_function_matches_oracle():
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_2205_14330_gb300 import pbr
    sc = scenes.tiny(n=2048, size=96)
    dev = "cuda"
    pos = torch.tensor(sc["pos"], device=dev, requires_grad=True)
    sh = torch.tensor(sc["sh"], device=dev, requires_grad=True)
    op = torch.tensor(sc["opacity"], device=dev, requires_grad=True)
    rad = torch.tensor(sc["radius"], device=dev)
    img = pbr.render(pos, sh, op, rad, sc["deg"], sc["cams"])
    w = torch.linspace(-1.0, 1.0, img.numel(), device=dev).view_as(img)
    loss = (img * w).sum() + 0.5 * (img ** 2).sum()
    loss.backward()
    # the same loss on the oracle image: dL/dI = w + I
    ref, _, _ = O.render(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"], sc["cams"])
    gI = w.double().cpu().numpy() + ref
    dpos, dsh, dop = O.backward(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"],
                                sc["cams"], gI)

    def rel(a, b):
        return float(np.linalg.norm(a.detach().double().cpu().numpy() - b) / np.linalg.norm(b))

    assert float(np.abs(img.detach().cpu().numpy() - ref).max()) <= 1e-4
    e = (rel(pos.grad, dpos), rel(sh.grad, dsh), rel(op.grad, dop))
    print(f"autograd grads rel L2 vs oracle: {e}")
    assert max(e) <= 1e-3
    # a second forward/backward through the same function object works
    pos.grad = None
    pbr.render(pos, sh, op, rad, sc["deg"], sc["cams"]).sum().backward()
    assert pos.grad is not None and torch.isfinite(pos.grad).all()
