"""Training step (Sec. 3.3): the Eq. 8 objective with anisotropic TV, the
optimiser update, and the captured full training iteration, against the
plain definitions in oracle/train_ref.py and the FP64 renderer."""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import train_ref as TR
from paper_2205_14330_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import __graft_entry__ as g
    g.build()
    from paper_2205_14330_gb300 import pbr
    r = pbr.Renderer(0)
    yield pbr, r
    r.close()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("kind,lam", [("l2", 0.01), ("l1", 0.3), ("l2", 0.0)])
def test_loss_tv_matches_definition(env, kind, lam):
    import torch
    pbr, _ = env
    cams = [scenes.camera((0, 0, 2), 37, 21), scenes.camera((0, 1, 2), 16, 40)]
    n = sum(c["width"] * c["height"] for c in cams)
    rng = np.random.default_rng(3)
    pred = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    tgt = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    loss, grad = pbr.image_loss_tv(torch.from_numpy(pred).cuda(), torch.from_numpy(tgt).cuda(),
                                   cams, lam, kind)
    ref_loss, ref_grad = TR.batch_loss_and_grad(pred, tgt, [(c["width"], c["height"]) for c in cams],
                                                lam, kind)
    assert abs(loss.item() - ref_loss) <= 1e-6 * ref_loss
    assert np.abs(grad.cpu().numpy() - ref_grad).max() <= 1e-5


@pytest.mark.parametrize("kind", ["sgd", "adam"])
def test_optimizer_matches_definition(env, kind):
    import torch
    pbr, _ = env
    rng = np.random.default_rng(4)
    p = rng.normal(size=1000).astype(np.float32)
    pd, md, vd = (torch.from_numpy(p).cuda(), torch.zeros(1000, device="cuda"),
                  torch.zeros(1000, device="cuda"))
    pr, mr, vr = p.astype(np.float64), np.zeros(1000), np.zeros(1000)
    for t in range(1, 4):
        g = rng.normal(size=1000).astype(np.float32)
        pbr.optimizer_step(pd, torch.from_numpy(g).cuda(), md, vd, lr=3e-3, step=t, kind=kind)
        if kind == "adam":
            pr, mr, vr = TR.adam_step(pr, g, mr, vr, t, 3e-3)
        else:
            pr = TR.sgd_step(pr, g, 3e-3)
    assert np.abs(pd.cpu().numpy() - pr).max() <= 1e-6


def test_training_iteration_graph(env):
    """Phase TRAIN = forward + Eq. 8 objective + backward + update; one SGD
    step moves the parameters by -lr times the oracle's gradient."""
    import torch
    pbr, R = env
    sc = scenes.tiny(n=1500, size=64)
    cams = sc["cams"] + [scenes.camera((1.5, 0.5, 2.0), 48, 40)]
    tgt_img, _, _ = O.render(sc["target_pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"],
                             cams)
    scene = pbr.Scene(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"])
    target = torch.from_numpy(tgt_img.astype(np.float32)).cuda()
    G = pbr.Graph(R, [scene], cams, target=target)
    lr_pos, lr_sh = 1e-3, 2e-3
    G.set_optimizer(kind="sgd", lr_pos=lr_pos, lr_sh=lr_sh, lambda_tv=0.01)
    p0, h0 = scene.pos.clone(), scene.sh.clone()
    G.launch(pbr.Graph.TRAIN)
    ok, _, _ = G.check()
    assert ok
    # oracle: image, Eq. 8 gradient of it, adjoint
    img, _, _ = O.render(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"], cams)
    loss_ref, g_img = TR.batch_loss_and_grad(img, tgt_img, [(c["width"], c["height"]) for c in cams],
                                             0.01, "l2")
    dpos, dsh, _ = O.backward(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"], cams,
                              g_img)
    step_pos = (scene.pos - p0).cpu().numpy()
    step_sh = (scene.sh - h0).cpu().numpy()
    e = (_rel(step_pos, -lr_pos * dpos), _rel(step_sh, -lr_sh * dsh))
    print(f"training step vs oracle: rel L2 pos {e[0]:.2e} sh {e[1]:.2e}; loss "
          f"{G.loss.item():.6f} vs {loss_ref:.6f}")
    assert max(e) <= 1e-3
    assert abs(G.loss.item() - loss_ref) <= 1e-4 * loss_ref
    # Adam: several replays lower the objective; the rate can be decayed in place
    G.set_optimizer(kind="adam", lr_pos=2e-4, lr_sh=3e-3, lambda_tv=0.01)
    losses = []
    for it in range(12):
        G.set_lr(2e-4 * 0.93 ** it, 3e-3 * 0.93 ** it)
        G.launch(pbr.Graph.TRAIN)
        losses.append(G.loss.item())
    assert G.check()[0]
    assert losses[-1] < losses[0]
    G.close()
