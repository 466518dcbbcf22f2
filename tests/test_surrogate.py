"""End-to-end surrogate on solver data (small): the network trains on focal
patches produced by the one-shot solver, beats the trivial mean-field
predictor on held-out seeds, and is faster per focal patch than the solver."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_surrogate_learns_solver_patches_and_is_faster(lib):
    import torch
    from paper_2010_00409_gb300 import surrogate as S
    patch = 24
    phys, prm, tgt, t_solver = S.make_dataset(48, seed=1, N=128, patch=patch)
    scale = tgt.abs().max()
    tgt = tgt / scale
    net = lib.Fno(len(S.PARAM_NAMES), width=16, layers=3, patch=patch, modes=6, hidden=32, out_channels=3,
                  max_batch=8, seed=0)
    hist = S.train(net, prm[:40], tgt[:40], steps=300, batch=8, lr=2e-3, log_every=50)
    assert hist[-1][1] < 0.5 * hist[0][1], hist
    errs, t_net = S.evaluate(net, prm[40:], tgt[40:], batch=8)
    # the method without the network for unseen parameters: at best the training-set mean field
    mean = tgt[:40].mean(0, keepdim=True)
    base = ((mean - tgt[40:]).flatten(1).norm(dim=1) / tgt[40:].flatten(1).norm(dim=1)).cpu().numpy()
    print("surrogate rel L2 %.3f (mean-field %.3f); s/patch surrogate %.2e solver %.2e" %
          (errs.mean(), base.mean(), t_net, t_solver))
    assert errs.mean() < base.mean()
    assert t_net < t_solver
    net.close()
