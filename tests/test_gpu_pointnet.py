"""Learned warm start: libcil's PointNet kernels (cil_pointnet_*) against the
FP64 reference with the same BF16 rounding of W2, W3, A1, A2.

Bars: features and transforms within BF16 tolerance (relative 2e-2 on the
max-pooled features, where a neighbouring BF16 rounding of one activation moves
a product by ~2^-8); per-parameter-block gradients within relative 2e-2 and
cosine similarity > 0.999; identical results on repeated calls; the loss falls
when training; and a short training already beats identity on held-out pairs.
"""
import numpy as np
import pytest
import torch

import paper_1807_00399_gb300 as cil
from oracle import pointnet as opn
from paper_1807_00399_gb300 import learned, synth

pytestmark = pytest.mark.gpu


def _setup(B=4, P=512, seed=0):
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    clouds, T = learned.make_batch(gen, B, P)
    params = opn.init_params(seed)
    rng = np.random.default_rng(seed)
    for k in params:
        params[k] = params[k] + rng.normal(0, 0.05, params[k].shape)
    net = cil.PointNet(B, P, params=opn.flatten(params).astype(np.float32))
    # the reference sees the same float32 parameters
    p32 = opn.unflatten(opn.flatten(params).astype(np.float32).astype(np.float64))
    return net, clouds, T, p32


def _oracle(p32, clouds, T):
    c = clouds.cpu().numpy().astype(np.float64)
    Tg = T.cpu().numpy().reshape(-1, 4, 4)
    out = opn.forward(p32, c[:, 0], c[:, 1], Tg[:, :3, :3], Tg[:, :3, 3], bf16=True)
    return out, c, Tg


def test_forward_matches_reference():
    net, clouds, T, p32 = _setup()
    B = clouds.shape[0]
    feat = torch.empty((B, 512), dtype=torch.float32, device="cuda")
    Tp = net.forward(clouds, feat_out=feat)
    torch.cuda.synchronize()
    out, _, _ = _oracle(p32, clouds, T)
    f_ref = np.concatenate([out["f_src"], out["f_dst"]], 1)
    f = feat.cpu().numpy()
    scale = np.abs(f_ref).max()
    assert np.abs(f - f_ref).max() <= 2e-2 * scale
    Tp = Tp.cpu().numpy().reshape(-1, 4, 4)
    R = Tp[:, :3, :3]
    np.testing.assert_allclose(np.einsum("bji,bjk->bik", R, R), np.tile(np.eye(3), (B, 1, 1)),
                               atol=1e-5)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-5)
    np.testing.assert_allclose(R, out["R"], atol=2e-2)
    np.testing.assert_allclose(Tp[:, :3, 3], out["t"], atol=2e-2 * max(1.0, np.abs(out["t"]).max()))
    net.close()


def test_gradients_match_reference():
    net, clouds, T, p32 = _setup(B=4, P=512, seed=1)
    grad = torch.empty(net.n_params, dtype=torch.float32, device="cuda")
    loss, _ = net.backward(clouds, T, grad_out=grad)
    torch.cuda.synchronize()
    out, c, Tg = _oracle(p32, clouds, T)
    g_ref = opn.backward(p32, out, c[:, 0], Tg[:, :3, :3], Tg[:, :3, 3])
    np.testing.assert_allclose(loss.cpu().numpy(), out["per_pair"], rtol=2e-2)
    g = opn.unflatten(grad.cpu().numpy().astype(np.float64))
    for k in opn.ORDER:
        a, b = g[k].ravel(), g_ref[k].ravel()
        nb = np.linalg.norm(b)
        if nb == 0:
            assert np.linalg.norm(a) == 0
            continue
        rel = np.linalg.norm(a - b) / nb
        cos = a @ b / (np.linalg.norm(a) * nb)
        assert rel <= 2e-2 and cos > 0.999, f"{k}: rel {rel:.3g} cos {cos:.6f}"
    net.close()


def test_repeatable():
    net, clouds, T, _ = _setup(B=3, P=256, seed=2)
    g1 = torch.empty(net.n_params, dtype=torch.float32, device="cuda")
    g2 = torch.empty_like(g1)
    net.backward(clouds, T, grad_out=g1)
    net.backward(clouds, T, grad_out=g2)
    torch.cuda.synchronize()
    assert torch.equal(g1, g2)
    net.close()


def test_training_reduces_loss():
    net = cil.PointNet(64, 1024, params=opn.flatten(opn.init_params(3)).astype(np.float32))
    hist, _ = learned.train(net, 150, B=64, lr=1e-3, seed=3, log_every=10)
    first = np.mean([h[1] for h in hist[:2]])
    last = np.mean([h[1] for h in hist[-2:]])
    assert last < 0.5 * first, f"loss {first:.4f} -> {last:.4f}"
    net.close()


def test_short_training_beats_identity_on_held_out_pairs():
    net = cil.PointNet(256, 4096, params=opn.flatten(opn.init_params(4)).astype(np.float32))
    learned.train(net, 400, B=128, lr=1e-3, seed=4)
    pairs, s_sub, d_sub = synth.warm_start_pairs(12345, 32, n=10_000)
    res = learned.evaluate(net, pairs, s_sub, d_sub, iters=30, max_corr_dist=0.1, runs=2)
    assert res["warm_start_rot_err_deg_median"] < res["identity_rot_err_deg_median"]
    assert res["success_learned_fallback"] >= res["success_identity"]
    assert res["success_learned_fallback"] > res["success_identity"] or \
        res["success_identity"] == 1.0
    net.close()


@pytest.mark.gpu
def test_committed_checkpoint_beats_identity_start():
    """The shipped warm-start weights (trained by the library's own kernels on
    200k generated pairs) against plain ICP from identity on held-out pairs."""
    net = cil.PointNet(64, 4096)
    learned.load_checkpoint(net, learned.CHECKPOINT)
    pairs, s_sub, d_sub = synth.warm_start_pairs(4242, 64, n=10_000)
    res = learned.evaluate(net, pairs, s_sub, d_sub, iters=30, max_corr_dist=0.1, runs=2)
    net.close()
    assert res["warm_start_rot_err_deg_median"] < 0.5 * res["identity_rot_err_deg_median"]
    assert res["success_learned_before_fallback"] > res["success_identity"]
    assert res["success_learned_fallback"] >= res["success_learned_before_fallback"]
    assert res["success_learned_fallback"] >= res["success_identity"]
