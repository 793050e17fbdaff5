"""Pins for the FP64 reference of the learned warm start: central finite
differences of the loss against every analytic gradient, Gram-Schmidt
orthonormality, closed-form losses, and max-pool permutation invariance."""
import numpy as np
import pytest

from oracle import pointnet as pn


def _problem(seed=0, B=2, P=32):
    rng = np.random.default_rng(seed)
    src = rng.uniform(-1, 1, (B, P, 3))
    dst = rng.uniform(-1, 1, (B, P, 3))
    Rg = np.stack([np.linalg.qr(rng.normal(size=(3, 3)))[0] for _ in range(B)])
    Rg *= np.sign(np.linalg.det(Rg))[:, None, None]
    tg = rng.normal(0, 0.3, (B, 3))
    params = pn.init_params(seed)
    for k in params:  # make the head non-trivial
        params[k] = params[k] + rng.normal(0, 0.05, params[k].shape)
    return params, src, dst, Rg, tg


def test_parameter_count():
    assert pn.n_params() == 192 + 64 + 8192 + 128 + 32768 + 256 + 131072 + 256 + 2304 + 9


def test_gradients_match_central_differences():
    params, src, dst, Rg, tg = _problem()
    out = pn.forward(params, src, dst, Rg, tg)
    g = pn.backward(params, out, src, Rg, tg)
    rng = np.random.default_rng(1)
    h = 1e-6
    for k in pn.ORDER:
        flat = params[k].ravel()
        idx = rng.choice(flat.size, size=min(12, flat.size), replace=False)
        for i in idx:
            pp = {kk: vv.copy() for kk, vv in params.items()}
            pm = {kk: vv.copy() for kk, vv in params.items()}
            pp[k].ravel()[i] += h
            pm[k].ravel()[i] -= h
            op = pn.forward(pp, src, dst, Rg, tg)
            om = pn.forward(pm, src, dst, Rg, tg)
            # skip probes that flip a max-pool argmax (the loss is only
            # piecewise smooth there)
            if not (np.array_equal(op["arg_src"], om["arg_src"]) and
                    np.array_equal(op["arg_dst"], om["arg_dst"])):
                continue
            fd = (op["loss"] - om["loss"]) / (2 * h)
            an = g[k].ravel()[i]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), f"{k}[{i}]: fd {fd} analytic {an}"


def test_gram_schmidt_is_a_rotation():
    rng = np.random.default_rng(2)
    a1 = rng.normal(size=(100, 3))
    a2 = rng.normal(size=(100, 3))
    R = pn.gram_schmidt(a1, a2)
    np.testing.assert_allclose(np.einsum("bji,bjk->bik", R, R), np.tile(np.eye(3), (100, 1, 1)),
                               atol=1e-12)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-12)
    # columns 1 and 2 span the same plane as a1, a2; column 1 is a1's direction
    np.testing.assert_allclose(R[:, :, 0], a1 / np.linalg.norm(a1, axis=1, keepdims=True),
                               atol=1e-12)
    np.testing.assert_allclose(pn.gram_schmidt(np.eye(3)[None, 0], np.eye(3)[None, 1])[0],
                               np.eye(3), atol=0)


def test_loss_closed_forms():
    rng = np.random.default_rng(3)
    P = rng.uniform(-1, 1, (4, 50, 3))
    R = np.tile(np.eye(3), (4, 1, 1))
    t = rng.normal(size=(4, 3))
    L, per, _ = pn.loss(R, t, P, R, np.zeros((4, 3)))
    np.testing.assert_allclose(per, (t ** 2).sum(1), rtol=1e-13)  # pure translation
    L0, per0, _ = pn.loss(R, t, P, R, t)
    assert L0 == 0.0


def test_initial_head_outputs_identity():
    params = pn.init_params(0)
    params["W5"][:] = 0
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (1, 64, 3))
    out = pn.forward(params, X, X, np.eye(3)[None], np.zeros((1, 3)))
    np.testing.assert_allclose(out["R"][0], np.eye(3), atol=1e-15)
    assert np.all(out["t"] == 0)


def test_max_pool_is_permutation_invariant():
    params, src, dst, Rg, tg = _problem(5, B=1, P=64)
    f, arg, _ = pn.encode(params, src)
    perm = np.random.default_rng(6).permutation(64)
    fp, argp, _ = pn.encode(params, src[:, perm])
    np.testing.assert_allclose(fp, f, rtol=1e-15)
    live = f > 0  # channels that are zero everywhere pick row 0 either way
    assert live.sum() > 100
    assert np.array_equal(perm[argp][live], arg[live])


def test_bf16_rounding_matches_definition():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -3.1415926, 0.0, 1.0 + 2 ** -7 + 2 ** -9],
                 np.float32)
    r = pn.bf16_round(x)
    # bfloat16 keeps 8 significand bits: spacing 2^-7 at 1.0; exact halfway
    # cases go to the even neighbour
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -6
    assert r[5] == 1.0 + 2 ** -7
    assert abs(r[3] + 3.140625) < 1e-12 and r[4] == 0.0
