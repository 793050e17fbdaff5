"""Independent pins of the FP64 PointNet reference's FORWARD (encoder, head,
rotation, loss), which the finite-difference test cannot pin (that one shows
only that the backward is the derivative of whatever the forward computes).

The network is restated here from its specification in words -- a shared
per-point MLP 3 -> 64 -> 128 -> 256 with ReLU after each layer, a global
max-pool over the points, the source and target features concatenated in that
order, an MLP 512 -> 256 (ReLU) -> 9, a 6-D rotation turned into R by
Gram-Schmidt and t from the last three outputs, and the mean squared
displacement of the source points as the loss -- with library building
blocks that share nothing with the reference's numpy code:

  * torch.nn.Linear / torch.nn.ReLU / torch.amax in float64 for the layers;
  * the rotation from a QR factorisation (torch.linalg.qr) of the 3x2 matrix
    [a1 a2] with its column signs fixed so that R's diagonal is positive, the
    third column from torch.linalg.cross;
  * gradients from torch.autograd;
  * bfloat16 rounding from torch's own float -> bfloat16 conversion;
  * a small closed-form case evaluated with plain Python loops.

Mistakes planted in the reference on the CPU (ReLU dropped, the bias added
after the ReLU, the features concatenated target-first, max-pool replaced by a
mean) must each fail the comparison, so the comparison is sensitive to them.
"""
import math

import numpy as np
import pytest
import torch

from oracle import pointnet as pn

TOL = 1e-12


def _params(seed):
    rng = np.random.default_rng(seed)
    p = pn.init_params(seed)
    for k in p:  # a non-trivial head and non-zero biases
        p[k] = p[k] + rng.normal(0, 0.05, p[k].shape)
    return p


def _clouds(seed, B=3, P=40):
    rng = np.random.default_rng(100 + seed)
    src = rng.uniform(-1, 1, (B, P, 3))
    dst = rng.uniform(-1, 1, (B, P, 3))
    Rg = np.stack([np.linalg.qr(rng.normal(size=(3, 3)))[0] for _ in range(B)])
    Rg *= np.sign(np.linalg.det(Rg))[:, None, None]
    tg = rng.normal(0, 0.3, (B, 3))
    return src, dst, Rg, tg


class TorchNet(torch.nn.Module):
    """The network written with torch modules (float64)."""

    def __init__(self, p, bf16=False):
        super().__init__()
        self.bf16 = bf16
        self.enc = torch.nn.ModuleList(
            [torch.nn.Linear(3, 64), torch.nn.Linear(64, 128), torch.nn.Linear(128, 256)])
        self.fc1 = torch.nn.Linear(512, 256)
        self.fc2 = torch.nn.Linear(256, 9)
        self.relu = torch.nn.ReLU()
        mods = list(self.enc) + [self.fc1, self.fc2]
        for m, (w, b) in zip(mods, (("W1", "b1"), ("W2", "b2"), ("W3", "b3"), ("W4", "b4"),
                                    ("W5", "b5"))):
            m.weight = torch.nn.Parameter(torch.tensor(p[w], dtype=torch.float64))
            m.bias = torch.nn.Parameter(torch.tensor(p[b], dtype=torch.float64))

    @staticmethod
    def _bf(x):
        return x.to(torch.bfloat16).to(torch.float64)

    def features(self, X):
        a = self.relu(self.enc[0](X))
        for layer in self.enc[1:]:
            if self.bf16:  # operands of the BF16 products rounded, accumulation in FP64
                a = torch.nn.functional.linear(self._bf(a), self._bf(layer.weight), layer.bias)
            else:
                a = layer(a)
            a = self.relu(a)
        return torch.amax(a, dim=1)  # global max-pool over the points

    def forward(self, src, dst):
        h = torch.cat([self.features(src), self.features(dst)], dim=-1)  # source first
        o = self.fc2(self.relu(self.fc1(h)))
        A = torch.stack([o[:, 0:3], o[:, 3:6]], dim=-1)  # [B, 3, 2]
        Q, Rr = torch.linalg.qr(A)
        s = torch.sign(torch.diagonal(Rr, dim1=-2, dim2=-1))
        Q = Q * s[:, None, :]
        b3 = torch.linalg.cross(Q[..., 0], Q[..., 1], dim=-1)
        R = torch.cat([Q, b3[..., None]], dim=-1)
        return R, o[:, 6:9], h


def _torch_loss(R, t, src, Rg, tg):
    moved = torch.einsum("bij,bpj->bpi", R, src) + t[:, None, :]
    want = torch.einsum("bij,bpj->bpi", Rg, src) + tg[:, None, :]
    return ((moved - want) ** 2).sum(-1).mean(-1)


def _compare(p, src, dst, Rg, tg, bf16=False):
    """Largest absolute differences between the reference and the torch
    restatement: features, R, t, per-pair loss."""
    out = pn.forward(p, src, dst, Rg, tg, bf16=bf16)
    net = TorchNet(p, bf16)
    with torch.no_grad():
        R, t, h = net(torch.tensor(src), torch.tensor(dst))
        per = _torch_loss(R, t, torch.tensor(src), torch.tensor(Rg), torch.tensor(tg))
    f = np.concatenate([out["f_src"], out["f_dst"]], 1)
    return {"feat": np.abs(f - h.numpy()).max() / max(1.0, np.abs(f).max()),
            "R": np.abs(out["R"] - R.numpy()).max(),
            "t": np.abs(out["t"] - t.numpy()).max() / max(1.0, np.abs(out["t"]).max()),
            "loss": np.abs(out["per_pair"] - per.numpy()).max() / max(1.0, per.abs().max().item())}


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("bf16", [False, True])
def test_forward_equals_torch_restatement(seed, bf16):
    p = _params(seed)
    src, dst, Rg, tg = _clouds(seed)
    d = _compare(p, src, dst, Rg, tg, bf16)
    for k, v in d.items():
        assert v <= TOL, f"{k}: {v:.3g}"


def test_gradients_equal_autograd():
    p = _params(7)
    src, dst, Rg, tg = _clouds(7, B=2, P=24)
    out = pn.forward(p, src, dst, Rg, tg)
    g = pn.backward(p, out, src, Rg, tg)
    net = TorchNet(p)
    R, t, _ = net(torch.tensor(src), torch.tensor(dst))
    L = _torch_loss(R, t, torch.tensor(src), torch.tensor(Rg), torch.tensor(tg)).mean()
    L.backward()
    mods = list(net.enc) + [net.fc1, net.fc2]
    names = (("W1", "b1"), ("W2", "b2"), ("W3", "b3"), ("W4", "b4"), ("W5", "b5"))
    for m, (w, b) in zip(mods, names):
        for name, ref in ((w, m.weight.grad), (b, m.bias.grad)):
            r = ref.numpy()
            err = np.abs(g[name] - r).max() / max(1e-300, np.abs(r).max())
            assert err <= 1e-9, f"{name}: rel {err:.3g}"


def test_bf16_rounding_equals_torch_conversion():
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-3, 1000),
                        rng.uniform(-50, 50, 1000)]).astype(np.float32)
    # exact halfway cases between neighbouring bfloat16 values
    base = rng.integers(0, 1 << 15, 200).astype(np.uint32) << 16
    halves = (base | 0x8000).view(np.float32)
    x = np.concatenate([x, halves, -halves])
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(pn.bf16_round(x), want)


def test_closed_form_embedding_network():
    """Layers 2-3 embed layer 1's output unchanged (identity blocks, zero
    bias), so each feature is max over the points of relu(w_j . x + b_j);
    the head passes the 12 first features of each cloud through (ReLU of
    non-negative values) and o = A4 W5^T + b5 picks chosen entries.  Every
    expected value below is computed with scalar Python loops."""
    p = {k: np.zeros(v) for k, v in pn.SHAPES.items()}
    rng = np.random.default_rng(21)
    p["W1"] = rng.normal(0, 1, (64, 3))
    p["b1"] = rng.normal(0, 0.2, 64)
    p["W2"][:64, :64] = np.eye(64)
    p["W3"][:128, :128] = np.eye(128)
    p["W4"][np.arange(12), np.arange(12)] = 1.0           # f_src[0:12]
    p["W4"][12 + np.arange(12), 256 + np.arange(12)] = 1.0  # f_dst[0:12]
    # o[0:3] = (f_s0 + 1, f_s1, f_s2), o[3:6] = (f_d0, f_d1 + 1, f_d2), t = (f_s3, f_d3, 0.5)
    p["W5"][0, 0] = p["W5"][1, 1] = p["W5"][2, 2] = 1.0
    p["W5"][3, 12] = p["W5"][4, 13] = p["W5"][5, 14] = 1.0
    p["W5"][6, 3] = p["W5"][7, 15] = 1.0
    p["b5"][:] = [1.0, 0, 0, 0, 1.0, 0, 0, 0, 0.5]
    src, dst, Rg, tg = _clouds(3, B=1, P=9)
    out = pn.forward(p, src, dst, Rg, tg)

    def feat(cloud, j):
        best = 0.0  # ReLU outputs are >= 0, so the max over points is >= 0
        for x in cloud:
            z = p["b1"][j] + sum(p["W1"][j][a] * x[a] for a in range(3))
            best = max(best, max(z, 0.0))
        return best

    fs = [feat(src[0], j) for j in range(64)]
    fd = [feat(dst[0], j) for j in range(64)]
    assert np.allclose(out["f_src"][0, :64], fs, rtol=0, atol=1e-13)
    assert np.allclose(out["f_dst"][0, :64], fd, rtol=0, atol=1e-13)
    assert np.all(out["f_src"][0, 64:] == 0) and np.all(out["f_dst"][0, 64:] == 0)
    a1 = [fs[0] + 1.0, fs[1], fs[2]]
    a2 = [fd[0], fd[1] + 1.0, fd[2]]
    n1 = math.sqrt(sum(v * v for v in a1))
    b1 = [v / n1 for v in a1]
    d = sum(b1[i] * a2[i] for i in range(3))
    u2 = [a2[i] - d * b1[i] for i in range(3)]
    n2 = math.sqrt(sum(v * v for v in u2))
    b2 = [v / n2 for v in u2]
    b3 = [b1[1] * b2[2] - b1[2] * b2[1], b1[2] * b2[0] - b1[0] * b2[2],
          b1[0] * b2[1] - b1[1] * b2[0]]
    R = [[b1[i], b2[i], b3[i]] for i in range(3)]  # columns b1, b2, b3
    assert np.allclose(out["R"][0], R, rtol=0, atol=1e-13)
    assert np.allclose(out["t"][0], [fs[3], fd[3], 0.5], rtol=0, atol=1e-13)
    tot = 0.0
    for x in src[0]:
        for i in range(3):
            moved = sum(R[i][j] * x[j] for j in range(3)) + out["t"][0][i]
            want = sum(Rg[0][i][j] * x[j] for j in range(3)) + tg[0][i]
            tot += (moved - want) ** 2
    assert abs(out["per_pair"][0] - tot / len(src[0])) <= 1e-12 * max(1.0, tot)


# --- planted mistakes (in the reference, on the CPU): each must be caught ---

def _mutant_no_relu(monkeypatch):
    monkeypatch.setattr(pn, "relu", lambda x: x)


def _mutant_bias_after_relu(monkeypatch):
    def encode(params, X, bf16=False):
        q = dict(params)
        X = np.asarray(X, np.float64)
        A1 = np.maximum(X @ q["W1"].T, 0) + q["b1"]
        A2 = np.maximum(A1 @ q["W2"].T, 0) + q["b2"]
        A3 = np.maximum(A2 @ q["W3"].T, 0) + q["b3"]
        arg = np.argmax(A3, axis=1)
        f = np.take_along_axis(A3, arg[:, None, :], axis=1)[:, 0, :]
        return f, arg, None
    monkeypatch.setattr(pn, "encode", encode)


def _mutant_target_first(monkeypatch):
    orig = pn.head
    monkeypatch.setattr(pn, "head", lambda params, fs, fd: orig(params, fd, fs))


def _mutant_mean_pool(monkeypatch):
    orig = pn.encode

    def encode(params, X, bf16=False):
        f, arg, cache = orig(params, X, bf16)
        Z3 = cache[5]
        return np.maximum(Z3, 0).mean(axis=1), arg, cache
    monkeypatch.setattr(pn, "encode", encode)


@pytest.mark.parametrize("mutant", [_mutant_no_relu, _mutant_bias_after_relu,
                                    _mutant_target_first, _mutant_mean_pool])
def test_planted_mistakes_are_caught(monkeypatch, mutant):
    p = _params(4)
    src, dst, Rg, tg = _clouds(4)
    mutant(monkeypatch)
    d = _compare(p, src, dst, Rg, tg)
    assert max(d.values()) > 1e-6, d
