"""FP64 reference of the learned warm start (PointNet-style regressor of a
rigid transform).  TEST INFRASTRUCTURE: used only by the tests, the smoke
check and the benchmark's CPU leg; the product library never imports it.

The paper has no learned component; this network and its loss are the ones
the build specifies for a warm start of point-to-plane ICP:

  encoder (shared by the source and the target cloud, P points each):
    Z1 = X W1^T + b1   (3 -> 64),   A1 = relu(Z1)
    Z2 = A1 W2^T + b2  (64 -> 128), A2 = relu(Z2)
    Z3 = A2 W3^T + b3  (128 -> 256), A3 = relu(Z3)
    f  = max over the P rows of A3 (256); ties go to the smallest row
  head (per pair):
    h  = [f_src, f_dst] (512)
    Z4 = h W4^T + b4   (512 -> 256), A4 = relu(Z4)
    o  = A4 W5^T + b5  (256 -> 9)
    R  = GramSchmidt(o[0:3], o[3:6]) with columns b1, b2, b3 = b1 x b2
    t  = o[6:9]
  loss (per pair, averaged over pairs):
    L  = mean over the source points p of |(R p + t) - (R_gt p + t_gt)|^2

Every step is written out with numpy matmuls in float64; `bf16=True`
rounds W2, W3 and the activations A1, A2 to bfloat16 (round to nearest even)
before the products, which is the precision the GPU encoder multiplies in.
relu'(0) is taken as 0.
"""
from __future__ import annotations

import numpy as np

SHAPES = {
    "W1": (64, 3), "b1": (64,), "W2": (128, 64), "b2": (128,), "W3": (256, 128), "b3": (256,),
    "W4": (256, 512), "b4": (256,), "W5": (9, 256), "b5": (9,),
}
ORDER = ["W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4", "W5", "b5"]


def n_params() -> int:
    return int(sum(np.prod(SHAPES[k]) for k in ORDER))


def bf16_round(x):
    """Round float values to the nearest bfloat16 (ties to even), returned as
    float64."""
    x32 = np.ascontiguousarray(x, np.float32)
    u = x32.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def relu(x):
    return np.maximum(x, 0.0)


def encode(params, X, bf16=False):
    """Encoder of one or more clouds X [C, P, 3] -> (f [C, 256], arg [C, 256],
    cache)."""
    X = np.asarray(X, np.float64)
    W2 = bf16_round(params["W2"]) if bf16 else params["W2"]
    W3 = bf16_round(params["W3"]) if bf16 else params["W3"]
    Z1 = X @ params["W1"].T + params["b1"]
    A1 = relu(Z1)
    A1m = bf16_round(A1) if bf16 else A1
    Z2 = A1m @ W2.T + params["b2"]
    A2 = relu(Z2)
    A2m = bf16_round(A2) if bf16 else A2
    Z3 = A2m @ W3.T + params["b3"]
    A3 = relu(Z3)
    arg = np.argmax(A3, axis=1)  # first occurrence = smallest row on ties
    f = np.take_along_axis(A3, arg[:, None, :], axis=1)[:, 0, :]
    return f, arg, (X, Z1, A1m, Z2, A2m, Z3, W2, W3)


def gram_schmidt(a1, a2):
    n1 = np.linalg.norm(a1, axis=-1, keepdims=True)
    b1 = a1 / n1
    u2 = a2 - (b1 * a2).sum(-1, keepdims=True) * b1
    n2 = np.linalg.norm(u2, axis=-1, keepdims=True)
    b2 = u2 / n2
    b3 = np.cross(b1, b2)
    return np.stack([b1, b2, b3], axis=-1)  # columns


def head(params, f_src, f_dst):
    h = np.concatenate([f_src, f_dst], axis=-1)
    Z4 = h @ params["W4"].T + params["b4"]
    A4 = relu(Z4)
    o = A4 @ params["W5"].T + params["b5"]
    R = gram_schmidt(o[:, 0:3], o[:, 3:6])
    t = o[:, 6:9]
    return R, t, (h, Z4, A4, o)


def loss(R, t, P_src, R_gt, t_gt):
    """Per-pair mean squared displacement and its total (mean over pairs)."""
    P = np.asarray(P_src, np.float64)
    e = np.einsum("bij,bpj->bpi", R - R_gt, P) + (t - t_gt)[:, None, :]
    per = (e ** 2).sum(-1).mean(-1)
    return per.mean(), per, e


def forward(params, src, dst, R_gt, t_gt, bf16=False):
    f_s, a_s, c_s = encode(params, src, bf16)
    f_d, a_d, c_d = encode(params, dst, bf16)
    R, t, ch = head(params, f_s, f_d)
    L, per, e = loss(R, t, src, R_gt, t_gt)
    return {"loss": L, "per_pair": per, "R": R, "t": t, "f_src": f_s, "f_dst": f_d,
            "arg_src": a_s, "arg_dst": a_d, "_cache": (c_s, c_d, ch, e)}


def _gs_backward(a1, a2, dR):
    """Backward of R = [b1 b2 b1xb2] with respect to a1, a2 (batched)."""
    n1 = np.linalg.norm(a1, axis=-1, keepdims=True)
    b1 = a1 / n1
    d = (b1 * a2).sum(-1, keepdims=True)
    u2 = a2 - d * b1
    n2 = np.linalg.norm(u2, axis=-1, keepdims=True)
    b2 = u2 / n2
    g1 = dR[..., 0]
    g2 = dR[..., 1]
    g3 = dR[..., 2]
    # b3 = b1 x b2
    g1 = g1 + np.cross(b2, g3)
    g2 = g2 + np.cross(g3, b1)
    # b2 = u2 / n2
    gu2 = (g2 - (g2 * b2).sum(-1, keepdims=True) * b2) / n2
    # u2 = a2 - d b1, d = b1 . a2
    ga2 = gu2 - (gu2 * b1).sum(-1, keepdims=True) * b1
    gb1 = g1 - d * gu2 - (gu2 * b1).sum(-1, keepdims=True) * a2
    # b1 = a1 / n1
    ga1 = (gb1 - (gb1 * b1).sum(-1, keepdims=True) * b1) / n1
    return ga1, ga2


def _encode_backward(params, arg, f, df, cache):
    X, Z1, A1m, Z2, A2m, Z3, W2, W3 = cache
    C, Pn, _ = X.shape
    dZ3 = np.zeros_like(Z3)
    rows = np.arange(C)[:, None]
    ch = np.arange(Z3.shape[2])[None, :]
    gate = (f > 0).astype(np.float64)  # relu'(Z3) at the chosen row
    dZ3[rows, arg, ch] = df * gate
    g = {}
    g["W3"] = np.einsum("cpo,cpi->oi", dZ3, A2m)
    g["b3"] = dZ3.sum((0, 1))
    dA2 = dZ3 @ W3
    dZ2 = dA2 * (Z2 > 0)
    g["W2"] = np.einsum("cpo,cpi->oi", dZ2, A1m)
    g["b2"] = dZ2.sum((0, 1))
    dA1 = dZ2 @ W2
    dZ1 = dA1 * (Z1 > 0)
    g["W1"] = np.einsum("cpo,cpi->oi", dZ1, X)
    g["b1"] = dZ1.sum((0, 1))
    return g


def backward(params, out, src, R_gt, t_gt):
    """Gradients of the mean loss with respect to every parameter."""
    c_s, c_d, (h, Z4, A4, o), e = out["_cache"]
    B = o.shape[0]
    P = np.asarray(src, np.float64)
    Pn = P.shape[1]
    # L = (1/B) sum_b (1/Pn) sum_p |e_bp|^2,  e = (R - R_gt) p + (t - t_gt)
    de = 2.0 * e / (B * Pn)
    dR = np.einsum("bpi,bpj->bij", de, P)
    dt = de.sum(1)
    ga1, ga2 = _gs_backward(o[:, 0:3], o[:, 3:6], dR)
    do = np.concatenate([ga1, ga2, dt], axis=-1)
    g = {}
    g["W5"] = do.T @ A4
    g["b5"] = do.sum(0)
    dA4 = do @ params["W5"]
    dZ4 = dA4 * (Z4 > 0)
    g["W4"] = dZ4.T @ h
    g["b4"] = dZ4.sum(0)
    dh = dZ4 @ params["W4"]
    df_s, df_d = dh[:, :256], dh[:, 256:]
    gs = _encode_backward(params, out["arg_src"], out["f_src"], df_s, c_s)
    gd = _encode_backward(params, out["arg_dst"], out["f_dst"], df_d, c_d)
    for k in gs:
        g[k] = gs[k] + gd[k]
    return g


def init_params(seed: int = 0):
    """He-uniform weights, zero biases, and a head whose initial output is the
    identity transform (a1 = e1, a2 = e2, t = 0)."""
    rng = np.random.default_rng(seed)
    p = {}
    for w, b in (("W1", "b1"), ("W2", "b2"), ("W3", "b3"), ("W4", "b4"), ("W5", "b5")):
        fan_in = SHAPES[w][1]
        lim = np.sqrt(6.0 / fan_in)
        p[w] = rng.uniform(-lim, lim, SHAPES[w])
        p[b] = np.zeros(SHAPES[b])
    p["W5"] *= 1e-2
    p["b5"] = np.array([1.0, 0, 0, 0, 1.0, 0, 0, 0, 0])
    return p


def flatten(params) -> np.ndarray:
    return np.concatenate([np.asarray(params[k], np.float64).ravel() for k in ORDER])


def unflatten(vec) -> dict:
    out, o = {}, 0
    for k in ORDER:
        n = int(np.prod(SHAPES[k]))
        out[k] = np.asarray(vec[o:o + n], np.float64).reshape(SHAPES[k])
        o += n
    return out
