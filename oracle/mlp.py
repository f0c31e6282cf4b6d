"""FP64 reference of the learned inverse-depth proposal (test infrastructure).

The paper initialises every inverse depth from a base solution (Sec. 4); the
learned proposal is an addition of this project: a small MLP maps each
point's template patch and a few samples along its epipolar lines to an
initial inverse depth, trained on the inverse depths the bundle adjustment
itself converges to. This module is the plain, slow definition the GPU path
is checked against: numpy in FP64, loops where they keep it readable. Only
tests/, __graft_entry__.smoke() and bench.py's CPU baseline may use it; the
product path never does.

Features of point n (pixel (u, v) in the reference frame 0), 96 values:
  * the 8 x 8 template patch I_0(u + dx, v + dy), dx, dy in -3 .. 4
    (row-major in dy, then dx; coordinates clamped into the image),
    normalised by its own mean mu and population standard deviation sigma:
    (I - mu) / (sigma + EPS);
  * a 16-bin matching cost along the epipolar line in each of two target
    frames: the first two frames g >= 1 (in frame order) that observe the
    point (one frame: used twice; none: NO_DATA everywhere). The inverse
    depths d_m = D_LO + (m + 1/2) (D_HI - D_LO) / 256, m = 0 .. 255, place
    every pattern pixel x_j of the point (the method's P-pixel pattern) at
    q = R_g x~_j + d_m t_g; the cost of d_m is the mean over j of
    (I_g(pi(q)) normalised as the patch - the template's normalised value
    at x_j)^2, NO_DATA when a projection is behind the camera or its 2 x 2
    footprint leaves the image; bin k holds the least cost of d_m,
    m = 16 k .. 16 k + 15. (Sixteen raw intensities at sixteen depths would
    sample the line tens of pixels apart, far coarser than the texture: the
    least cost per bin keeps the match wherever it falls in the bin.)
Network: x (96) -> 128 -> 128 -> 128 -> 1, GELU (the exact form
x Phi(x)) after each hidden layer; y = w4 . h3 + b4 is the inverse depth.
Loss of a batch: mean of (y - target)^2 / 2. Adam (Kingma and Ba 2015).
"""
from __future__ import annotations

import math

import numpy as np

PATCH = 8
PATCH_LO = -3
N_SAMPLES = 16          # bins per frame
N_SUB = 16              # inverse depths per bin
N_FRAMES = 2
D_LO, D_HI = 0.5, 2.0
EPS = 1.0 / 255.0
NO_DATA = 4.0
N_IN = PATCH * PATCH + N_FRAMES * N_SAMPLES  # 96
N_HID = 128

# parameter order of the flat FP32 vector the GPU kernels use
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_HID, N_HID)), ("b3", (N_HID,)), ("w4", (N_HID,)), ("b4", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], dtype=np.float64).ravel() for k, _ in SHAPES])


def unpack(v: np.ndarray) -> dict:
    out, o = {}, 0
    for k, s in SHAPES:
        n = int(np.prod(s))
        out[k] = np.asarray(v[o:o + n], dtype=np.float64).reshape(s)
        o += n
    return out


def init_params(seed: int = 0) -> dict:
    """He-style initialisation: N(0, 2 / fan_in) weights, zero biases; b4 = 1
    (the mean inverse depth of a normalised scene)."""
    rng = np.random.default_rng(seed)
    p = {}
    for k, s in SHAPES:
        if k.startswith("W"):
            p[k] = rng.normal(0.0, math.sqrt(2.0 / s[1]), size=s)
        elif k == "w4":
            p[k] = rng.normal(0.0, math.sqrt(1.0 / s[0]), size=s)
        else:
            p[k] = np.zeros(s)
    p["b4"][0] = 1.0
    return p


# ----------------------------------------------------------------------------
# features
# ----------------------------------------------------------------------------
def features(images: np.ndarray, K, poses: np.ndarray, uv: np.ndarray, vis: np.ndarray,
             pattern: np.ndarray) -> np.ndarray:
    """images [F, H, W] (the values the solver reads), K = (fx, fy, cx, cy),
    poses [F, 12] row-major [R | t], uv [N, 2], vis [N, F], pattern [P, 2]
    -> [N, 96]."""
    images = np.asarray(images, dtype=np.float64)
    F, H, W = images.shape
    fx, fy, cx, cy = (float(k) for k in K)
    N = uv.shape[0]
    out = np.zeros((N, N_IN))
    nd = N_SAMPLES * N_SUB
    dm = D_LO + (np.arange(nd) + 0.5) * (D_HI - D_LO) / nd
    for n in range(N):
        u, v = int(uv[n, 0]), int(uv[n, 1])
        patch = np.empty((PATCH, PATCH))
        for i in range(PATCH):
            for j in range(PATCH):
                y = min(max(v + PATCH_LO + i, 0), H - 1)
                x = min(max(u + PATCH_LO + j, 0), W - 1)
                patch[i, j] = images[0, y, x]
        mu = patch.mean()
        sigma = math.sqrt(((patch - mu) ** 2).mean())
        scale = 1.0 / (sigma + EPS)
        out[n, :PATCH * PATCH] = ((patch - mu) * scale).ravel()
        frames = [g for g in range(1, F) if vis[n, g]][:N_FRAMES]
        if not frames:
            out[n, PATCH * PATCH:] = NO_DATA
            continue
        if len(frames) == 1:
            frames = frames * 2
        tmpl = np.array([(images[0, v + oy, u + ox] - mu) * scale for ox, oy in pattern])
        # normalised coordinates of the pattern pixels, [P, 3]
        xt = np.stack([(u + pattern[:, 0] - cx) / fx, (v + pattern[:, 1] - cy) / fy,
                       np.ones(len(pattern))], axis=1)
        for s, g in enumerate(frames):
            R = poses[g, :9].reshape(3, 3)
            t = poses[g, 9:]
            q = (xt @ R.T)[None, :, :] + dm[:, None, None] * t[None, None, :]  # [nd, P, 3]
            front = q[..., 2] > 0
            qz = np.where(front, q[..., 2], 1.0)
            val, ok = _bilinear_all(images[g], fx * q[..., 0] / qz + cx, fy * q[..., 1] / qz + cy)
            ok &= front
            c = np.where(ok, ((val - mu) * scale - tmpl[None, :]) ** 2, 0.0).mean(axis=1)
            cost = np.where(ok.all(axis=1), c, NO_DATA)
            out[n, PATCH * PATCH + s * N_SAMPLES:PATCH * PATCH + (s + 1) * N_SAMPLES] = \
                cost.reshape(N_SAMPLES, N_SUB).min(1)
    return out


def _bilinear_all(img: np.ndarray, u: np.ndarray, v: np.ndarray):
    """Bilinear samples at arrays of positions and whether each 2 x 2
    footprint lies inside the image (out-of-image samples are 0)."""
    H, W = img.shape
    x0, y0 = np.floor(u), np.floor(v)
    ok = (x0 >= 0) & (y0 >= 0) & (x0 + 1 <= W - 1) & (y0 + 1 <= H - 1)
    xi = np.where(ok, x0, 0).astype(np.int64)
    yi = np.where(ok, y0, 0).astype(np.int64)
    a, b = u - x0, v - y0
    top = (1 - a) * img[yi, xi] + a * img[yi, np.minimum(xi + 1, W - 1)]
    bot = (1 - a) * img[np.minimum(yi + 1, H - 1), xi] + a * img[np.minimum(yi + 1, H - 1), np.minimum(xi + 1, W - 1)]
    return np.where(ok, (1 - b) * top + b * bot, 0.0), ok


# ----------------------------------------------------------------------------
# network
# ----------------------------------------------------------------------------
def _erf(x: np.ndarray) -> np.ndarray:
    return np.vectorize(math.erf, otypes=[np.float64])(x)


def gelu(x: np.ndarray) -> np.ndarray:
    """x Phi(x), Phi the standard normal distribution function."""
    x = np.asarray(x, dtype=np.float64)
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x: np.ndarray) -> np.ndarray:
    """d/dx x Phi(x) = Phi(x) + x phi(x)."""
    x = np.asarray(x, dtype=np.float64)
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(p: dict, X: np.ndarray):
    """Returns y [B] and the cache of pre-activations for backward."""
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    z3 = h2 @ p["W3"].T + p["b3"]
    h3 = gelu(z3)
    y = h3 @ p["w4"] + p["b4"][0]
    return y, (X, z1, h1, z2, h2, z3, h3)


def loss_and_grad(p: dict, X: np.ndarray, target: np.ndarray):
    """Mean of (y - target)^2 / 2 over the batch and its gradient (dict)."""
    y, (X, z1, h1, z2, h2, z3, h3) = forward(p, X)
    B = X.shape[0]
    r = y - np.asarray(target, dtype=np.float64)
    loss = 0.5 * float(np.mean(r * r))
    dy = r / B
    g = {"w4": h3.T @ dy, "b4": np.array([dy.sum()])}
    dz3 = np.outer(dy, p["w4"]) * gelu_grad(z3)
    g["W3"] = dz3.T @ h2
    g["b3"] = dz3.sum(0)
    dz2 = (dz3 @ p["W3"]) * gelu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * gelu_grad(z1)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(0)
    return loss, g


def adam_step(theta: np.ndarray, grad: np.ndarray, m: np.ndarray, v: np.ndarray, step: int,
              lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (step counts from 1); returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
