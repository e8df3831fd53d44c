"""FP64 oracle of the learned boundary network (a library addition; the paper treats periodic
domains only).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Network: x (16, the 15 strip values + one zero pad) -> z1 = W1 x + b1 (64) -> h1 = GELU(z1)
         -> z2 = W2 h1 + b2 (64) -> h2 = GELU(z2) -> y = W3 h2 + b3 (1),
GELU(z) = z (1 + erf(z / sqrt 2)) / 2 (exact form).  The GPU multiplies BF16 operands with FP32
accumulation: the weights and every GEMM input (x, h1, h2) are rounded to BF16 (round to nearest
even) before each product, biases stay FP32.  This oracle applies the same roundings and
accumulates in FP64.  Parameter vector layout (FP32, 5313 values):
    W1[64][16], b1[64], W2[64][64], b2[64], W3[1][64], b3[1]   (row-major, out x in).

Parity unpinned beyond self-consistency: the paper defines no network.  The pins are a
finite-difference check of the backward pass, the BF16 rounding against torch's own
conversion, and closed-form cases (zero weights, a linear network in the GELU's tail).
"""
from __future__ import annotations

import math

import numpy as np

IN, HID, OUT = 16, 64, 1
SIZES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (OUT, HID)), ("b3", (OUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = p[o: o + n].reshape(shape)
        o += n
    return out


def pack(d) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SIZES])


def bf16(x) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64: the float32 bit
    pattern's low 16 bits are rounded away."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out


_erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def init_params(seed: int = 0) -> np.ndarray:
    """He-style initialisation (FP32 values)."""
    rng = np.random.default_rng(seed)
    d = {"W1": rng.normal(0, math.sqrt(2.0 / 15), (HID, IN)), "b1": np.zeros(HID),
         "W2": rng.normal(0, math.sqrt(2.0 / HID), (HID, HID)), "b2": np.zeros(HID),
         "W3": rng.normal(0, math.sqrt(1.0 / HID), (OUT, HID)), "b3": np.zeros(OUT)}
    d["W1"][:, IN - 1] = 0.0
    return pack(d).astype(np.float32).astype(np.float64)


def forward(p, x, quantize: bool = True):
    """y[rows] and the cache for backward; x is [rows][16]."""
    w = unpack(p)
    q = bf16 if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    W1, W2, W3 = q(w["W1"]), q(w["W2"]), q(w["W3"])
    x0 = q(x)
    z1 = x0 @ W1.T + w["b1"]
    h1 = gelu(z1)
    h1q = q(h1)
    z2 = h1q @ W2.T + w["b2"]
    h2 = gelu(z2)
    h2q = q(h2)
    y = (h2q @ W3.T + w["b3"])[:, 0]
    return y, {"x": x0, "z1": z1, "h1": h1q, "z2": z2, "h2": h2q, "W1": W1, "W2": W2, "W3": W3}


def loss_and_grad(p, x, t, quantize: bool = True):
    """Mean squared error L = mean_r (y_r - t_r)^2 and dL/dp (FP64).  In the quantized form the
    backward pass uses the BF16 weights and the BF16 layer inputs of the forward pass, and
    rounds the back-propagated GEMM operands (dz2, dz1) to BF16 like the GPU does."""
    y, c = forward(p, x, quantize)
    q = bf16 if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    n = y.shape[0]
    r = y - np.asarray(t, dtype=np.float64)
    L = float(np.mean(r * r))
    dy = (2.0 / n) * r[:, None]                  # [rows][1]
    g = {"W3": dy.T @ c["h2"], "b3": dy.sum(0)}
    dh2 = dy @ c["W3"]                           # [rows][64]
    dz2 = q(dh2 * gelu_grad(c["z2"]))
    g["W2"] = dz2.T @ c["h1"]
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ c["W2"]
    dz1 = q(dh1 * gelu_grad(c["z1"]))
    g["W1"] = dz1.T @ c["x"]
    g["b1"] = dz1.sum(0)
    return L, pack(g)


def adam_step(p, m, v, grad, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma & Ba) of FP32 master weights; returns (p, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


# --------------------------------------------------------------------------------------------
# edge strips (the network's input) of a D2Q5 population field
# --------------------------------------------------------------------------------------------

# Canonical orientation per edge: the strip runs along the inward normal, and the populations
# are listed as [rest, inward, outward, tangential+, tangential-] after rotating the edge onto
# the left edge (a proper rotation, so one network serves all four edges).
#   edge 0 (x = x0, normal +x): velocities (0,0), (+1,0), (-1,0), (0,+1), (0,-1)
#   edge 1 (x = x1, normal -x): rotated by 180 degrees: (0,0), (-1,0), (+1,0), (0,-1), (0,+1)
#   edge 2 (y = y0, normal +y): rotated by +90 degrees: (0,0), (0,+1), (0,-1), (-1,0), (+1,0)
#   edge 3 (y = y1, normal -y): rotated by -90 degrees: (0,0), (0,-1), (0,+1), (+1,0), (-1,0)
CANON = [[(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)],
         [(0, 0), (-1, 0), (1, 0), (0, -1), (0, 1)],
         [(0, 0), (0, 1), (0, -1), (-1, 0), (1, 0)],
         [(0, 0), (0, -1), (0, 1), (1, 0), (-1, 0)]]
NORMAL = [(1, 0), (-1, 0), (0, 1), (0, -1)]
RMS_FLOOR = 1e-30


def edge_cells(region, e):
    """(x, y) of the edge-e cells of region = (x0, y0, nx, ny), in order of the edge coordinate."""
    x0, y0, nx, ny = region
    if e == 0:
        return [(x0, y0 + k) for k in range(ny)]
    if e == 1:
        return [(x0 + nx - 1, y0 + k) for k in range(ny)]
    if e == 2:
        return [(x0 + k, y0) for k in range(nx)]
    return [(x0 + k, y0 + ny - 1) for k in range(nx)]


def strips(post, shape, c, f, region):
    """Network inputs of every edge cell of `region` from post-collision populations post[5][cells]
    of a 2D grid `shape` (velocity list c[5][2+], weights f[5]).  Returns (x[rows][16], s[rows],
    edge[rows], pos[rows]) with x = h / s, h the 15 values g_i / f*_i of the strip cells at depth
    0, 1, 2 (depth-major, canonical order inside), s = max(rms(h), 1e-30)."""
    nx = shape[0]
    idx = {(int(ci[0]), int(ci[1])): i for i, ci in enumerate(c)}
    X, S, E, P = [], [], [], []
    for e in range(4):
        n = NORMAL[e]
        for k, (cx, cy) in enumerate(edge_cells(region, e)):
            h = []
            for depth in range(3):
                px, py = cx + depth * n[0], cy + depth * n[1]
                for v in CANON[e]:
                    i = idx[v]
                    h.append(post[i, px + nx * py] / f[i])
            h = np.array(h)
            s = max(float(np.sqrt(np.mean(h * h))), RMS_FLOOR)
            X.append(np.concatenate([h / s, [0.0]]))
            S.append(s)
            E.append(e)
            P.append(k)
    return np.array(X), np.array(S), np.array(E), np.array(P)


def targets(post, shape, c, f, region):
    """Training target of every edge cell, in the order of strips(): the post-collision
    population of the inward velocity at the cell just outside the region, divided by f* and by
    the strip's scale s (so that the network's output times s f* is that population)."""
    nx = shape[0]
    idx = {(int(ci[0]), int(ci[1])): i for i, ci in enumerate(c)}
    _, S, _, _ = strips(post, shape, c, f, region)
    T = []
    for e in range(4):
        n = NORMAL[e]
        i = idx[CANON[e][1]]
        for cx, cy in edge_cells(region, e):
            ox, oy = cx - n[0], cy - n[1]
            T.append(post[i, ox + nx * oy] / f[i])
    return np.array(T) / S


SEGMENT = 16  # border rows per passivity group (one warp's rows on the GPU)


def ghost_values(p, post, shape, c, f, quantize: bool = True):
    """Entering populations of the four edges of a whole open grid predicted by the network,
    passivity-bounded per group of 16 consecutive border rows (edges in the order x = 0,
    x = nx - 1, y = 0, y = ny - 1): ghost[4][L] (L = max(nx, ny)) in solver units, the layout of
    the ghost-fed open step."""
    nx, ny = shape[0], shape[1]
    region = (0, 0, nx, ny)
    X, S, E, P = strips(post, shape, c, f, region)
    y, _ = forward(p, X, quantize)
    idx = {(int(ci[0]), int(ci[1])): i for i, ci in enumerate(c)}
    L = max(nx, ny)
    ghost = np.zeros((4, L))
    vin = S * y                 # entering populations in units of f*
    hout = X[:, 2] * S          # outward populations leaving through the same cells
    # passivity bound per group of 16 consecutive border rows: if the entering weighted energy
    # exceeds the leaving one, the group's entering populations are scaled down together
    for g0 in range(0, len(vin), SEGMENT):
        sl = slice(g0, g0 + SEGMENT)
        ein, eout = float(np.sum(vin[sl] ** 2)), float(np.sum(hout[sl] ** 2))
        if ein > eout:
            vin[sl] *= math.sqrt(eout / ein)
    for v, e, k in zip(vin, E, P):
        ghost[e, k] = v * f[idx[CANON[e][1]]]
    return ghost
