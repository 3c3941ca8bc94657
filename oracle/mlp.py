"""FP64 reference of the learned-guess MLP (forward and backward) -- TEST
INFRASTRUCTURE ONLY (tests and the benchmark's CPU leg).

32 -> 64 -> 64 -> 2 with SiLU, L = (1/n) sum_i sum_j (out_ij - y_ij)^2.
Plain numpy; a matrix product serves as each layer.  Parameter layout:
W1[64][32], b1[64], W2[64][64], b2[64], W3[2][64], b3[2].
Pinned by finite differences in tests/test_oracle_mlp.py.
"""
import numpy as np

IN, HID, OUT = 32, 64, 2
SHAPES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (OUT, HID)), ("b3", (OUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = p[o:o + n].reshape(shp)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(p, X):
    w = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ w["W1"].T + w["b1"]
    a1 = z1 * sigmoid(z1)
    z2 = a1 @ w["W2"].T + w["b2"]
    a2 = z2 * sigmoid(z2)
    out = a2 @ w["W3"].T + w["b3"]
    return out, (X, z1, a1, z2, a2)


def loss_and_grad(p, X, Y):
    w = unpack(p)
    out, (X, z1, a1, z2, a2) = forward(p, X)
    n = X.shape[0]
    d = out - Y
    loss = float(np.sum(d * d) / n)
    dout = 2.0 * d / n
    g = {"W3": dout.T @ a2, "b3": dout.sum(0)}
    s2 = sigmoid(z2)
    dz2 = (dout @ w["W3"]) * (s2 * (1.0 + z2 * (1.0 - s2)))
    g["W2"] = dz2.T @ a1
    g["b2"] = dz2.sum(0)
    s1 = sigmoid(z1)
    dz1 = (dz2 @ w["W2"]) * (s1 * (1.0 + z1 * (1.0 - s1)))
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(0)
    return loss, pack(g)


def bf16_round(a):
    """Round float32 values to bfloat16 (nearest, ties to even) and back."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)
