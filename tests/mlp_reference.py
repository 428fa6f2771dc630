"""CPU reference of the learned seed's forward and backward (numpy, float64 arithmetic with
BF16 rounding at the points where the kernel stores BF16), for checking the GPU gradients."""
import numpy as np

H = 64


def bf16(a):
    """Round to bfloat16 (nearest, ties to even) and back to float64."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p):
    o = 0
    out = {}
    for name, shape in (("w1", (H, 2)), ("b1", (H,)), ("w2", (H, H)), ("b2", (H,)), ("w3", (H, H)), ("b3", (H,)),
                        ("w4", (H,)), ("b4", ())):
        size = int(np.prod(shape)) if shape else 1
        out[name] = np.asarray(p[o:o + size], dtype=np.float64).reshape(shape)
        o += size
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def loss_and_grad(params, f, y, valid):
    """Sum of squared errors and its gradient, in the flat parameter order."""
    P = unpack(params)
    w1, w2, w3, w4 = bf16(P["w1"]), bf16(P["w2"]), bf16(P["w3"]), bf16(P["w4"])
    b1, b2, b3, b4 = P["b1"], P["b2"], P["b3"], float(P["b4"])
    z1 = f @ w1.T + b1
    a1 = bf16(silu(z1))
    z2 = a1 @ w2.T + b2
    a2 = bf16(silu(z2))
    z3 = a2 @ w3.T + b3
    a3 = bf16(silu(z3))
    o = a3 @ w4 + b4
    err = np.where(valid, o - y, 0.0)
    dO = 2.0 * err
    g = {"w4": a3.T @ dO, "b4": np.array(dO.sum())}
    dZ3 = dO[:, None] * w4[None, :] * silu_grad(z3)
    g["b3"] = dZ3.sum(0)
    dZ3b = bf16(dZ3)
    g["w3"] = dZ3b.T @ a2  # [out][in]
    dZ2 = (dZ3b @ w3) * silu_grad(z2)
    g["b2"] = dZ2.sum(0)
    dZ2b = bf16(dZ2)
    g["w2"] = dZ2b.T @ a1
    dZ1 = (dZ2b @ w2) * silu_grad(z1)
    g["b1"] = dZ1.sum(0)
    g["w1"] = dZ1.T @ f
    flat = np.concatenate([g[k].ravel() for k in ("w1", "b1", "w2", "b2", "w3", "b3", "w4", "b4")])
    return float((err ** 2).sum()), flat


def grad_magnitudes(params, f, y, valid):
    """Per element of the gradient, the sum over rows of |each product that enters it|: the same
    backward as ``loss_and_grad`` with every factor replaced by its absolute value.  A relative
    perturbation delta of every factor on a path moves that element by at most ~ (path length)
    delta times this sum, which bounds the GPU's deviation element by element."""
    P = unpack(params)
    w1, w2, w3, w4 = bf16(P["w1"]), bf16(P["w2"]), bf16(P["w3"]), bf16(P["w4"])
    b1, b2, b3, b4 = P["b1"], P["b2"], P["b3"], float(P["b4"])
    z1 = f @ w1.T + b1
    a1 = bf16(silu(z1))
    z2 = a1 @ w2.T + b2
    a2 = bf16(silu(z2))
    z3 = a2 @ w3.T + b3
    a3 = bf16(silu(z3))
    o = a3 @ w4 + b4
    dO = np.abs(np.where(valid, 2.0 * (o - y), 0.0))
    g = {"w4": np.abs(a3).T @ dO, "b4": np.array(dO.sum())}
    dZ3 = dO[:, None] * np.abs(w4)[None, :] * np.abs(silu_grad(z3))
    g["b3"] = dZ3.sum(0)
    g["w3"] = dZ3.T @ np.abs(a2)
    dZ2 = (dZ3 @ np.abs(w3)) * np.abs(silu_grad(z2))
    g["b2"] = dZ2.sum(0)
    g["w2"] = dZ2.T @ np.abs(a1)
    dZ1 = (dZ2 @ np.abs(w2)) * np.abs(silu_grad(z1))
    g["b1"] = dZ1.sum(0)
    g["w1"] = dZ1.T @ np.abs(f)
    return np.concatenate([g[k].ravel() for k in ("w1", "b1", "w2", "b2", "w3", "b3", "w4", "b4")])
