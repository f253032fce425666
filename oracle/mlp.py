"""FP64 reference of the learned sub-domain proposal network (TEST INFRASTRUCTURE ONLY; never imported by
the library).  A 24 -> 64 -> 64 -> 64 multilayer perceptron with ReLU, softmax cross-entropy over the 64
depth-3 cells of the (u, v) domain, plain formulas written out.

Parameter vector (9920 floats): W1 [64, 24], b1 [64], W2 [64, 64], b2 [64], W3 [64, 64], b3 [64], each
W row-major as [out, in]."""
import numpy as np

N_IN, N_HID, N_OUT = 24, 64, 64
SHAPES = [(64, 24), (64,), (64, 64), (64,), (64, 64), (64,)]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES)   # 9920


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, k = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(theta[k:k + n].reshape(s))
        k += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(p, dtype=np.float64).reshape(-1) for p in parts])


def forward(theta, X):
    """Logits [B, 64] and the intermediate values."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ W3.T + b3
    return z3, (X, z1, h1, z2, h2)


def softmax(z):
    z = z - z.max(axis=1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=1, keepdims=True)


def loss(theta, X, y):
    """Mean softmax cross-entropy."""
    z3, _ = forward(theta, X)
    p = softmax(z3)
    return float(-np.mean(np.log(p[np.arange(len(y)), np.asarray(y)])))


def loss_and_grad(theta, X, y):
    """Mean softmax cross-entropy and its gradient with respect to the parameter vector."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    z3, (X, z1, h1, z2, h2) = forward(theta, X)
    B = X.shape[0]
    p = softmax(z3)
    y = np.asarray(y)
    L = float(-np.mean(np.log(p[np.arange(B), y])))
    dz3 = p.copy()
    dz3[np.arange(B), y] -= 1.0
    dz3 /= B
    dW3 = dz3.T @ h2
    db3 = dz3.sum(0)
    dh2 = dz3 @ W3
    dz2 = dh2 * (z2 > 0)
    dW2 = dz2.T @ h1
    db2 = dz2.sum(0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (z1 > 0)
    dW1 = dz1.T @ X
    db1 = dz1.sum(0)
    return L, pack([dW1, db1, dW2, db2, dW3, db3])


def bf16(x):
    """Round float32 values to bfloat16 (round to nearest, ties to even), returned as float32."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).reshape(a.shape)


def forward_bf16(theta, X):
    """Logits in the precision the inference kernel takes its decision in: inputs, weights and hidden
    activations rounded to bfloat16, products summed in FP32 or better, biases in FP32."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    Xb = bf16(X).astype(np.float64)
    z1 = Xb @ bf16(W1).astype(np.float64).T + b1.astype(np.float32)
    h1 = bf16(np.maximum(z1, 0.0)).astype(np.float64)
    z2 = h1 @ bf16(W2).astype(np.float64).T + b2.astype(np.float32)
    h2 = bf16(np.maximum(z2, 0.0)).astype(np.float64)
    return h2 @ bf16(W3).astype(np.float64).T + b3.astype(np.float32)
