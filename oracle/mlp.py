"""FP64 reference of the learned con2prim guess network (5 -> 64 -> 64 -> 1, tanh).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The network is not in the
paper: it predicts the log of the con2prim root mu from five features of the
Kastaun et al. variables, and the FP64 root solve refines it.  This module is
the plain statement of its forward pass, mean-squared loss and gradients, in
float64 numpy, for checking the library's tensor-core kernels.

Parameter vector (fp32 in the library), flat in this order:
  W1 [64][5], b1 [64], W2 [64][64], b2 [64], w3 [64], b3 [1]    (4609 values)
followed in the library's state by the feature mean [5] and std [5] and the
target mean, std and bracket half-width (log space).
"""
import numpy as np

NIN, NH = 5, 64
NPARAM = NH * NIN + NH + NH * NH + NH + NH + 1


def unpack(p):
    p = np.asarray(p, np.float64)
    o = 0
    W1 = p[o:o + NH * NIN].reshape(NH, NIN); o += NH * NIN
    b1 = p[o:o + NH]; o += NH
    W2 = p[o:o + NH * NH].reshape(NH, NH); o += NH * NH
    b2 = p[o:o + NH]; o += NH
    w3 = p[o:o + NH]; o += NH
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def forward(p, X):
    """X [n][5] normalised features -> (y [n], cache)."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    X = np.asarray(X, np.float64)
    H1 = np.tanh(X @ W1.T + b1)
    H2 = np.tanh(H1 @ W2.T + b2)
    y = H2 @ w3 + b3
    return y, (X, H1, H2)


def loss_and_grad(p, X, t):
    """Mean squared error of y against t and its gradient w.r.t. p (chain rule)."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    y, (X, H1, H2) = forward(p, X)
    n = len(t)
    r = y - np.asarray(t, np.float64)
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n
    dw3 = H2.T @ dy
    db3 = dy.sum()
    dZ2 = np.outer(dy, w3) * (1.0 - H2 * H2)
    dW2 = dZ2.T @ H1
    db2 = dZ2.sum(0)
    dZ1 = (dZ2 @ W2) * (1.0 - H1 * H1)
    dW1 = dZ1.T @ X
    db1 = dZ1.sum(0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, [db3]])
    return loss, g


def bf16_round(x):
    """Round float values to bfloat16 (nearest even), returned as float64."""
    a = np.asarray(x, np.float32).copy()
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
