"""Oracle: the learned Davidson preconditioner's network in plain FP64 numpy.

TEST INFRASTRUCTURE ONLY (checks the CUDA training kernels).

Not in the paper: the preconditioner is the learned replacement of the diagonal
Davidson correction t_i = r_i / (theta - D_i).  The network maps 4 features of one
wave-function element to one output,
    h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  h3 = relu(W3 h2 + b3),  y = w4 . h3 + b4,
widths 4 -> 256 -> 256 -> 256 -> 1, trained on the mean squared error
    loss = (1/B) sum_b (y_b - t_b)^2.
Parameters are packed in the order W1 (256x4), b1, W2 (256x256), b2, W3 (256x256), b3,
w4 (256), b4 (1), row-major.  Gradients are written out by the chain rule here; they are
pinned by central finite differences.
"""
import numpy as np

WIDTH = 256
N_IN = 4
SHAPES = [(WIDTH, N_IN), (WIDTH,), (WIDTH, WIDTH), (WIDTH,), (WIDTH, WIDTH), (WIDTH,),
          (WIDTH,), (1,)]


def n_params():
    return int(sum(np.prod(s) for s in SHAPES))


def unpack(theta):
    out, o = [], 0
    for s in SHAPES:
        k = int(np.prod(s))
        out.append(theta[o:o + k].reshape(s))
        o += k
    return out


def pack(parts):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def forward(theta, X):
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(theta)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ W3.T + b3
    h3 = np.maximum(z3, 0.0)
    y = h3 @ w4 + b4[0]
    return y, (X, z1, h1, z2, h2, z3, h3)


def loss_and_grad(theta, X, T):
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(theta)
    B = X.shape[0]
    y, (X, z1, h1, z2, h2, z3, h3) = forward(theta, X)
    d = y - T
    loss = float(np.mean(d * d))
    dy = 2.0 * d / B                      # dloss/dy
    gw4 = h3.T @ dy
    gb4 = np.array([dy.sum()])
    dz3 = np.outer(dy, w4) * (z3 > 0)
    gW3 = dz3.T @ h2
    gb3 = dz3.sum(axis=0)
    dz2 = (dz3 @ W3) * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(axis=0)
    return loss, pack([gW1, gb1, gW2, gb2, gW3, gb3, gw4, gb4])
