"""CPU reference of the cost-surrogate MLP (numpy, float64).

TEST INFRASTRUCTURE ONLY: used by the tests to check the device kernels'
forward pass and gradients.  Network: in -> hidden -> hidden -> out with
ReLU after the two hidden layers; loss = mean over all outputs of
(Y - T)^2.  Parameters are one flat vector in the order W1 b1 W2 b2 W3 b3,
each W row-major [out][in].  Gradients by the chain rule, written out
layer by layer; pinned in the tests by central finite differences.
"""
import numpy as np


def unpack(p, n_in, hidden, n_out):
    p = np.asarray(p, dtype=np.float64)
    shapes = [(hidden, n_in), (hidden,), (hidden, hidden), (hidden,), (n_out, hidden), (n_out,)]
    out, o = [], 0
    for s in shapes:
        size = int(np.prod(s))
        out.append(p[o:o + size].reshape(s))
        o += size
    assert o == p.size
    return out


def forward(p, X, n_in, hidden, n_out):
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, hidden, n_out)
    Z1 = X @ W1.T + b1
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ W2.T + b2
    H2 = np.maximum(Z2, 0.0)
    Y = H2 @ W3.T + b3
    return Y, (X, Z1, H1, Z2, H2)


def loss_and_grad(p, X, T, n_in, hidden, n_out):
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, hidden, n_out)
    Y, (X, Z1, H1, Z2, H2) = forward(p, X, n_in, hidden, n_out)
    D = Y - T
    loss = np.mean(D ** 2)
    dY = 2.0 * D / D.size
    gW3 = dY.T @ H2
    gb3 = dY.sum(axis=0)
    dH2 = dY @ W3
    dZ2 = dH2 * (Z2 > 0)
    gW2 = dZ2.T @ H1
    gb2 = dZ2.sum(axis=0)
    dH1 = dZ2 @ W2
    dZ1 = dH1 * (Z1 > 0)
    gW1 = dZ1.T @ X
    gb1 = dZ1.sum(axis=0)
    grad = np.concatenate([g.reshape(-1) for g in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return loss, grad
