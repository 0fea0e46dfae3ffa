"""FP64 reference of the lead-model network -- TEST INFRASTRUCTURE ONLY.

The network maps u (the energy scaled to [-1, 1]) through three hidden layers
of 128 tanh units to a linear output; parameters are stored as, for layers
l = 0..3, W_l (out x in, row-major) followed by b_l.  The loss is the mean
squared error over every output of the batch.  Written from the definitions
of a fully connected network and of backpropagation (chain rule), in float64
numpy, so that the GPU kernels' forward pass and gradients can be checked;
pinned in tests/test_oracle.py by central finite differences.
"""
import numpy as np


def layout(dims):
    """(W offset, b offset) per layer and the total parameter count."""
    offs, o = [], 0
    for l in range(len(dims) - 1):
        w = o
        o += dims[l + 1] * dims[l]
        b = o
        o += dims[l + 1]
        offs.append((w, b))
    return offs, o


def unpack(params, dims):
    offs, _ = layout(dims)
    Ws, bs = [], []
    for l, (w, b) in enumerate(offs):
        Ws.append(params[w:w + dims[l + 1] * dims[l]].reshape(dims[l + 1], dims[l]))
        bs.append(params[b:b + dims[l + 1]])
    return Ws, bs


def forward(params, dims, u):
    """Activations of every layer for inputs u (B x dims[0])."""
    params = np.asarray(params, np.float64)
    Ws, bs = unpack(params, dims)
    acts = [np.asarray(u, np.float64).reshape(-1, dims[0])]
    for l in range(len(Ws)):
        z = acts[-1] @ Ws[l].T + bs[l]
        acts.append(np.tanh(z) if l < len(Ws) - 1 else z)
    return acts


def loss_and_grad(params, dims, u, target):
    """Mean squared error and its gradient with respect to the parameters."""
    params = np.asarray(params, np.float64)
    Ws, bs = unpack(params, dims)
    acts = forward(params, dims, u)
    y = acts[-1]
    t = np.asarray(target, np.float64).reshape(y.shape)
    n = y.size
    loss = float(np.sum((y - t) ** 2) / n)
    grad = np.zeros_like(params)
    offs, _ = layout(dims)
    delta = 2.0 * (y - t) / n                      # d loss / d z of the output layer
    for l in range(len(Ws) - 1, -1, -1):
        w, b = offs[l]
        grad[w:w + Ws[l].size] = (delta.T @ acts[l]).ravel()
        grad[b:b + bs[l].size] = delta.sum(axis=0)
        if l > 0:
            delta = (delta @ Ws[l]) * (1.0 - acts[l] ** 2)   # through tanh of layer l
    return loss, grad
