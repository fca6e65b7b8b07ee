"""FP64 reference of the CNN closure (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Four 3x3 convolutions with periodic padding, channels 1 -> 32 -> 32 -> 32 -> 1, tanh after
the first three, acting on the closure's input grid field; its output is added to the
explicit term F on the collocation grid, so the weights are parameters p of F
(Supplementary A.4: parameters handled as part of the explicit term; eq. 6 for dJ/dp).
Convolution is the cross-correlation y[o, i, j] = b[o] + sum_{c, a, b} W[o, c, a, b]
x[c, i + a - 1, j + b - 1] (indices modulo the grid size).
"""
import numpy as np

CH = (1, 32, 32, 32, 1)


def n_params():
    return sum(co * ci * 9 + co for ci, co in zip(CH[:-1], CH[1:]))


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = [], 0
    for ci, co in zip(CH[:-1], CH[1:]):
        W = p[o:o + co * ci * 9].reshape(co, ci, 3, 3)
        o += co * ci * 9
        b = p[o:o + co]
        o += co
        out.append((W, b))
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def conv(x, W, b):
    """x [ci, M, M] -> [co, M, M]."""
    y = np.zeros((W.shape[0],) + x.shape[1:]) + b[:, None, None]
    for a in range(3):
        for c in range(3):
            xs = np.roll(np.roll(x, -(a - 1), axis=1), -(c - 1), axis=2)  # xs[i, j] = x[i + a - 1, j + c - 1]
            y += np.einsum("oc,cij->oij", W[:, :, a, c], xs)
    return y


def conv_t(g, W):
    """Adjoint of x -> conv(x, W, 0): g [co, M, M] -> [ci, M, M]."""
    x = np.zeros((W.shape[1],) + g.shape[1:])
    for a in range(3):
        for c in range(3):
            t = np.einsum("oc,oij->cij", W[:, :, a, c], g)
            x += np.roll(np.roll(t, a - 1, axis=1), c - 1, axis=2)
    return x


def conv_wgrad(x, g):
    """d<g, conv(x, W, b)>/dW and /db."""
    dW = np.zeros((g.shape[0], x.shape[0], 3, 3))
    for a in range(3):
        for c in range(3):
            xs = np.roll(np.roll(x, -(a - 1), axis=1), -(c - 1), axis=2)
            dW[:, :, a, c] = np.einsum("oij,cij->oc", g, xs)
    return dW, g.sum(axis=(1, 2))


class CNN:
    def __init__(self, p):
        self.layers = unpack(p)

    def _fwd(self, x):
        hs = [x[None]]
        pre = []
        for k, (W, b) in enumerate(self.layers):
            z = conv(hs[-1], W, b)
            pre.append(z)
            hs.append(np.tanh(z) if k < 3 else z)
        return hs, pre

    def forward(self, x):
        return self._fwd(x)[0][-1][0]

    def jvp(self, x, dx):
        hs, pre = self._fwd(x)
        d = dx[None]
        for k, (W, b) in enumerate(self.layers):
            dz = conv(d, W, np.zeros_like(b))
            d = (1.0 - np.tanh(pre[k]) ** 2) * dz if k < 3 else dz
        return d[0]

    def _back(self, x, g):
        hs, pre = self._fwd(x)
        grads = []
        d = g[None]
        for k in range(3, -1, -1):
            W, b = self.layers[k]
            if k < 3:
                d = d * (1.0 - np.tanh(pre[k]) ** 2)
            grads.append(conv_wgrad(hs[k], d))
            d = conv_t(d, W)
        return d[0], pack(grads[::-1])

    def vjp(self, x, g):
        return self._back(x, g)[0]

    def param_vjp(self, x, g):
        return self._back(x, g)[1]
