"""Pins for the FP64 CNN closure oracle and the parameter gradient of the multistep adjoint.

* convolution vs a brute-force direct sum with explicit periodic indices;
* conv adjoints and the network's input VJP by dot tests against the JVP;
* parameter VJP vs central differences;
* Kolmogorov with the closure: state and parameter gradients of a trajectory objective vs
  central differences (eq. 6 with the parameters entering F at every step).
"""
import numpy as np

import synthetic
from oracle import cnn, imex
from oracle import kolmogorov as okol
from oracle.imex import inner


def test_param_count():
    assert cnn.n_params() == 19105


def test_conv_bruteforce():
    rng = np.random.default_rng(0)
    M, ci, co = 5, 2, 3
    x = rng.standard_normal((ci, M, M))
    W = rng.standard_normal((co, ci, 3, 3))
    b = rng.standard_normal(co)
    y = cnn.conv(x, W, b)
    for o in range(co):
        for i in range(M):
            for j in range(M):
                s = b[o]
                for c in range(ci):
                    for a in range(3):
                        for d in range(3):
                            s += W[o, c, a, d] * x[c, (i + a - 1) % M, (j + d - 1) % M]
                assert abs(y[o, i, j] - s) < 1e-12


def test_conv_adjoints():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((4, 6, 6))
    W = rng.standard_normal((5, 4, 3, 3))
    g = rng.standard_normal((5, 6, 6))
    assert abs(np.sum(cnn.conv(x, W, np.zeros(5)) * g) - np.sum(x * cnn.conv_t(g, W))) < 1e-11
    dW, db = cnn.conv_wgrad(x, g)
    E = rng.standard_normal(W.shape)
    assert abs(np.sum(cnn.conv(x, E, np.zeros(5)) * g) - np.sum(dW * E)) < 1e-11


def test_network_vjp_and_param_grad():
    p = synthetic.cnn_params(3, scale_out=1.0)
    net = cnn.CNN(p)
    rng = np.random.default_rng(2)
    x = rng.standard_normal((8, 8))
    dx = rng.standard_normal((8, 8))
    g = rng.standard_normal((8, 8))
    assert abs(np.sum(net.jvp(x, dx) * g) - np.sum(dx * net.vjp(x, g))) < 1e-10
    h = 1e-6
    fd = (np.sum(net.forward(x + h * dx) * g) - np.sum(net.forward(x - h * dx) * g)) / (2 * h)
    assert abs(fd - np.sum(dx * net.vjp(x, g))) < 1e-6 * abs(fd)
    gp = net.param_vjp(x, g)
    for s in range(4):
        d = np.random.default_rng(10 + s).standard_normal(p.size)
        fd = (np.sum(cnn.CNN(p + h * d).forward(x) * g) - np.sum(cnn.CNN(p - h * d).forward(x) * g)) / (2 * h)
        assert abs(fd - gp @ d) < 1e-6 * abs(fd)


def test_kolmogorov_closure_gradients_fd():
    N, Re, dt, nsteps = 16, 1000.0, 4e-3, 8
    p0 = synthetic.cnn_params(4, scale_out=0.5)
    X0 = okol.Kolmogorov(N, Re).project(synthetic.kolmogorov_ic(N, 11))
    target = okol.Kolmogorov(N, Re).project(synthetic.kolmogorov_ic(N, 12))

    def run(p, X0_):
        prob = okol.Kolmogorov(N, Re, closure=cnn.CNN(p))
        X = imex.multistep_forward(prob, X0_, nsteps, dt)
        J = 0.5 * np.sum(np.abs(X[-1] - target) ** 2)
        return prob, X, J

    prob, X, J = run(p0, X0)
    gx, gp = imex.multistep_adjoint_params(prob, X, lambda n: X[n] - target if n == nsteps else None, dt)
    gx2 = imex.multistep_adjoint(prob, X, lambda n: X[n] - target if n == nsteps else None, dt)
    np.testing.assert_allclose(gx, gx2, atol=1e-14 * np.max(np.abs(gx)))
    for s in range(3):
        d = np.random.default_rng(30 + s).standard_normal(p0.size)
        eps = 1e-6
        fd = (run(p0 + eps * d, X0)[2] - run(p0 - eps * d, X0)[2]) / (2 * eps)
        assert abs(fd - gp @ d) <= 1e-6 * abs(fd)
        dx = okol.Kolmogorov(N, Re).project(synthetic.kolmogorov_ic(N, 40 + s))
        eps = 1e-6 * np.linalg.norm(X0) / np.linalg.norm(dx)
        fd = (run(p0, X0 + eps * dx)[2] - run(p0, X0 - eps * dx)[2]) / (2 * eps)
        assert abs(fd - inner(gx, dx)) <= 1e-6 * abs(fd)
