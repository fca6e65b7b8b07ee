"""GPU tests of the closure-training support calls (spadj_restrict, spadj_adam) against their
definitions written out on the host: the spectral truncation keeps kx < Nc/2, |ky| < Nc/2 of every
member with the coarse ky = -Nc/2 row zero, and one Adam step (Kingma & Ba) follows its published
update with the bias corrections."""
import numpy as np
import pytest

import synthetic
from tests.gpu_util import dev, host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _kol(N, B, closure=False):
    from paper_2506_14792_gb300 import spadj
    return spadj.Problem(spadj.SPADJ_KOLMOGOROV2D, spadj.SPADJ_SBDF2, [N], [2 * np.pi], [1000.0, 0.0], 4e-3, batch=B,
                         closure=closure)


@pytest.mark.parametrize("Nf,Nc,B", [(32, 16, 3), (1024, 64, 2), (64, 64, 1)])
def test_restrict_is_the_spectral_truncation(Nf, Nc, B):
    fine = np.stack([synthetic.kolmogorov_ic(Nf, 40 + b) for b in range(B)])  # [B][Nf/2][Nf]
    want = np.zeros((B, Nc // 2, Nc), dtype=complex)
    for kx in range(Nc // 2):
        for j in range(Nc):
            ky = j if j < Nc // 2 else j - Nc
            if ky == -Nc // 2:
                continue
            want[:, kx, j] = fine[:, kx, ky % Nf]
    p = _kol(Nc, B)
    out = torch.full((B * (Nc // 2) * Nc,), 7.0 + 7.0j, dtype=torch.complex128, device="cuda")
    p.restrict(Nf, dev(fine.ravel()), out)
    assert np.array_equal(host(out).reshape(B, Nc // 2, Nc), want)


def test_restrict_rejects_bad_sizes():
    from paper_2506_14792_gb300 import spadj
    p = _kol(16, 1)
    f = torch.zeros(4 * 8, dtype=torch.complex128, device="cuda")  # one member of 8 modes: coarser than the problem
    c = torch.zeros(8 * 16, dtype=torch.complex128, device="cuda")
    with pytest.raises(spadj.SpadjError) as e:
        p.restrict(8, f, c)
    assert e.value.status == spadj.SPADJ_ERR_INVALID


def test_adam_step_follows_its_definition():
    p = _kol(16, 2, closure=True)
    n = p.state_len(2)
    rng = np.random.default_rng(3)
    x, m, v = rng.standard_normal(n), 0.1 * rng.standard_normal(n), rng.random(n)
    gs = [rng.standard_normal(n) for _ in range(3)]
    lr, b1, b2, eps = 3e-3, 0.9, 0.999, 1e-8
    X, Mm, V = dev(x.copy()), dev(m.copy()), dev(v.copy())
    for t, g in enumerate(gs, start=1):
        p.adam(dev(g), t, Mm, V, X, lr=lr, b1=b1, b2=b2, eps=eps)
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        x = x - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    assert np.max(np.abs(host(X) - x)) <= 1e-14 * np.max(np.abs(x))
    assert np.max(np.abs(host(Mm) - m)) <= 1e-15 * np.max(np.abs(m))
    assert np.max(np.abs(host(V) - v)) <= 1e-15 * np.max(np.abs(v))
