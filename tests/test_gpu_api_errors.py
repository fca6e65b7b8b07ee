"""Argument checks of the newer entry points, through the C-ABI on a GPU: every bad call
returns an error status (raised by the binding) and leaves the problem usable."""
import numpy as np
import pytest

from tests.gpu_util import dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_eigen_rejects_bad_batches():
    from paper_2506_14792_gb300 import spadj, stability
    N, P = 16, 2
    prob = stability.shear_evp_problem(N, "poiseuille", P)
    x = torch.ones((P, 3 * N), dtype=torch.complex128, device="cuda")
    psi = torch.ones_like(x)
    out = torch.zeros((P, 10), dtype=torch.float64, device="cuda")
    good = [(1.0, 0.0, 2000.0), (1.1, 0.0, 2000.0)]
    for prm, n_iter in (([(1.0, 0.0, -5.0), (1.0, 0.0, 1.0)], 5), (good, 0)):
        with pytest.raises(spadj.SpadjError):
            prob.eigen(prm, [-0.25j, -0.25j], n_iter, x, psi, out)
    x3 = torch.ones((3, 3 * N), dtype=torch.complex128, device="cuda")
    with pytest.raises(spadj.SpadjError):  # more pencils than the problem's batch
        prob.eigen(good + [(1.2, 0.0, 2000.0)], [-0.25j] * 3, 5, x3, torch.ones_like(x3),
                   torch.zeros((3, 10), dtype=torch.float64, device="cuda"))
    prob.eigen(good, [-0.25j, -0.27j], 5, x, psi, out)  # still usable
    assert np.all(np.isfinite(out.cpu().numpy()))
    with pytest.raises(spadj.SpadjError):  # base flow must be 0 or 1
        spadj.Problem(spadj.SPADJ_SHEAR_EVP, 0, (0, 0, N), (0.0, 0.0, 0.0), (2,), 1.0, batch=1)


def test_schedule_and_host_slot_options():
    from paper_2506_14792_gb300 import spadj
    from tests.rb_util import gpu_problem
    p = gpu_problem(16, 12, dt=1e-2)
    with pytest.raises(spadj.SpadjError):
        p.set_dt_schedule([1e-2, -1e-3])
    with pytest.raises(spadj.SpadjError):
        p.set_option(9, -1)
    x0 = dev(np.zeros((3, 8, 12), dtype=np.complex128))
    g = torch.zeros((3, 8, 12), dtype=torch.complex128, device="cuda")
    p.set_option(9, 100)  # more host slots than steps: one per step
    p.gradient(x0, 4, g, ckpt_slots=1)
    from tests.test_gpu_couette import gpu_problem as cou_problem
    c = cou_problem(8, 4, 8)
    with pytest.raises(spadj.SpadjError):  # step-size schedules are defined for the RB problem only
        c.set_dt_schedule([1e-2])
