"""The learned closure's gain over the plain coarse solver, judged against the fine solve.

Fine 1024^2 Kolmogorov trajectories (Re = 1000, dt 2.5e-4) generated by the library's own
solver from seeded k^-3 fields spun up 400 fine steps; windows of 16 coarse steps (dt 4e-3,
16 fine steps each) restricted to 64^2.  The CNN closure is trained through the coarse
adjoint (spadj_gradient's dJ/dp) on 128 windows with Adam and model selection on 16
validation windows, then judged on 16 held-out windows: its relative error against the
restricted fine solution at T/2 and T must be below the plain coarse solver's (measured on
the GB300: T/4 0.01494 -> 0.01475, T/2 0.0283 -> 0.02746, T 0.05018 -> 0.04688)."""
import numpy as np
import pytest

import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NF, NC, RE = 1024, 64, 1000.0
DTF, RATIO, NCO, SPIN = 2.5e-4, 16, 16, 400


def _data(seeds):
    from paper_2506_14792_gb300 import closure_training as ct
    x0 = torch.from_numpy(np.concatenate([synthetic.kolmogorov_ic(NF, s).ravel() for s in seeds])).cuda()
    return ct.make_dataset(x0, len(seeds), NF, NC, RE, DTF, RATIO, NCO, spin=SPIN)


def test_trained_closure_beats_plain_coarse_solver():
    from paper_2506_14792_gb300 import closure_training as ct
    ntr, nva, nte = 128, 16, 16
    tr = _data(range(1000, 1000 + ntr))
    va = _data(range(3000, 3000 + nva))
    te = _data(range(2000, 2000 + nte))
    dt_c = DTF * RATIO
    at = [NCO // 4, NCO // 2, NCO]
    params = torch.from_numpy(synthetic.cnn_params(7, scale_out=0.01)).cuda()
    zero = torch.zeros_like(params)
    best, hist = ct.train_selected(params, tr, ntr, va, nva, NC, RE, dt_c, iters=150, every=25, lr=3e-3)
    plain = ct.rollout_errors(zero, te, nte, NC, RE, dt_c, at)
    cnn = ct.rollout_errors(best, te, nte, NC, RE, dt_c, at)
    mp = {k: float(plain[k].mean()) for k in at}
    mc = {k: float(cnn[k].mean()) for k in at}
    print("held-out relative error vs fine: plain", mp, "cnn", mc, "validation history", hist)
    assert mc[NCO // 2] < mp[NCO // 2]
    assert mc[NCO] < 0.98 * mp[NCO]
