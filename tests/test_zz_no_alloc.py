"""spadj_transform_noalloc: the transform entry point that allocates nothing, for callers
whose device memory belongs to their own allocator (or who cannot pay for cudaMalloc's
device synchronisation).  Called through the C-ABI and compared with spadj_transform on
the same inputs, two calls in a row (the static scratch is shared by every call and keeps
the previous call's contents).  Collected last so that a failure here cannot hide any
other test."""
import ctypes

import numpy as np
import pytest

import synthetic
from tests.gpu_util import dev, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("Nx,Nz", [(16, 12), (256, 64)])
def test_noalloc_transform_matches_transform(Nx, Nz):
    from paper_2506_14792_gb300 import spadj
    from tests.rb_util import gpu_problem
    p = gpu_problem(Nx, Nz)
    L = spadj.lib()
    Kx, Mz, Mx = Nx // 2, 3 * Nz // 2, 3 * Nx // 2
    for call in range(2):
        c = synthetic.random_coeffs((Kx, Nz), seed=100 + call)
        c[0] = c[0].real
        g = np.random.default_rng(200 + call).standard_normal((Mz, Mx))
        for kind in (spadj.C2G, spadj.G2C, spadj.C2G_ADJ, spadj.G2C_ADJ):
            to_grid = kind in (spadj.C2G, spadj.G2C_ADJ)
            x = dev(c) if to_grid else dev(g)
            shape = (Mz, Mx) if to_grid else (Kx, Nz)
            dtype = torch.float64 if to_grid else torch.complex128
            ref = torch.zeros(shape, dtype=dtype, device="cuda")
            out = torch.full(shape, float("nan"), dtype=dtype, device="cuda")
            p.transform(kind, x, ref)
            xin = torch.view_as_real(x) if x.is_complex() else x
            oo = torch.view_as_real(out) if out.is_complex() else out
            st = L.spadj_transform_noalloc(p.h, kind, ctypes.c_void_p(xin.data_ptr()), ctypes.c_void_p(oo.data_ptr()))
            assert st == spadj.SPADJ_OK, L.spadj_last_error(p.h)
            torch.cuda.synchronize()
            assert rel_err(out.cpu().numpy(), ref.cpu().numpy()) < 1e-13


def test_noalloc_rejects_oversize():
    from paper_2506_14792_gb300 import spadj
    from tests.rb_util import gpu_problem
    p = gpu_problem(49152, 8)  # (3*8/2) * (49152/2) = 294912 > 262144; tiny pencils, cheap set-up
    L = spadj.lib()
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = L.spadj_transform_noalloc(p.h, spadj.C2G, ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()))
    assert st == spadj.SPADJ_ERR_INVALID
    assert b"exceeds the static scratch" in L.spadj_last_error(p.h)
