"""Host check (no GPU) of the banded step solve of the plane-Couette / channel pencils: the
factors and the sweep order the GPU kernel uses (recombined, mode-ordered pencil matrix, band LU
with partial pivoting, forward sweep, 1/U_jj scaling, column-oriented back sweep; the adjoint
factorising J A'^H J), run on the host through spadj_couette_pencil_solve_host, against the
oracle's dense solve of the same pencil (a0 M + L) x = [S1S0 v; 0] and its adjoint.  Pencils with
the mean (gauge) row, with kx = 0, ky = 0 and both nonzero; SBDF1 and SBDF2 shifts; both base
flows; 1e-12 relative (the band form's measured error against a long-double solve is 1e-14
forward and 1e-13 adjoint at N = 64)."""
import numpy as np
import pytest

from oracle import couette as oco
from paper_2506_14792_gb300 import spadj

RE, DT = 1000.0, 5e-3
PENCILS = [(0.0, 0.0), (0.0, 1.0), (0.5, 0.0), (2.5, 3.0), (15.75, 31.0)]


def _dense(o, a, b, a0, v, transpose):
    N = o.N
    Mm, Lm = o.pencil_matrices(a, b, mean=(a == 0 and b == 0))
    A = a0 * Mm + Lm
    if not transpose:
        rhs = np.zeros(o.nvar, complex)
        for f in range(3):
            rhs[f * N:(f + 1) * N] = o.SS @ v[f * N:(f + 1) * N]
        return np.linalg.solve(A, rhs)[:3 * N]
    y = np.linalg.solve(A.conj().T, np.concatenate([v, np.zeros(N + 7)]))
    return np.concatenate([o.SS.T @ y[f * N:(f + 1) * N] for f in range(3)])


@pytest.mark.parametrize("N,base", [(8, "couette"), (16, "couette"), (32, "couette"), (64, "couette"),
                                    (16, "poiseuille"), (32, "poiseuille")])
def test_banded_pencil_solve_matches_dense(N, base):
    o = oco.Couette(4, 4, N, RE, pencils=False, base=base)
    rng = np.random.default_rng(N)
    for a, b in PENCILS:
        for a0 in (1.0 / DT, 1.5 / DT):
            for transpose in (False, True):
                v = rng.standard_normal(3 * N) + 1j * rng.standard_normal(3 * N)
                got = spadj.couette_pencil_solve_host(N, a, b, RE, a0, v, transpose=transpose,
                                                       base=0 if base == "couette" else 1)
                want = _dense(o, a, b, a0, v, transpose)
                err = np.max(np.abs(got - want)) / np.max(np.abs(want))
                assert err < 1e-12, (N, base, a, b, a0, transpose, err)


def test_host_solve_rejects_bad_arguments():
    with pytest.raises(spadj.SpadjError):
        spadj.couette_pencil_solve_host(10, 0.5, 0.5, RE, 200.0, np.zeros(30, complex))  # n_z not a multiple of 4
    with pytest.raises(spadj.SpadjError):
        spadj.couette_pencil_solve_host(16, 0.5, 0.5, -1.0, 200.0, np.zeros(48, complex))
