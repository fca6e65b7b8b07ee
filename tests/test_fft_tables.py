"""Host-side check (no GPU) of the FFT plans' scaled-twiddle records, the table the CUDA
butterflies read (Goedecker's multiply-add form: a twiddle w = c + i s applied as
lambda (v + tau i v)).

A small host program built with nvcc against the library's own FFT header dumps the plan and
the records for several lengths.  The records must reproduce every twiddle of every pass,
exp(SIGN 2 pi i m k / (R Ns)), to rounding; |tau| <= 1 must hold; and a Stockham FFT that
consumes the records the way the device butterflies do (swaps by the flag word, per-component
scales) must equal numpy's FFT in both directions.
"""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2506_14792_gb300", "csrc")
LENGTHS = [2, 3, 4, 6, 8, 12, 24, 48, 64, 96, 128, 192, 288, 384, 576, 768]

DUMP = r'''
#include <cstdio>
#include <cstdlib>
#include "fft.cuh"
int main(int argc, char** argv) {
  for (int a = 1; a < argc; ++a) {
    spadj::FFTPlan p = spadj::make_plan(std::atoi(argv[a]));
    std::vector<double2> t = spadj::scaled_twiddle_table(p);
    std::printf("plan %d %d", p.n, p.nrad);
    for (int i = 0; i < p.nrad; ++i) std::printf(" %d", (int)p.rad[i]);
    std::printf(" entries %d\n", spadj::scaled_twiddle_entries(p));
    for (const double2& e : t) std::printf("%a %a\n", e.x, e.y);
  }
  return 0;
}
'''


@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    if shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("fft_tables")
    src = d / "dump.cu"
    src.write_text(DUMP)
    exe = d / "dump"
    subprocess.run(["nvcc", "-std=c++17", "-I", CSRC, "-o", str(exe), str(src)], check=True, capture_output=True)
    out = subprocess.run([str(exe)] + [str(n) for n in LENGTHS], check=True, capture_output=True, text=True).stdout
    lines = out.strip().splitlines()
    res, i = {}, 0
    while i < len(lines):
        f = lines[i].split()
        n, nrad = int(f[1]), int(f[2])
        rad = [int(x) for x in f[3:3 + nrad]]
        ent = int(f[-1])
        cnt = max(2 * ent, 1)
        recs = [tuple(float.fromhex(x) for x in lines[i + 1 + j].split()) for j in range(cnt)]
        res[n] = (rad, ent, recs)
        i += 1 + cnt
    return res


def _flags(d):
    return struct.unpack("<q", struct.pack("<d", d))[0]


def _rec_len(R):
    return 2 if R == 2 else 6


def _passes(rad, ent, recs, sign):
    """Yield (R, Ns, records of the pass) in pass order for one direction."""
    base = 0 if sign < 0 else ent
    off, Ns = 0, 1
    for R in rad:
        n_ent = Ns * _rec_len(R) if Ns > 1 else 0
        yield R, Ns, recs[base + off: base + off + n_ent]
        off += n_ent
        Ns *= R


def _coef(scales, im):
    """The complex coefficient given by its per-component scales and imaginary flag."""
    ax, ay = scales
    if im:
        assert ax == -ay
        return 1j * ay
    assert ax == ay
    return ax


def test_plans_factor_the_length(tables):
    for n, (rad, ent, recs) in tables.items():
        assert int(np.prod(rad)) == n
        assert all(r in (2, 3, 4) for r in rad)


def test_records_reproduce_the_twiddles(tables):
    for n, (rad, ent, recs) in tables.items():
        for sign in (-1, 1):
            for R, Ns, pr in _passes(rad, ent, recs, sign):
                if Ns == 1:
                    continue
                L = _rec_len(R)
                for k in range(Ns):
                    r = pr[k * L:(k + 1) * L]
                    w = [np.exp(sign * 2j * np.pi * m * k / (R * Ns)) for m in range(R)]
                    if R == 4:
                        t1, t2 = r[0]
                        t3, fw = r[1]
                        f = _flags(fw)
                        lam2, rho, lam1, kap = _coef(r[2], f & 1), _coef(r[3], f & 2), _coef(r[4], f & 4), \
                            _coef(r[5], not (f & 4))
                        taus = (t1, t2, t3)
                        got = [lam1 * (1 + 1j * t1), lam2 * (1 + 1j * t2), rho * lam1 * (1 + 1j * t3)]
                        assert abs(kap - sign * 1j * lam1) <= 1e-16
                    elif R == 3:
                        t1, t2 = r[0]
                        f = _flags(r[5][0])
                        rho, lam1, half, kap = _coef(r[1], f & 2), _coef(r[2], f & 4), _coef(r[3], f & 4), \
                            _coef(r[4], not (f & 4))
                        taus = (t1, t2)
                        got = [lam1 * (1 + 1j * t1), rho * lam1 * (1 + 1j * t2)]
                        assert abs(half + 0.5 * lam1) <= 1e-16
                        assert abs(kap - sign * 1j * lam1 * np.sqrt(3) / 2) <= 2e-16
                    else:
                        t1, fw = r[0]
                        lam1 = _coef(r[1], _flags(fw) & 4)
                        taus = (t1,)
                        got = [lam1 * (1 + 1j * t1)]
                    assert all(abs(t) <= 1.0 for t in taus)
                    for m in range(1, R):
                        assert abs(got[m - 1] - w[m]) <= 4e-16, (n, sign, R, Ns, k, m)


def _swap(z, im):
    return complex(z.imag, z.real) if im else z


def _add(u, a, z):
    return complex(u.real + a[0] * z.real, u.imag + a[1] * z.imag)


def _sub(u, a, z):
    return complex(u.real - a[0] * z.real, u.imag - a[1] * z.imag)


def _q(v, t):
    return complex(v.real - t * v.imag, v.imag + t * v.real)


def _stockham(x, rad, passes, sign):
    """Stockham autosort FFT consuming the records as the device butterflies do."""
    n = len(x)
    a, b = np.array(x, dtype=complex), np.zeros(n, dtype=complex)
    for R, Ns, pr in passes:
        nbf = n // R
        L = _rec_len(R)
        for j in range(nbf):
            k = j % Ns
            base = (j - k) * R + k
            v = [a[j + m * nbf] for m in range(R)]
            if Ns == 1:
                y = [sum(v[m] * np.exp(sign * 2j * np.pi * m * o / R) for m in range(R)) for o in range(R)]
            else:
                r = pr[k * L:(k + 1) * L]
                if R == 4:
                    f = _flags(r[1][1])
                    q1 = _q(v[1], r[0][0])
                    q2 = _swap(_q(v[2], r[0][1]), f & 1)
                    q3 = _swap(_q(v[3], r[1][0]), f & 2)
                    A, B = _add(v[0], r[2], q2), _sub(v[0], r[2], q2)
                    E, F = _swap(_add(q1, r[3], q3), f & 4), _swap(_sub(q1, r[3], q3), not (f & 4))
                    y = [_add(A, r[4], E), _add(B, r[5], F), _sub(A, r[4], E), _sub(B, r[5], F)]
                elif R == 3:
                    f = _flags(r[5][0])
                    q1 = _q(v[1], r[0][0])
                    q2 = _swap(_q(v[2], r[0][1]), f & 2)
                    E, F = _swap(_add(q1, r[1], q2), f & 4), _swap(_sub(q1, r[1], q2), not (f & 4))
                    Mv = _add(v[0], r[3], E)
                    y = [_add(v[0], r[2], E), _add(Mv, r[4], F), _sub(Mv, r[4], F)]
                else:
                    qv = _swap(_q(v[1], r[0][0]), _flags(r[0][1]) & 4)
                    y = [_add(v[0], r[1], qv), _sub(v[0], r[1], qv)]
            for m in range(R):
                b[base + m * Ns] = y[m]
        a, b = b, a
    return a


PLANS = r'''
#include <cstdio>
#include <cstdlib>
#include "fft.cuh"
int main(int argc, char** argv) {
  for (int a = 1; a < argc; ++a) std::printf("%d\n", spadj::make_plan(std::atoi(argv[a])).nrad);
  return 0;
}
'''


def test_plan_rejects_unsupported_lengths(tmp_path):
    """Lengths that are not 2^a 3^b, or that would need more than the plan's eight passes, are
    refused (nrad = -1) instead of overrunning the radix list."""
    if shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    (tmp_path / "plans.cu").write_text(PLANS)
    exe = tmp_path / "plans"
    subprocess.run(["nvcc", "-std=c++17", "-I", CSRC, "-o", str(exe), str(tmp_path / "plans.cu")], check=True,
                   capture_output=True)
    ns = [1, 192, 1536, 4 * 3 ** 7, 4 * 3 ** 8, 3 ** 9, 5, 0, -4]
    out = subprocess.run([str(exe)] + [str(n) for n in ns], check=True, capture_output=True, text=True).stdout.split()
    nrad = dict(zip(ns, (int(v) for v in out)))
    assert nrad[1] == 0 and nrad[192] == 4 and nrad[1536] == 6 and nrad[4 * 3 ** 7] == 8
    assert all(nrad[n] == -1 for n in (4 * 3 ** 8, 3 ** 9, 5, 0, -4))


@pytest.mark.parametrize("n", [6, 12, 48, 96, 192, 384])
def test_record_butterflies_equal_numpy_fft(tables, n):
    rad, ent, recs = tables[n]
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for sign in (-1, 1):
        got = _stockham(x, rad, list(_passes(rad, ent, recs, sign)), sign)
        want = np.fft.fft(x) if sign < 0 else np.fft.ifft(x) * n
        assert np.max(np.abs(got - want)) <= 4e-15 * np.max(np.abs(want)), (n, sign)
