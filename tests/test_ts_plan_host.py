"""The host-side plan of the FP64 tangent's factorised sums (`csrc/ts_plan.cpp`), built into a
small driver and run on the CPU. Every coarse-block and coupling entry of the FP64 tangent
(Eq. NewtonUpdate2) is a combination of 738 sums of a per-point field against a product of
one-dimensional factors of the reference basis; the plan takes each sum one direction at a time.
Emulating the plan on random point fields must give the direct point sums of the definitions
(phi_0,1 = (1 -+ x)/2, psi_s = phi_a phi_b with a + b = s, N_a the trilinear shape functions in the
corner order of the element); and no step may read a value that no earlier step wrote, or write
what it reads.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TS_SUMS, TS_FIELDS = 738, 57
TF_L, TF_ADV, TF_VP, TF_G, TF_YCF, TF_YFC, TF_ZCF, TF_ZFC = 0, 9, 12, 21, 27, 39, 51, 54
TJ_L, TJ_VP, TJ_DD, TJ_OD, TJ_CFN, TJ_FCN, TJ_CFD, TJ_FCD = 0, 243, 459, 486, 522, 618, 714, 726


@pytest.fixture(scope="module")
def plans(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("needs g++")
    exe = str(tmp_path_factory.mktemp("tsplan") / "ts_plan_driver")
    subprocess.run([gxx, "-std=c++17", "-O1", os.path.join(ROOT, "tests", "ts_plan_driver.cpp"),
                    os.path.join(ROOT, "paper_0809_4802_gb300", "csrc", "ts_plan.cpp"), "-o", exe],
                   check=True, capture_output=True)
    tok = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    out, k = {}, 0
    while k < len(tok):
        assert tok[k] == "rule"
        n1, ok, nb, npl = (int(t) for t in tok[k + 1:k + 5])
        k += 5
        basis = np.array(tok[k:k + nb], dtype=np.float64)
        k += nb
        plan = np.array(tok[k:k + npl], dtype=np.int64)
        k += npl
        out[n1] = (ok, basis, plan)
    return out


def phi(b, t):
    return 0.5 * (1 + t) if b else 0.5 * (1 - t)


def psi(s, t):
    return phi(s >= 1, t) * phi(s == 2, t)


def corner_bit(a, d):
    # corner order (-,-,-) (+,-,-) (+,+,-) (-,+,-) (-,-,+) (+,-,+) (+,+,+) (-,+,+)
    return ((a + 1) >> 1) & 1 if d == 0 else ((a >> 1) & 1 if d == 1 else (a >> 2) & 1)


def d1(al):
    return 1 if al == 0 else 0


def d2(al):
    return 1 if al == 2 else 2


def direct_sums(n1, F):
    """The 738 sums from their definitions, by plain point sums."""
    x = np.polynomial.legendre.leggauss(n1)[0]
    nq = n1 ** 3
    pts = [(x[q % n1], x[(q // n1) % n1], x[q // (n1 * n1)]) for q in range(nq)]
    S = lambda f, w: sum(F[f, q] * w(pts[q]) for q in range(nq))  # noqa: E731
    E = np.zeros(TS_SUMS)
    for f in range(9):
        for t in range(27):
            E[TJ_L + 27 * f + t] = S(TF_L + f, lambda p: psi(t % 3, p[0]) * psi((t // 3) % 3, p[1]) * psi(t // 9, p[2]))
    for al in range(3):
        a1, a2 = d1(al), d2(al)
        for fl in range(4):
            fld = TF_ADV + al if fl == 0 else TF_VP + 3 * al + fl - 1
            for ty in range(18):
                xb, ps = ty & 1, ty >> 1
                E[TJ_VP + 72 * al + 18 * fl + ty] = S(fld, lambda p: phi(xb, p[al]) * psi(ps % 3, p[a1]) * psi(ps // 3, p[a2]))
        for ty in range(9):
            E[TJ_DD + 9 * al + ty] = S(TF_G + al, lambda p: psi(ty % 3, p[a1]) * psi(ty // 3, p[a2]))
        for ty in range(4):
            w = lambda p: phi(ty & 1, p[a1]) * phi(ty >> 1, p[a2])  # noqa: E731
            E[TJ_CFD + 4 * al + ty] = S(TF_ZCF + al, w)
            E[TJ_FCD + 4 * al + ty] = S(TF_ZFC + al, w)
    for pp in range(3):
        al, be, ga = (1 if pp == 2 else 0), (1 if pp == 0 else 2), 2 - pp
        for ty in range(12):
            E[TJ_OD + 12 * pp + ty] = S(TF_G + 3 + pp, lambda p: phi(ty & 1, p[al]) * phi((ty >> 1) & 1, p[be]) * psi(ty >> 2, p[ga]))
    for cf in range(12):
        for a in range(8):
            bits = [corner_bit(a, d) for d in range(3)]
            t = bits[0] + 2 * bits[1] + 4 * bits[2]   # the sums of N_a are kept in tensor order
            w = lambda p: phi(bits[0], p[0]) * phi(bits[1], p[1]) * phi(bits[2], p[2])  # noqa: E731
            E[TJ_CFN + 8 * cf + t] = S(TF_YCF + cf, w)
            E[TJ_FCN + 8 * cf + t] = S(TF_YFC + cf, w)
    return E


@pytest.mark.parametrize("n1", [2, 3])
def test_factorised_sums_equal_the_point_sums(plans, n1):
    ok, B, P = plans[n1]
    assert ok
    nq = n1 ** 3
    ld = nq | 1
    total = TS_SUMS + TS_FIELDS * ld
    x = np.polynomial.legendre.leggauss(n1)[0]
    # basis rows: psi_0..2, phi_0..1, 1, the Gauss points
    for i in range(n1):
        assert np.allclose([B[4 * s + i] for s in range(3)], [psi(s, x[i]) for s in range(3)], rtol=0, atol=1e-15)
        assert np.allclose([B[12 + i], B[16 + i], B[20 + i], B[24 + i]], [phi(0, x[i]), phi(1, x[i]), 1.0, x[i]],
                           rtol=0, atol=1e-15)
    rng = np.random.default_rng(n1)
    F = rng.standard_normal((TS_FIELDS, nq))
    A = np.full(total, np.nan)
    for f in range(TS_FIELDS):
        A[TS_SUMS + f * ld:TS_SUMS + f * ld + nq] = F[f]
    assert P[0] == 8 and all(P[k] <= P[k + 1] for k in range(6)) and P[6] == P.size
    for st in range(6):
        new, reads = {}, set()
        for j in range(P[st], P[st + 1]):
            en = int(P[j])
            i, o, row = en & 4095, (en >> 12) & 4095, en >> 24
            assert i + n1 <= total and o < total and row < 8
            vals = A[i:i + n1]
            assert not np.isnan(vals).any(), (st, j)     # read only what was written before
            reads.update(range(i, i + n1))
            assert o not in new                            # every output once per step
            new[o] = float(np.dot(B[4 * row:4 * row + n1], vals))
        assert not (reads & set(new)), st                 # a step never overwrites its inputs
        for o, v in new.items():
            A[o] = v
    E = direct_sums(n1, F)
    np.testing.assert_allclose(A[:TS_SUMS], E, rtol=0, atol=1e-13 * np.abs(E).max())
    # the number of partial sums: 8.5 k FMA per element for the 27-point rule
    if n1 == 3:
        assert P.size - 8 == 2841
