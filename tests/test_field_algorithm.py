"""The field solve's arithmetic as the post-sweep kernel performs it, modelled on the CPU with exact
integers, against the oracle's tridiagonal Poisson solve (section "PIC/MCC simulation procedure",
Eq. poisson, with the rf Dirichlet value at x = 0 and Gauss's law over the half cells at the
electrodes).

The kernel takes the deposits D_s,j (fixed point, 2^32 per particle) and forms, in one scan of plain
integer sums, R_j = sum_{1<=k<=j} D_k and M_j = sum_{1<=k<=j} k D_k; the double sum
S_{j+1} = sum_{i<=j} R_i is then (j + 1) R_j - M_j exactly, and FP64 is used once per node, in a fixed
order (fused multiply-adds where the kernel has them). This test restates those steps in Python
(arbitrary-precision integers; fused multiply-adds rounded once through exact fractions) and checks
the identity and the resulting potential and field against the oracle within the GPU parity
tolerance (1e-12 of the largest value).

This checks the restated arithmetic, not the kernel itself. The kernel is tied to the same oracle
by tests/test_gpu_parity.py::test_poisson_matches_oracle, which uploads identical deposits, runs
the post-sweep kernel's solve and compares its potential and field with the oracle's for N = 1 to
4096, and by the full-size step tests (tests/test_gpu_fullsize.py), which compare the FP64 field of
every step."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O

E_CHARGE, EPS0, TWO32 = 1.602176634e-19, 8.8541878128e-12, 4294967296.0


def fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def i128_to_double(x):
    hi, lo = x >> 64, x & ((1 << 64) - 1)
    return fma(float(hi), 2.0 ** 64, float(lo))


def kernel_field(De, Di, w, dx, V0):
    N = len(De) - 1
    pr = [E_CHARGE * w[s] * dx / (TWO32 * EPS0) for s in (0, 1)]
    pw = [E_CHARGE * w[s] / (TWO32 * 0.5 * dx) for s in (0, 1)]
    inv_dx, m_inv_2dx, hdx_eps, inv_N = 1.0 / dx, -1.0 / (2.0 * dx), dx / (2.0 * EPS0), 1.0 / N
    R = [[0] * N, [0] * N]
    M = [[0] * N, [0] * N]
    for sp, D in ((0, De), (1, Di)):
        r = m = 0
        for j in range(N):
            if j >= 1:
                r += D[j]
                m += j * D[j]
            R[sp][j], M[sp][j] = r, m

    def Rr(j):
        return fma(pr[1], float(R[1][j]), -pr[0] * float(R[0][j]))

    def Sx(j1):  # S_{j1} from the sums through node j1 - 1
        S0 = j1 * R[0][j1 - 1] - M[0][j1 - 1]
        S1 = j1 * R[1][j1 - 1] - M[1][j1 - 1]
        return fma(pr[1], i128_to_double(S1), -pr[0] * i128_to_double(S0))

    g1 = (Sx(N) - V0) * inv_N
    phi, E = np.zeros(N + 1), np.zeros(N + 1)
    for j in range(N + 1):
        if j == 0:
            rw = fma(pw[1], float(Di[0]), -pw[0] * float(De[0]))
            phi[j], E[j] = V0, -g1 * inv_dx - rw * hdx_eps
        elif j == N:
            rw = fma(pw[1], float(Di[N]), -pw[0] * float(De[N]))
            phi[j], E[j] = 0.0, -(g1 - Rr(N - 1)) * inv_dx + rw * hdx_eps
        else:
            phi[j] = V0 + float(j) * g1 - Sx(j)
            E[j] = ((g1 - Rr(j - 1)) + (g1 - Rr(j))) * m_inv_2dx
    return phi, E, R, M


def deposits(rng, N, n_per_cell, sheath):
    """Quasi-neutral bulk, electron-depleted sheaths of `sheath` cells at both electrodes; Poisson
    counts of particles times 2^32 plus sub-particle CIC fractions."""
    z = np.arange(N + 1)
    ne = np.where((z < sheath) | (z > N - sheath), 0.05, 1.0)
    De = [int(rng.poisson(n_per_cell * x)) * (1 << 32) + int(rng.integers(0, 1 << 32)) for x in ne]
    Di = [int(rng.poisson(n_per_cell)) * (1 << 32) + int(rng.integers(0, 1 << 32)) for _ in z]
    for D in (De, Di):  # half-cell volumes at the electrodes
        D[0] //= 2
        D[N] //= 2
    return De, Di


@pytest.mark.parametrize("N,n_per_cell,w,V0", [(37, 500, (2e9, 2e9), 150.0), (512, 4000, (3e8, 3e8), -300.0),
                                               (200, 2000, (1e9, 7e8), 250.0)])
def test_kernel_arithmetic_matches_the_oracle_solve(N, n_per_cell, w, V0):
    rng = np.random.default_rng(N)
    dx = 0.025 / N
    De, Di = deposits(rng, N, n_per_cell, max(2, N // 10))
    phi, E, R, M = kernel_field(De, Di, w, dx, V0)
    # the identity: (j + 1) R_j - M_j is the double sum of the R_i
    for sp in (0, 1):
        S = 0
        for j in range(N):
            S += R[sp][j]
            assert (j + 1) * R[sp][j] - M[sp][j] == S
    rho = np.array([float(Fraction(E_CHARGE) * (Fraction(w[1]) * Di[j] - Fraction(w[0]) * De[j])
                          / (Fraction(TWO32) * Fraction(dx) * (Fraction(1, 2) if j in (0, N) else 1)))
                    for j in range(N + 1)])
    phi_o, E_o = O.poisson(rho, dx, V0)
    assert np.max(np.abs(E - E_o)) <= 1e-12 * np.max(np.abs(E_o))
    assert np.max(np.abs(phi - phi_o)) <= 1e-12 * max(np.max(np.abs(phi_o)), 1.0)
