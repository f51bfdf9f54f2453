"""Conjugate symmetry of the oracle's quadrature (CPU only), the fact the device's halved quadrature
rests on: for real A_i, f_i(conj z) = conj f_i(z), a region symmetric about the real axis and a
real probe block, the nodes pair up as z_{N-1-j} = conj z_j, the solves as Y_{N-1-j} = conj Y_j, and
the moments S_k equal 2 Re of the sum over the nodes above the real axis."""
import numpy as np

import synth
from oracle import ciss


def test_quadrature_of_a_real_problem_is_conjugate_symmetric():
    p = synth.delay_1d(n=64, seed=0)
    rng = np.random.default_rng(3)
    V = rng.standard_normal((p.n, 4)).astype(np.complex128)
    N, M = 32, 4
    m = ciss.moments(p, p.region, N, M, V, keep_Y=True)
    z, Y = m["z"], m["Y"]
    for j in range(N):
        assert abs(z[N - 1 - j] - np.conj(z[j])) <= 1e-14 * max(1.0, abs(z[j]))
        assert np.abs(Y[N - 1 - j] - np.conj(Y[j])).max() <= 1e-12 * np.abs(Y[j]).max()
    upper = [j for j in range(N) if z[j].imag > 0]
    assert len(upper) == N // 2
    for k in range(M):
        half = sum(m["w"][j] * m["zeta"][j] ** k * Y[j] for j in upper)
        assert np.abs(2 * half.real - m["S"][k]).max() <= 1e-11 * np.abs(m["S"][k]).max()
