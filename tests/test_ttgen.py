"""Pins for the seeded input generators (ttgen/): each claim of its docstrings that the
benchmark and the parity tests rely on, checked against plain numpy on small sizes."""

import numpy as np

import ttgen
from oracle import tt


def test_bond_bounds():
    assert ttgen.bond_bounds(6, 2, 0) == [1, 2, 4, 8, 4, 2, 1]
    assert ttgen.bond_bounds(6, 2, 3) == [1, 2, 3, 3, 3, 2, 1]
    assert ttgen.bond_bounds(3, 4, 0) == [1, 4, 4, 1]


def test_rand_tt_spectral_is_right_canonical_unit_norm_with_decaying_spectra():
    L, chi = 12, 16
    T = ttgen.rand_tt_spectral(L, 2, chi, 7)
    assert tt.bonds_of(T) == ttgen.bond_bounds(L, 2, chi)
    for c in T[1:]:                                     # right-orthonormal cores 2..L
        m = c.reshape(c.shape[0], -1)
        np.testing.assert_allclose(m @ m.T, np.eye(m.shape[0]), atol=1e-12)
    assert abs(np.linalg.norm(T[0]) - 1.0) <= 1e-12
    assert abs(np.linalg.norm(tt.dense(T)) - 1.0) <= 1e-12
    # the 1/k profiles compound: the realised Schmidt values at the middle bond decay faster
    # than 1/k (about k^-3 at this size), monotonically, over more than two decades
    x = tt.dense(T).reshape(2 ** (L // 2), -1)
    s = np.linalg.svd(x, compute_uv=False)[:chi]
    assert np.all(np.diff(s) <= 1e-12)
    k = np.arange(1, chi + 1)
    slope = np.polyfit(np.log(k[1:]), np.log(s[1:] / s[0]), 1)[0]
    assert -4.0 < slope < -2.0, slope
    assert s[-1] / s[0] < 1e-2


def test_rand_tt_canonical_forms():
    A = ttgen.rand_tt(7, 3, 5, 3, canon="left")
    for c in A[:-1]:
        m = c.reshape(-1, c.shape[2])
        np.testing.assert_allclose(m.T @ m, np.eye(m.shape[1]), atol=1e-12)
    B = ttgen.rand_tt(7, 3, 5, 3, canon="right")
    np.testing.assert_allclose(tt.dense(A), tt.dense(B), atol=1e-12 * np.abs(tt.dense(A)).max())


def test_tt_svd_is_exact_without_truncation_and_respects_the_cap():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(3 ** 6)
    T = ttgen.tt_svd(x, 6, 3)
    np.testing.assert_allclose(tt.dense(T), x, atol=1e-12 * np.abs(x).max())
    assert max(tt.bonds_of(ttgen.tt_svd(x, 6, 3, chi=4))) <= 4


def test_interleave_2d_bit_order():
    L = 2
    n = 2 ** L
    f = np.arange(n * n, dtype=float).reshape(n, n)    # f[x, y] = 4 x + y
    q = ttgen.interleave_2d(f, L)
    for x in range(n):
        for y in range(n):
            bx = [(x >> (L - 1 - k)) & 1 for k in range(L)]
            by = [(y >> (L - 1 - k)) & 1 for k in range(L)]
            idx = 0
            for k in range(L):                           # site k: s_k = 2 bx_k + by_k, coarsest first
                idx = idx * 4 + 2 * bx[k] + by[k]
            assert q[idx] == f[x, y]


def test_turbulence_2d_is_divergence_free_unit_energy_and_encoded():
    L = 5
    ut, vt, u, v = ttgen.turbulence_2d(L=L, chi=64, seed=3, kmin=2.0, kmax=8.0)
    n = 2 ** L
    assert abs(np.mean(u ** 2 + v ** 2) / 2 - 1.0) <= 1e-12
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    kx, ky = np.meshgrid(k1, k1, indexing="ij")
    uh, vh = np.fft.fft2(u), np.fft.fft2(v)
    div = kx * uh + ky * vh                              # spectral divergence (up to 2 pi i)
    assert np.linalg.norm(div) <= 1e-10 * np.linalg.norm(kx * uh)
    # energy only on the shell 2 <= |k| <= 8
    kk = np.sqrt(kx ** 2 + ky ** 2)
    assert np.abs(uh[(kk < 2) | (kk > 8)]).max() <= 1e-9 * np.abs(uh).max()
    np.testing.assert_allclose(tt.dense(ut), ttgen.interleave_2d(u, L), atol=1e-10)
    np.testing.assert_allclose(tt.dense(vt), ttgen.interleave_2d(v, L), atol=1e-10)


def _grid_3d(L):
    n = 2 ** L
    j = np.arange(n) / n
    return np.meshgrid(j, j, j, indexing="ij")


def _dense_3d(T, L):
    """d=8 QTT -> (x, y, z) grid: site k holds (bx, by, bz) at scale 2^-k, s = 4 bx + 2 by + bz."""
    q = tt.dense(T).reshape((2, 2, 2) * L)
    perm = [3 * k for k in range(L)] + [3 * k + 1 for k in range(L)] + [3 * k + 2 for k in range(L)]
    n = 2 ** L
    return q.transpose(perm).reshape(n, n, n)


def test_qtt_mode_3d_is_an_exact_cosine_mode():
    L = 3
    X, Y, Z = _grid_3d(L)
    k, amp, ph = (1.0, -2.0, 3.0), 0.7, 0.4
    T = ttgen.qtt_mode_3d(L, k, amp, ph)
    ref = amp * np.cos(2 * np.pi * (k[0] * X + k[1] * Y + k[2] * Z) + ph)
    np.testing.assert_allclose(_dense_3d(T, L), ref, atol=1e-12)
    assert max(tt.bonds_of(T)) == 2


def test_turbulence_3d_fields_are_solenoidal_with_exact_derivatives():
    L = 3
    fields, derivs = ttgen.turbulence_3d_fields(L=L, n_modes=4, seed=5, chis=[64] * 12, kmin=1.0, kmax=3.0)
    n = 2 ** L
    u = [_dense_3d(f, L) for f in fields]
    kk = np.fft.fftfreq(n, d=1.0 / n)
    K = np.meshgrid(kk, kk, kk, indexing="ij")
    scale = max(np.abs(x).max() for x in u)
    for j in range(3):
        for i in range(3):
            spectral = np.real(np.fft.ifftn(2j * np.pi * K[j] * np.fft.fftn(u[i])))
            np.testing.assert_allclose(_dense_3d(derivs[j][i], L), spectral, atol=1e-9 * scale * 2 * np.pi * 3)
    div = sum(_dense_3d(derivs[i][i], L) for i in range(3))
    assert np.abs(div).max() <= 1e-9 * scale * 2 * np.pi * 3
