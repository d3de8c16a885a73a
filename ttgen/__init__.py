"""Seeded synthetic tensor-train inputs (numpy, float64).

Shared by the tests, ``bench.py`` and ``smoke()``: both the CUDA path and the
oracle receive exactly these arrays. This module holds none of the TTM
arithmetic (no Contract, Swap, truncation rule or gauge move); it only draws
random numbers and encodes fields as TTs with plain numpy QR / SVD calls.

Core layout everywhere: (D_l, d, D_r), row-major, D_0 = D_L = 1; the full tensor
index is (s_1, ..., s_L) with s_1 the slowest (the coarsest bit for quantics).
"""

import numpy as np


def bond_bounds(L, d, chi):
    """D_i = min(d^i, d^(L-i), chi) for i = 0..L."""
    out = []
    for i in range(L + 1):
        v = min(d ** i, d ** (L - i))
        if chi:
            v = min(v, chi)
        out.append(int(v))
    return out


def _left_sweep(cores):
    C = [c.copy() for c in cores]
    for k in range(len(C) - 1):
        Dl, d, Dr = C[k].shape
        Q, R = np.linalg.qr(C[k].reshape(Dl * d, Dr))
        C[k] = Q.reshape(Dl, d, Q.shape[1])
        C[k + 1] = np.tensordot(R, C[k + 1], axes=(1, 0))
    return [np.ascontiguousarray(c) for c in C]


def _right_sweep(cores):
    C = [c.copy() for c in cores]
    for k in range(len(C) - 1, 0, -1):
        Dl, d, Dr = C[k].shape
        Q, R = np.linalg.qr(C[k].reshape(Dl, d * Dr).T)
        C[k] = np.ascontiguousarray(Q.T.reshape(Q.shape[1], d, Dr))
        C[k - 1] = np.tensordot(C[k - 1], R.T, axes=(2, 0))
    return [np.ascontiguousarray(c) for c in C]


def rand_tt(L, d, chi, seed, canon=None, scale=1.0):
    """Gaussian N(0,1) cores with bonds min(d^i, d^(L-i), chi).

    canon: None, "left" (QR sweep left to right) or "right".
    """
    rng = np.random.default_rng(seed)
    D = bond_bounds(L, d, chi)
    cores = [rng.standard_normal((D[k], d, D[k + 1])) for k in range(L)]
    if canon == "left":
        cores = _left_sweep(cores)
    elif canon == "right":
        cores = _right_sweep(cores)
    if scale != 1.0:
        cores[0] = cores[0] * scale
    return cores


def rand_tt_spectral(L, d, chi, seed, decay=1.0):
    """Right-canonical random TT with a j^-decay profile inserted on every bond.

    Each core starts right-orthonormal (QR of a Gaussian (d*D_r) x D_l block,
    transposed); its rows are scaled by a normalised j^-decay profile on its left
    bond; a final right-to-left QR sweep restores right-canonical form, norm 1.
    The profiles of successive bonds compound, so the realised Schmidt spectra
    decay much faster than the profile. With decay = 1 the middle bond gives
    log-log slopes of about -3 (L = 12, chi = 16), -4.7 (L = 16, chi = 64) and
    -6.8 (L = 30, chi = 512); at chi = 512 it spans 1 .. 7e-14.
    """
    rng = np.random.default_rng(seed)
    D = bond_bounds(L, d, chi)
    cores = []
    for k in range(L):
        G = rng.standard_normal((d * D[k + 1], D[k]))
        Q, _ = np.linalg.qr(G)
        core = Q.T.reshape(D[k], d, D[k + 1])
        if k > 0:
            sig = np.arange(1, D[k] + 1, dtype=np.float64) ** (-decay)
            sig /= np.linalg.norm(sig)
            core = sig[:, None, None] * core
        cores.append(core)
    C = _right_sweep(cores)
    C[0] = C[0] / np.linalg.norm(C[0])   # right-canonical: the norm sits in core 1
    return C


def qtt_trig(L, omega, phase=0.0, kind="cos"):
    """Exact rank-2 QTT of cos(omega*x + phase) (or sin) on x_j = j / 2^L, j = 0..2^L-1.

    Site k (1-based) holds bit s_k of j with weight 2^-k, so x = sum_k s_k 2^-k.
    The row vector [cos a, sin a] is rotated by the angle omega*s_k*2^-k per site.
    """
    cores = []
    for k in range(1, L + 1):
        if L == 1:
            c = np.zeros((1, 2, 1))
            for s in range(2):
                a = phase + omega * s * 2.0 ** -k
                c[0, s, 0] = np.cos(a) if kind == "cos" else np.sin(a)
            cores.append(c)
            break
        if k == 1:
            c = np.zeros((1, 2, 2))
            for s in range(2):
                a = phase + omega * s * 2.0 ** -k
                c[0, s] = [np.cos(a), np.sin(a)]
        elif k < L:
            c = np.zeros((2, 2, 2))
            for s in range(2):
                b = omega * s * 2.0 ** -k
                c[:, s, :] = [[np.cos(b), np.sin(b)], [-np.sin(b), np.cos(b)]]
        else:
            c = np.zeros((2, 2, 1))
            for s in range(2):
                b = omega * s * 2.0 ** -k
                if kind == "cos":
                    c[:, s, 0] = [np.cos(b), -np.sin(b)]
                else:
                    c[:, s, 0] = [np.sin(b), np.cos(b)]
        cores.append(c)
    return cores


def qtt_exp(L, a):
    """Exact rank-1 QTT of exp(a*x) on x_j = j / 2^L."""
    return [np.array([[[1.0], [np.exp(a * 2.0 ** -k)]]]).reshape(1, 2, 1) for k in range(1, L + 1)]


def qtt_linear(L, c0=0.0, c1=1.0):
    """Exact rank-2 QTT of c0 + c1*x on x_j = j / 2^L (state vector [1, partial x])."""
    cores = []
    for k in range(1, L + 1):
        t = [0.0, 2.0 ** -k]
        if k == 1:
            c = np.zeros((1, 2, 2))
            for s in range(2):
                c[0, s] = [1.0, t[s]]
        elif k < L:
            c = np.zeros((2, 2, 2))
            for s in range(2):
                c[:, s, :] = [[1.0, t[s]], [0.0, 1.0]]
        else:
            c = np.zeros((2, 2, 1))
            for s in range(2):
                c[:, s, 0] = [c0 + c1 * t[s], c1]
        cores.append(c)
    if L == 1:
        return [np.array([c0, c0 + c1 * 0.5]).reshape(1, 2, 1)]
    return cores


def constant_tt(L, d, c):
    """Rank-1 TT of the constant c."""
    cores = [np.ones((1, d, 1)) for _ in range(L)]
    cores[0] = cores[0] * c
    return cores


def tt_svd(x, L, d, chi=0, rtol=0.0):
    """Encode a dense d^L array as a TT by sequential truncated SVDs (left to right).

    Keeps at most ``chi`` values per bond and drops trailing values whose squared
    sum is below ``rtol^2`` times the total. Returns the cores.
    """
    rest = np.asarray(x, dtype=np.float64).reshape(1, -1)
    cores = []
    Dl = 1
    for k in range(L - 1):
        M = rest.reshape(Dl * d, -1)
        U, s, Vt = np.linalg.svd(M, full_matrices=False)
        r = s.size
        if rtol > 0:
            tail = np.cumsum((s ** 2)[::-1])[::-1]
            ok = np.nonzero(tail < (rtol ** 2) * tail[0])[0]
            if ok.size:
                r = max(1, int(ok[0]))
        if chi:
            r = min(r, chi)
        cores.append(U[:, :r].reshape(Dl, d, r))
        rest = s[:r, None] * Vt[:r]
        Dl = r
    cores.append(rest.reshape(Dl, d, 1))
    return cores


def interleave_2d(field, L):
    """(2^L x 2^L) array -> d=4 quantics vector: site k holds (x bit, y bit) at scale 2^(L-k),
    s_k = 2*bx_k + by_k (coarsest scale first)."""
    f = np.asarray(field).reshape((2,) * L + (2,) * L)
    perm = []
    for k in range(L):
        perm += [k, L + k]
    return f.transpose(perm).reshape(-1)


def turbulence_2d(L=10, chi=64, seed=2000, kmin=4.0, kmax=128.0):
    """Divergence-free 2D synthetic turbulence (u, v) on a periodic 2^L x 2^L grid, as d=4 QTTs.

    Stream-function modes with random phases on integer wavevectors kmin <= |k| <= kmax,
    per-mode |u_hat| ~ |k|^(-4/3) so the shell energy follows E(k) ~ k^(-5/3);
    u = d(psi)/dy, v = -d(psi)/dx (so div u = 0); both scaled by one factor so that
    mean(u^2 + v^2) / 2 = 1 (a common factor keeps the field divergence-free); encoded with
    interleaved bits and compressed by TT-SVD to ``chi``.
    Returns (u_tt, v_tt, u_dense, v_dense).
    """
    n = 2 ** L
    rng = np.random.default_rng(seed)
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    kx, ky = np.meshgrid(k1, k1, indexing="ij")
    kk = np.sqrt(kx ** 2 + ky ** 2)
    band = (kk >= kmin) & (kk <= kmax)
    amp = np.zeros_like(kk)
    amp[band] = kk[band] ** (-4.0 / 3.0 - 1.0)
    phase = rng.uniform(-np.pi, np.pi, size=kk.shape)
    psi_hat = amp * np.exp(1j * phase)
    u = np.real(np.fft.ifft2(1j * ky * psi_hat))
    v = np.real(np.fft.ifft2(-1j * kx * psi_hat))
    scale = np.sqrt(np.mean(u ** 2 + v ** 2) / 2.0)
    u /= scale
    v /= scale
    ut = tt_svd(interleave_2d(u, L), L, 4, chi)
    vt = tt_svd(interleave_2d(v, L), L, 4, chi)
    return ut, vt, u, v


def qtt_mode_3d(L, kvec, amp, phase):
    """Exact rank-2 d=8 QTT of amp*cos(2 pi k.x + phase) on the periodic grid x = j / 2^L per axis.

    Site k holds (x, y, z) bits at scale 2^-k with s = 4*bx + 2*by + bz.
    """
    kx, ky, kz = kvec
    cores = []
    for k in range(1, L + 1):
        ang = np.zeros(8)
        for s in range(8):
            bx, by, bz = (s >> 2) & 1, (s >> 1) & 1, s & 1
            ang[s] = 2.0 * np.pi * (kx * bx + ky * by + kz * bz) * 2.0 ** -k
        if k == 1:
            c = np.zeros((1, 8, 2))
            for s in range(8):
                a = phase + ang[s]
                c[0, s] = [amp * np.cos(a), amp * np.sin(a)]
        elif k < L:
            c = np.zeros((2, 8, 2))
            for s in range(8):
                b = ang[s]
                c[:, s, :] = [[np.cos(b), np.sin(b)], [-np.sin(b), np.cos(b)]]
        else:
            c = np.zeros((2, 8, 1))
            for s in range(8):
                b = ang[s]
                c[:, s, 0] = [np.cos(b), -np.sin(b)]
        cores.append(c)
    return cores


def _tt_sum(ts):
    """Block-diagonal sum of TTs (bond = sum of bonds)."""
    L = len(ts[0])
    out = []
    for k in range(L):
        cs = [t[k] for t in ts]
        if k == 0:
            out.append(np.concatenate(cs, axis=2))
        elif k == L - 1:
            out.append(np.concatenate(cs, axis=0))
        else:
            Dl = sum(c.shape[0] for c in cs)
            Dr = sum(c.shape[2] for c in cs)
            C = np.zeros((Dl, cs[0].shape[1], Dr))
            a = b = 0
            for c in cs:
                C[a:a + c.shape[0], :, b:b + c.shape[2]] = c
                a += c.shape[0]
                b += c.shape[2]
            out.append(C)
    return out


def _round_tt(cores, chi):
    """Compress a TT to bond <= chi: right-to-left QR sweep, then left-to-right truncated SVDs."""
    C = _right_sweep(cores)
    for k in range(len(C) - 1):
        Dl, d, Dr = C[k].shape
        U, s, Vt = np.linalg.svd(C[k].reshape(Dl * d, Dr), full_matrices=False)
        r = min(chi, s.size)
        C[k] = U[:, :r].reshape(Dl, d, r)
        C[k + 1] = np.tensordot(s[:r, None] * Vt[:r], C[k + 1], axes=(1, 0))
    return C


def turbulence_3d_fields(L=10, n_modes=96, seed=4000, chis=None, kmin=4.0, kmax=128.0):
    """Solenoidal 3D random-phase velocity (u_x, u_y, u_z) and its 9 derivatives d_j u_i as d=8 QTTs.

    Built directly in TT form (a dense 2^L-cubed grid would not fit): ``n_modes`` integer
    wavevectors sampled in the shell kmin <= |k| <= kmax with weight ~ E(k) ~ k^(-5/3),
    amplitude vectors orthogonal to k (div u = 0), random phases. Each mode is a rank-2
    QTT; the sums are compressed to the bonds in ``chis`` (12 entries: 3 fields then 9
    derivatives). Derivatives are exact: d/dx_j cos(2pi k.x + t) = 2pi k_j cos(2pi k.x + t + pi/2).
    Returns (fields[3], derivs[3][3]) where derivs[j][i] = d_j u_i.
    """
    rng = np.random.default_rng(seed)
    ks = []
    while len(ks) < n_modes:
        k = rng.integers(-int(kmax), int(kmax) + 1, size=3)
        r = float(np.linalg.norm(k))
        if r < kmin or r > kmax:
            continue
        # accept with probability ~ E(k) / (shell area) ~ k^(-5/3) / k^2, relative to kmin
        if rng.uniform() < (r / kmin) ** (-5.0 / 3.0 - 2.0 + 2.0):
            ks.append(k.astype(np.float64))
    modes = []
    for k in ks:
        e = rng.standard_normal(3)
        e -= e.dot(k) / k.dot(k) * k
        e /= np.linalg.norm(e)
        amp = np.linalg.norm(k) ** (-5.0 / 6.0 - 1.0)
        modes.append((k, e * amp, rng.uniform(-np.pi, np.pi)))
    if chis is None:
        chis = [64] * 12
    fields = []
    for i in range(3):
        parts = [qtt_mode_3d(L, k, a[i], t) for (k, a, t) in modes]
        fields.append(_round_tt(_tt_sum(parts), chis[i]))
    derivs = [[None] * 3 for _ in range(3)]
    idx = 3
    for j in range(3):
        for i in range(3):
            parts = [qtt_mode_3d(L, k, 2.0 * np.pi * k[j] * a[i], t + np.pi / 2) for (k, a, t) in modes]
            derivs[j][i] = _round_tt(_tt_sum(parts), chis[idx])
            idx += 1
    return fields, derivs


def pair_batch(n_pairs, L, d, chi_lo, chi_hi, seed):
    """Batch of random left-canonical TT pairs with chi_A, chi_B ~ U{chi_lo..chi_hi}."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(n_pairs):
        ca = int(rng.integers(chi_lo, chi_hi + 1))
        cb = int(rng.integers(chi_lo, chi_hi + 1))
        A = rand_tt(L, d, ca, seed * 1000 + 2 * p, canon="left")
        B = rand_tt(L, d, cb, seed * 1000 + 2 * p + 1, canon="left")
        out.append((A, B))
    return out
