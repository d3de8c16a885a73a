"""Tensor-train basics for the oracle (float64, numpy). Test infrastructure only.

Conventions (shared by every function here, and by the C-ABI):
  * a TT of length L is a list of cores; core k has shape (D_k, d, D_{k+1}),
    row-major, with D_0 = D_L = 1 (Eq. TT and Eq. bond of the paper);
  * the full tensor is indexed (s_1, ..., s_L) with s_1 the slowest index
    (C order), so ``dense(T).reshape((d,)*L)[s_1, ..., s_L]`` is the product
    of matrices T_1[:, s_1, :] ... T_L[:, s_L, :].

Parity pins for this file live in ``tests/test_oracle_tt.py``.
"""

import numpy as np


def bonds_of(cores):
    """Bond dimensions [D_0, ..., D_L] of a TT (Eq. bond layout)."""
    return [int(cores[0].shape[0])] + [int(c.shape[2]) for c in cores]


def bond_rule(L, d, chi):
    """Maximal bonds D_i = min(d^i, d^(L-i), chi) (Eq. bond, generalised from d=2 to d).

    Pinned by: chi_max = d^floor(L/2) makes the TT exact (Sec. II), checked in tests.
    """
    out = []
    for i in range(L + 1):
        v = min(d ** i, d ** (L - i))
        if chi and chi > 0:
            v = min(v, chi)
        out.append(int(v))
    return out


def dense(cores):
    """Brute-force contraction of a TT to its full d^L vector (Eq. TT, O1).

    Contracts left to right: the running matrix has rows = (s_1..s_k) and
    columns = the open bond. Pinned by: rank-1 TTs (an outer product of vectors)
    and the closed-form QTT fields in tests.
    """
    acc = np.ones((1, 1))
    for c in cores:
        Dl, d, Dr = c.shape
        acc = (acc @ c.reshape(Dl, d * Dr)).reshape(-1, Dr)
    return acc.reshape(-1)


def hadamard_kron(A, B):
    """Exact product TT with Kronecker cores Pi^s = K^s (x) M^s (Eq. carriageXi, O2).

    Bond (ia, ib) -> ia * D_B + ib. Pinned by: dense(hadamard_kron(A,B)) equals
    dense(A) * dense(B) elementwise (tests).
    """
    out = []
    for Ka, Mb in zip(A, B):
        Dla, d, Dra = Ka.shape
        Dlb, d2, Drb = Mb.shape
        assert d == d2
        P = np.empty((Dla * Dlb, d, Dra * Drb))
        for s in range(d):
            P[:, s, :] = np.kron(Ka[:, s, :], Mb[:, s, :])
        out.append(P)
    return out


def left_canonical(cores):
    """QR sweep left to right: cores 1..L-1 left-orthonormal, the norm moves to core L.

    Each core is reshaped to (D_l*d) x D_r and split by a reduced Householder QR
    (LAPACK via numpy); R is merged into the next core. Bonds can shrink to
    min(D_l*d, D_r). Represents the same tensor (pinned by dense() in tests).
    """
    T = [np.array(c, dtype=np.float64, copy=True) for c in cores]
    for k in range(len(T) - 1):
        Dl, d, Dr = T[k].shape
        Q, R = np.linalg.qr(T[k].reshape(Dl * d, Dr))
        T[k] = Q.reshape(Dl, d, Q.shape[1])
        T[k + 1] = np.tensordot(R, T[k + 1], axes=(1, 0))
    return T


def right_canonical(cores):
    """QR sweep right to left (LQ of each core): cores 2..L right-orthonormal."""
    T = [np.array(c, dtype=np.float64, copy=True) for c in cores]
    for k in range(len(T) - 1, 0, -1):
        Dl, d, Dr = T[k].shape
        Q, R = np.linalg.qr(T[k].reshape(Dl, d * Dr).T)
        T[k] = Q.T.reshape(Q.shape[1], d, Dr)
        T[k - 1] = np.tensordot(T[k - 1], R.T, axes=(2, 0))
    return T


def inner(X, Y):
    """<X, Y> through the two-layer environment E_k[a, b] (the "." product used in Gamma, Sec. III).

    E_0 = [[1]]; E_k[a, b] = sum_{a', b', s} E_{k-1}[a', b'] X_k[a', s, a] Y_k[b', s, b].
    Pinned by: equals dense(X) . dense(Y) (tests).
    """
    E = np.ones((1, 1))
    for Xk, Yk in zip(X, Y):
        E = np.einsum('ab,asc,bsd->cd', E, Xk, Yk, optimize=True)
    return float(E[0, 0])


def norm(X):
    """||X||_2: left-orthogonalise a copy; the norm is that of the last core."""
    T = left_canonical(X)
    return float(np.linalg.norm(T[-1]))


def difference(X, Y):
    """TT of X - Y with block-stacked cores (bond D_X + D_Y), no cancellation by squaring."""
    L = len(X)
    out = []
    for k in range(L):
        Xk, Yk = X[k], Y[k]
        ax, d, bx = Xk.shape
        ay, _, by = Yk.shape
        if L == 1:
            out.append(Xk - Yk)
        elif k == 0:
            out.append(np.concatenate([Xk, -Yk], axis=2))
        elif k == L - 1:
            out.append(np.concatenate([Xk, Yk], axis=0))
        else:
            C = np.zeros((ax + ay, d, bx + by))
            C[:ax, :, :bx] = Xk
            C[ax:, :, bx:] = Yk
            out.append(C)
    return out


def diff_norm(X, Y):
    """||X - Y||_2 via the block-stacked difference TT, left-orthogonalised."""
    return norm(difference(X, Y))


def inner3(W, A, B):
    """<W, A o B> = sum_s W(s) A(s) B(s) through the three-layer environment.

    L_k[w, a, b] = sum L_{k-1}[w', a', b'] W_k[w', s, w] A_k[a', s, a] B_k[b', s, b],
    all three layers joined on the same physical index s (the COPY tensor).
    Pinned by: equals sum(dense(W) * dense(A) * dense(B)) (tests).
    """
    E = np.ones((1, 1, 1))
    for Wk, Ak, Bk in zip(W, A, B):
        d = Wk.shape[1]
        # contract the B layer, then the A layer on the same s, then the W layer on the same s
        T1 = np.tensordot(E, Bk, axes=(2, 0))                     # [x, a, s, d]
        En = np.zeros((Wk.shape[2], Ak.shape[2], Bk.shape[2]))
        for s in range(d):
            T2 = np.tensordot(Ak[:, s, :], T1[:, :, s, :], axes=(0, 1))   # [c, x, d]
            En += np.tensordot(Wk[:, s, :], T2, axes=(0, 1))               # [w, c, d]
        E = En
    return float(E[0, 0, 0])


def _project_dense_gradient(Gfull, X, k):
    """Project a dense gradient dF/dX_full onto core k of the TT X.

    dF/dX_k[a', s, a] = sum_{p, q} Lk[p, a'] Gfull[p, s, q] Rk[a, q], where Lk is
    the (d^(k) x D_k) matrix of cores 1..k-1 and Rk the (D_{k+1} x d^(L-k-1))
    matrix of cores k+1..L (chain rule on the linear map X_k -> X_full).
    """
    L = len(X)
    d = X[0].shape[1]
    left = np.ones((1, 1))
    for c in X[:k]:
        Dl, _, Dr = c.shape
        left = (left @ c.reshape(Dl, d * Dr)).reshape(-1, Dr)
    right = np.ones((1, 1))
    for c in reversed(X[k + 1:]):
        Dl, _, Dr = c.shape
        right = (c.reshape(Dl * d, Dr) @ right).reshape(Dl, -1)
    G = Gfull.reshape(left.shape[0], d, right.shape[1])
    return np.einsum('pa,psq,bq->asb', left, G, right, optimize=True)


def grad_inner3_dense(W, A, B):
    """Gradients of f = <W, A o B> w.r.t. every core of A and of B (O6, dense).

    dF/dA_full = W o B and dF/dB_full = W o A, then projected onto each core.
    Pinned by central finite differences in tests.
    """
    w, a, b = dense(W), dense(A), dense(B)
    gA = [_project_dense_gradient(w * b, A, k) for k in range(len(A))]
    gB = [_project_dense_gradient(w * a, B, k) for k in range(len(B))]
    return float(np.sum(w * a * b)), gA, gB


def grad_sqdist_dense(A, B, C):
    """Gradients of g = ||A o B - C||^2 w.r.t. every core of A and B (O6, dense).

    dG/dA_full = 2 (A o B - C) o B and dG/dB_full = 2 (A o B - C) o A.
    Pinned by central finite differences in tests.
    """
    a, b, c = dense(A), dense(B), dense(C)
    r = a * b - c
    gA = [_project_dense_gradient(2.0 * r * b, A, k) for k in range(len(A))]
    gB = [_project_dense_gradient(2.0 * r * a, B, k) for k in range(len(B))]
    return float(np.dot(r, r)), gA, gB


def sqdist_via_environments(A, B, C):
    """||A o B - C||^2 = <A o B, A o B> - 2 <C, A o B> + ||C||^2 with small environments.

    <A o B, A o B> uses the four-layer environment (A, A, B, B) on the shared
    physical index; only for small bonds (chi^4 memory).
    """
    E = np.ones((1, 1, 1, 1))
    for Ak, Bk in zip(A, B):
        E = np.einsum('pqrt,psa,qsb,rsc,tsd->abcd', E, Ak, Ak, Bk, Bk, optimize=True)
    ab2 = float(E.reshape(-1)[0])
    return ab2 - 2.0 * inner3(C, A, B) + inner(C, C)
