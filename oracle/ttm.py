"""The paper's TTM algorithm, step by step, on the CPU in float64. Test infrastructure only.

Follows Sec. II.B of arXiv:2410.19747 (Eq. tensor, Eq. contract, Eq. eps, Fig. 1)
in the paper's order and notation:

  phi = K^{s_1} ... K^{s_N}      (the TT "A")
  psi = M^{w_1} ... M^{w_N}      (the TT "B")
  Omega = Pi^{e_1} ... Pi^{e_N}  (the product A o B)

Readings where the paper is silent or ambiguous:
  A1  psi enters the concatenated chain reversed, each carriage with its two bond
      legs exchanged: slot N+j holds M_{N+1-j}^T, i.e. Mt[a, s, b] = M[b, s, a].
  A2  after a Swap the singular values go into the carriage that carries the
      moving psi leg, so the gauge centre travels with the mover and sits on the
      right-most carriage of every next pair (the statement that accompanies
      Eq. eps); the other new carriage is right-orthonormal (V^T).
  A3  after each Contract the centre is moved by QR decompositions rightwards
      through Pi_i ... Pi_N into the next mover.
  A4  two caps beyond Eq. eps: ``chi_max`` caps every Swap SVD, ``chi_out`` caps
      the output through a final left-to-right TT-SVD rounding (only run if a
      bond of Omega exceeds it).
  A5  the truncation rule keeps the smallest k >= 1 whose discarded tail obeys
      sum_{j>k} lam_j^2 < eps * sum_j lam_j^2 (strict); eps = 0 keeps every
      singular value including zeros; then k = min(k, cap).
"""

import numpy as np

from . import tt as _tt


def truncation_rank(lam, eps, cap=0):
    """Rank kept under Eq. eps plus an optional cap (reading A5). Returns (k, w).

    lam: singular values sorted descending. w is the discarded weight
    sum_{j>k} lam_j^2 (absolute, not relative).
    """
    lam2 = np.asarray(lam, dtype=np.float64) ** 2
    n = lam2.size
    total = float(lam2.sum())
    k = n
    if total > 0.0 and eps > 0.0:
        # tail[kk] = sum of lam2[kk:], the weight dropped when kk values are kept
        tail = np.concatenate([np.cumsum(lam2[::-1])[::-1], [0.0]])
        for kk in range(1, n + 1):
            if tail[kk] < eps * total:
                k = kk
                break
    if total == 0.0:
        k = 1
    if cap and cap > 0:
        k = min(k, int(cap))
    k = max(1, min(k, n))
    return k, float(lam2[k:].sum())


def contract(K, M):
    """Contract (Eq. contract): Pi^e_{mn} = sum_{s,w} (sum_a K^s_{ma} M^w_{an}) delta_{s w e}.

    K: (D_l, d, D_a), M: (D_a, d, D_r) -> Pi: (D_l, d, D_r). The local COPY tensor
    delta is built explicitly so the code reads as the equation.
    """
    d = K.shape[1]
    delta = np.zeros((d, d, d))
    for s in range(d):
        delta[s, s, s] = 1.0
    return np.einsum('msa,awn,swe->men', K, M, delta, optimize=True)


def swap(X, Y, eps=0.0, cap=0):
    """Swap (Fig. 1C, Eq. eps): exchange two adjacent carriages X (left) and Y (right).

    1. contract the shared bond: Theta[l, s, t, r] = sum_m X[l, s, m] Y[m, t, r];
    2. permute the two physical legs: -> [l, t, s, r];
    3. reshape to the matrix [(l, t), (s, r)] and take its SVD;
    4. drop the smallest singular values by Eq. eps (reading A5);
    5. the left carriage (now carrying Y's leg t) takes U Lambda (reading A2);
       the right one (carrying X's leg s) takes V^T and is right-orthonormal.
    Returns (newY, newX, lam, k, w).
    """
    Dl, d1, Dm = X.shape
    Dm2, d2, Dr = Y.shape
    assert Dm == Dm2
    theta = np.tensordot(X, Y, axes=(2, 0))          # [l, s, t, r]
    theta = theta.transpose(0, 2, 1, 3)              # [l, t, s, r]
    mat = theta.reshape(Dl * d2, d1 * Dr)
    U, lam, Vt = np.linalg.svd(mat, full_matrices=False)
    k, w = truncation_rank(lam, eps, cap)
    newY = (U[:, :k] * lam[:k]).reshape(Dl, d2, k)
    newX = Vt[:k].reshape(k, d1, Dr)
    return newY, newX, lam, k, w


def qr_move(C, Cnext):
    """Move the gauge centre one carriage right: C = Q R, Q stays, R joins Cnext."""
    Dl, d, Dr = C.shape
    Q, R = np.linalg.qr(C.reshape(Dl * d, Dr))
    return Q.reshape(Dl, d, Q.shape[1]), np.tensordot(R, Cnext, axes=(1, 0))


def tt_round(T, eps=0.0, cap=0):
    """TT-SVD rounding (Oseledets 2011, cited in Sec. II.A): right-canonicalise, then
    truncate every bond left to right with the rule of ``truncation_rank``.

    Returns (cores, discarded weights). Pinned by: untruncated rounding is exact;
    error <= sqrt(sum w) (orthogonal truncations); tests.
    """
    C = _tt.right_canonical(T)
    ws = []
    for k in range(len(C) - 1):
        Dl, d, Dr = C[k].shape
        U, lam, Vt = np.linalg.svd(C[k].reshape(Dl * d, Dr), full_matrices=False)
        r, w = truncation_rank(lam, eps, cap)
        ws.append(w)
        C[k] = U[:, :r].reshape(Dl, d, r)
        C[k + 1] = np.tensordot(lam[:r, None] * Vt[:r], C[k + 1], axes=(1, 0))
    return C, ws


def conventional(A, B, eps=0.0, cap=0):
    """Conventional route of Sec. II.A: exact Kronecker cores (Eq. carriageXi) then rounding."""
    return tt_round(_tt.hadamard_kron(A, B), eps, cap)


def ttm(A, B, eps=0.0, chi_max=0, chi_out=0):
    """TTM product Omega = A o B by the swap-and-contract sweep of Sec. II.B.

    Returns (cores of Omega, report dict). The report holds the schedule counts,
    every discarded weight, the maximum bond seen in the chain after every Swap
    and Contract, and the bound sum_j sqrt(w_j) on ||Omega - A o B|| (reading of
    the global-truncation statement next to Eq. eps).
    """
    N = len(A)
    assert len(B) == N and N >= 1
    # a1: phi left-canonical; psi left-canonical in its own order, then reversed with
    # its bond legs exchanged, which makes the reversed part right-orthonormal.
    K = _tt.left_canonical(A)
    Mc = _tt.left_canonical(B)
    Mt = [m.transpose(2, 1, 0).copy() for m in Mc]   # Mt[j] = M_{j+1}^T

    rep = {"n_swaps": 0, "n_contracts": 0, "n_qr": 0, "weights": [], "bond_trace": [],
           "max_bond": 0}

    def note(chain_bonds):
        m = max(chain_bonds)
        rep["max_bond"] = max(rep["max_bond"], m)
        return m

    Pi = [None] * (N + 1)   # 1-indexed sites
    # a2: the two carriages of site N are adjacent across the size-1 junction.
    Pi[N] = contract(K[N - 1], Mt[N - 1])
    rep["n_contracts"] += 1
    rep["bond_trace"].append(note([Pi[N].shape[0], Pi[N].shape[2]] +
                                  [k.shape[2] for k in K[:N - 1]] +
                                  [m.shape[0] for m in Mt[:N - 1]]))
    for i in range(N - 1, 0, -1):
        mover = Mt[i - 1]
        # a3: centre from Pi_{i+1} through Pi_N into the mover (QR gauge moves).
        for j in range(i + 1, N + 1):
            if j < N:
                Pi[j], Pi[j + 1] = qr_move(Pi[j], Pi[j + 1])
            else:
                Pi[j], mover = qr_move(Pi[j], mover)
            rep["n_qr"] += 1
        # a4 + a5: the mover passes Pi_N, ..., Pi_{i+1} (i-1 swaps in the paper's count).
        for j in range(N, i, -1):
            mover, Pi[j], lam, k, w = swap(Pi[j], mover, eps, chi_max)
            rep["n_swaps"] += 1
            rep["weights"].append(w)
            note([k])
        # a6: the mover is now next to K_i.
        Pi[i] = contract(K[i - 1], mover)
        rep["n_contracts"] += 1
        rep["bond_trace"].append(note([p.shape[2] for p in Pi[i:N + 1]] +
                                      [k.shape[2] for k in K[:i - 1]] +
                                      [m.shape[0] for m in Mt[:i - 1]] + [1]))
    out = Pi[1:]
    # a7: optional final rounding to chi_out. Omega is right-canonical with the
    # centre on Pi_1, so a left-to-right truncated SVD sweep is optimal per bond.
    if chi_out and chi_out > 0 and max(_tt.bonds_of(out)) > chi_out:
        for k in range(N - 1):
            Dl, d, Dr = out[k].shape
            U, lam, Vt = np.linalg.svd(out[k].reshape(Dl * d, Dr), full_matrices=False)
            r, w = truncation_rank(lam, eps, chi_out)
            rep["weights"].append(w)
            out[k] = U[:, :r].reshape(Dl, d, r)
            out[k + 1] = np.tensordot(lam[:r, None] * Vt[:r], out[k + 1], axes=(1, 0))
    rep["discarded_weight"] = float(sum(rep["weights"]))
    rep["err_bound"] = float(sum(np.sqrt(max(w, 0.0)) for w in rep["weights"]))
    rep["bonds"] = _tt.bonds_of(out)
    return out, rep
