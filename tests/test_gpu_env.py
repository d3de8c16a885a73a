"""GPU parity of the environment and adjoint kernels (ttm_inner, ttm_inner3, ttm_backward)
against the oracle's environments, dense gradients and central finite differences."""

import numpy as np
import pytest

import ttgen
from oracle import tt as ott

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_19747_gb300 as pkg
    pkg.build()
    hh = pkg.Handle(0)
    yield hh
    hh.close()


def dev(cores):
    return [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in cores]


def unit(T):
    # left-canonical train scaled to norm 1 (the norm sits in the last core), so that the
    # functionals are O(1) and central differences are meaningful
    T = [c.copy() for c in T]
    T[-1] = T[-1] / np.linalg.norm(T[-1])
    return T


def abs_scale(*ts):
    # sum of |terms| of the dense product, the natural scale of an inner product's rounding
    out = np.ones(1)
    for t in ts:
        out = out * np.abs(ott.dense(t))
    return float(np.sum(out))


@pytest.mark.parametrize("L,d,cx,cy", [(6, 3, 5, 4), (5, 2, 3, 4), (4, 4, 7, 9), (9, 2, 70, 40)])
def test_inner_two_layers(h, L, d, cx, cy):
    import paper_2410_19747_gb300 as pkg
    X = ttgen.rand_tt(L, d, cx, 11 + L)
    Y = ttgen.rand_tt(L, d, cy, 12 + L)
    v = pkg.ttm_inner(h, dev(X), dev(Y))
    ref = ott.inner(X, Y)
    assert abs(v - ref) <= 1e-12 * abs_scale(X, Y)


@pytest.mark.parametrize("L,d,cw,ca,cb", [(6, 3, 4, 5, 3), (5, 2, 3, 4, 2), (4, 4, 6, 5, 7), (8, 2, 70, 16, 12)])
def test_inner_three_layers(h, L, d, cw, ca, cb):
    import paper_2410_19747_gb300 as pkg
    W = ttgen.rand_tt(L, d, cw, 21 + L)
    A = ttgen.rand_tt(L, d, ca, 22 + L)
    B = ttgen.rand_tt(L, d, cb, 23 + L)
    v = pkg.ttm_inner3(h, dev(W), dev(A), dev(B))
    ref = float(np.sum(ott.dense(W) * ott.dense(A) * ott.dense(B)))
    assert abs(v - ref) <= 1e-12 * abs_scale(W, A, B)


@pytest.mark.parametrize("kind", ["inner", "sqdist"])
@pytest.mark.parametrize("L,d,ca,cb,cw", [(6, 3, 4, 3, 5), (5, 4, 5, 4, 3), (7, 2, 6, 5, 4)])
def test_backward_matches_dense_gradients(h, kind, L, d, ca, cb, cw):
    import paper_2410_19747_gb300 as pkg
    A = ttgen.rand_tt(L, d, ca, 31 + L)
    B = ttgen.rand_tt(L, d, cb, 32 + L)
    W = ttgen.rand_tt(L, d, cw, 33 + L)
    val, gA, gB = pkg.ttm_backward(h, kind, dev(A), dev(B), dev(W))
    if kind == "inner":
        ref, rA, rB = ott.grad_inner3_dense(W, A, B)
    else:
        ref, rA, rB = ott.grad_sqdist_dense(A, B, W)
    assert abs(val - ref) <= 1e-10 * max(1.0, abs(ref))
    for got, exp in list(zip(gA, rA)) + list(zip(gB, rB)):
        g = got.cpu().numpy()
        assert g.shape == exp.shape
        assert np.abs(g - exp).max() <= 1e-10 * max(1.0, np.abs(exp).max())


def test_backward_central_differences_config5_shape(h):
    # L=10, d=4, chi=12 (config-5 shape at reduced bond): central differences (h=1e-6) of the
    # dense loss on random entries of every core, for both losses.
    import paper_2410_19747_gb300 as pkg
    L, d, chi = 10, 4, 12
    rng = np.random.default_rng(5000)
    A = unit(ttgen.rand_tt(L, d, chi, 5001, canon="left"))
    B = unit(ttgen.rand_tt(L, d, chi, 5002, canon="left"))
    W = unit(ttgen.rand_tt(L, d, chi, 5003, canon="left"))
    W_sq = [c.copy() for c in W]
    W_sq[-1] = W_sq[-1] * 1e-3     # C of the size of A o B, so no term of g swamps the others
    for kind in ("inner", "sqdist"):
        if kind == "sqdist":
            W = W_sq
        val, gA, gB = pkg.ttm_backward(h, kind, dev(A), dev(B), dev(W))

        def f(A_, B_):
            a, b, w = ott.dense(A_), ott.dense(B_), ott.dense(W)
            if kind == "inner":
                return float(np.sum(w * a * b))
            r = a * b - w
            return float(r @ r)

        hh = 1e-6
        for side, T, G in (("A", A, gA), ("B", B, gB)):
            for k in range(L):
                idx = tuple(rng.integers(0, s) for s in T[k].shape)
                tp = [c.copy() for c in T]
                tm = [c.copy() for c in T]
                tp[k][idx] += hh
                tm[k][idx] -= hh
                fd = (f(tp, B) - f(tm, B)) / (2 * hh) if side == "A" else (f(A, tp) - f(A, tm)) / (2 * hh)
                g = float(G[k].cpu().numpy()[idx])
                scale = float(np.abs(G[k].cpu().numpy()).max())
                assert abs(g - fd) <= 1e-6 * max(scale, 1e-30), (kind, side, k, g, fd, scale)


def test_autograd_function(h):
    import paper_2410_19747_gb300 as pkg
    L, d = 5, 3
    A = dev(ttgen.rand_tt(L, d, 4, 41))
    B = dev(ttgen.rand_tt(L, d, 3, 42))
    W = dev(ttgen.rand_tt(L, d, 5, 43))
    for c in A + B:
        c.requires_grad_(True)
    loss = pkg.product_loss(h, "sqdist", A, B, W)
    (3.0 * loss).backward()
    val, gA, gB = pkg.ttm_backward(h, "sqdist", [c.detach() for c in A], [c.detach() for c in B], W)
    assert abs(loss.item() - val) <= 1e-12 * abs(val)
    for c, g in zip(A + B, gA + gB):
        assert torch.allclose(c.grad, 3.0 * g, rtol=1e-12, atol=0)


def test_env_full_size_config5_inner(h):
    # full config-5 sizes for the three-layer loss: L=20, d=4, chi=128; value against the
    # oracle's three-layer environment, and a sampled directional derivative against
    # central differences of the oracle's value.
    import paper_2410_19747_gb300 as pkg
    L, d, chi = 20, 4, 128
    A = unit(ttgen.rand_tt(L, d, chi, 5011, canon="left"))
    B = unit(ttgen.rand_tt(L, d, chi, 5012, canon="left"))
    W = unit(ttgen.rand_tt(L, d, chi, 5013, canon="left"))
    val, gA, gB = pkg.ttm_backward(h, "inner", dev(A), dev(B), dev(W))
    ref = ott.inner3(W, A, B)
    # |<W, A o B>| <= ||W|| max|A o B| <= 1 for unit trains; rounding is relative to that scale
    assert abs(val - ref) <= 1e-12
    # <W, A o B> is linear in each core: f(A_k + t D) - f(A_k - t D) = 2 t <grad, D> exactly
    rng = np.random.default_rng(7)
    for k in (0, 9, 19):
        D = rng.standard_normal(A[k].shape)
        Ap = [c.copy() for c in A]
        Am = [c.copy() for c in A]
        Ap[k] = Ap[k] + 1e-3 * D
        Am[k] = Am[k] - 1e-3 * D
        fd = (ott.inner3(W, Ap, B) - ott.inner3(W, Am, B)) / 2e-3
        gk = gA[k].cpu().numpy()
        g = float(np.sum(gk * D))
        assert abs(g - fd) <= 1e-9 * (abs(fd) + np.linalg.norm(gk) * np.linalg.norm(D)) + 1e-12


@pytest.mark.parametrize("kind", ["inner", "sqdist"])
def test_backward_recomputed_environments_equal_stored(kind):
    """Below the environment budget only every ceil(sqrt(L))-th left environment is kept and the
    others are recomputed on the way back: the same kernels on the same inputs, so the
    gradients are identical to those of the stored sweep."""
    import paper_2410_19747_gb300 as pkg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    L, d = 16, 2
    A = dev(ttgen.rand_tt(L, d, 8, 61))
    B = dev(ttgen.rand_tt(L, d, 6, 62))
    W = dev(ttgen.rand_tt(L, d, 7, 63))
    hs, hc = pkg.Handle(0), pkg.Handle(0, env_budget_bytes=4096)
    try:
        v0, a0, b0 = pkg.ttm_backward(hs, kind, A, B, W)
        v1, a1, b1 = pkg.ttm_backward(hc, kind, A, B, W)
    finally:
        hs.close()
        hc.close()
    assert v0 == v1
    for x, y in zip(a0 + b0, a1 + b1):
        assert torch.equal(x, y)


def test_sqdist_config5_shape_with_recomputed_environments():
    """||A o B - C||^2 at L = 20, d = 4 (config 5) with chi = 6, the four-layer environments
    recomputed from checkpoints: the value against the oracle's environments, and directional
    derivatives of every third core against central differences of the oracle's value (the
    loss is quadratic in each core, so the difference quotient is exact up to rounding)."""
    import paper_2410_19747_gb300 as pkg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    L, d, chi = 20, 4, 6
    A = unit(ttgen.rand_tt(L, d, chi, 5021, canon="left"))
    B = unit(ttgen.rand_tt(L, d, chi, 5022, canon="left"))
    C = unit(ttgen.rand_tt(L, d, chi, 5023, canon="left"))
    C[-1] = C[-1] * 1e-3
    h = pkg.Handle(0, env_budget_bytes=1 << 14)
    try:
        val, gA, gB = pkg.ttm_backward(h, "sqdist", dev(A), dev(B), dev(C))
    finally:
        h.close()
    ref = ott.sqdist_via_environments(A, B, C)
    assert abs(val - ref) <= 1e-12 * max(1.0, abs(ref))
    rng = np.random.default_rng(9)
    for k in range(0, L, 6):
        for side, T, G in (("A", A, gA), ("B", B, gB)):
            D = rng.standard_normal(T[k].shape)
            tp = [c.copy() for c in T]
            tm = [c.copy() for c in T]
            tp[k] = tp[k] + 1e-3 * D
            tm[k] = tm[k] - 1e-3 * D
            if side == "A":
                fd = (ott.sqdist_via_environments(tp, B, C) - ott.sqdist_via_environments(tm, B, C)) / 2e-3
            else:
                fd = (ott.sqdist_via_environments(A, tp, C) - ott.sqdist_via_environments(A, tm, C)) / 2e-3
            gk = G[k].cpu().numpy()
            g = float(np.sum(gk * D))
            assert abs(g - fd) <= 1e-8 * (abs(fd) + np.linalg.norm(gk) * np.linalg.norm(D)) + 1e-12, (side, k, g, fd)
