"""Pins of the CPU oracle against facts fixed by the paper and by mathematics (no GPU).

Every test here checks the oracle against something other than itself: exact worked cases, closed
forms (flat, conformally flat and curvilinear-flat metrics), invariants (g^il g_lj = delta, metric
compatibility of the Christoffel symbols), a library inverse and exact rational arithmetic, central
finite differences and torch autograd through an independent transcription.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import gridgen
import oracle

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
PAIRS = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
P = {}
for _p, (_a, _b) in enumerate(PAIRS):
    P[(_a, _b)] = P[(_b, _a)] = _p


def full_sym(arr6):
    """[6, n] packed -> [3, 3, n] full."""
    n = arr6.shape[-1]
    out = np.empty((3, 3, n))
    for a in range(3):
        for b in range(3):
            out[a, b] = arr6[P[(a, b)]]
    return out


def unpack_inputs(x):
    G = full_sym(x[0:6])
    D = np.empty((3, 3, 3, x.shape[1]))          # D[i][j][k] = d_k g_ij
    for a in range(3):
        for b in range(3):
            for c in range(3):
                D[a, b, c] = x[6 + 3 * P[(a, b)] + c]
    K = full_sym(x[24:30])
    alpha = x[30]
    beta = x[31:34]
    B = x[34:43].reshape(3, 3, -1)               # B[i][j] = d_j beta_i
    return G, D, K, alpha, beta, B


def unpack_outputs(y):
    H = full_sym(y[0:6])
    Gam = np.empty((3, 3, 3, y.shape[1]))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                Gam[i, j, k] = y[6 + 6 * i + P[(j, k)]]
    Nb = y[24:33].reshape(3, 3, -1)             # Nb[i][j] = nabla_j beta_i
    dtg = full_sym(y[33:39])
    return H, Gam, Nb, dtg


def pack_inputs(G, D, K, alpha, beta, B):
    n = G.shape[-1]
    x = np.empty((43, n))
    for p, (a, b) in enumerate(PAIRS):
        x[p] = G[a, b]
        x[24 + p] = K[a, b]
        for c in range(3):
            x[6 + 3 * p + c] = D[a, b, c]
    x[30] = alpha
    x[31:34] = beta
    x[34:43] = B.reshape(9, n)
    return x


def normwise(a, b):
    s = np.max(np.abs(b))
    return np.max(np.abs(a - b)) / (s if s > 0 else 1.0)


# ----------------------------------------------------------------------------------------------- inverse

def test_inverse_worked_case_bitwise():
    rows = {}
    with open(os.path.join(GOLD, "inverse_worked_case.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, *v = line.split()
                rows[k] = [float(t) for t in v]
    x = np.zeros((43, 1))
    x[0:6, 0] = rows["g"]
    x[30, 0] = 1.0
    y = oracle.forward(x)
    assert y[0:6, 0].tolist() == rows["ginv"]
    assert oracle.metric_det(x[0:6])[0] == rows["det"][0]


def test_inverse_identity_and_library():
    x = gridgen.random_grid(4096, 0)
    y = oracle.forward(x)
    G = full_sym(x[0:6]).transpose(2, 0, 1)
    H = full_sym(y[0:6]).transpose(2, 0, 1)
    err = np.abs(H @ G - np.eye(3)).max()
    assert err <= 1e-13, err
    Hlib = np.linalg.inv(G)
    assert np.abs(H - Hlib).max() <= 1e-14


def test_inverse_exact_rational_bruteforce():
    """Exact inverse over the rationals of the binary64 inputs on a tiny grid (4^3 points)."""
    x = gridgen.random_grid(64, 7)
    y = oracle.forward(x)
    worst = 0.0
    for t in range(64):
        M = [[Fraction(x[P[(a, b)], t]) for b in range(3)] for a in range(3)]
        # Gauss-Jordan with exact arithmetic
        A = [row[:] + [Fraction(int(a == b)) for b in range(3)] for a, row in enumerate(M)]
        for c in range(3):
            piv = next(r for r in range(c, 3) if A[r][c] != 0)
            A[c], A[piv] = A[piv], A[c]
            inv = 1 / A[c][c]
            A[c] = [v * inv for v in A[c]]
            for r in range(3):
                if r != c and A[r][c] != 0:
                    f = A[r][c]
                    A[r] = [vr - f * vc for vr, vc in zip(A[r], A[c])]
        for p, (a, b) in enumerate(PAIRS):
            exact = A[a][3 + b]
            worst = max(worst, abs(float((Fraction(y[p, t]) - exact) / exact)) if exact != 0 else abs(y[p, t]))
    assert worst <= 8e-16, worst


# ------------------------------------------------------------------------------------------ Christoffel

def test_flat_metric_gives_zero_christoffel_and_listing1_form():
    n = 512
    x = gridgen.random_grid(n, 11)
    x[0:6] = np.array([1, 0, 0, 1, 0, 1.0])[:, None]
    x[6:24] = 0.0
    y = oracle.forward(x)
    assert np.all(y[6:24] == 0.0)                           # Gamma == 0 exactly
    assert np.array_equal(y[24:33], x[34:43])              # nabla beta == d beta exactly
    G, D, K, alpha, beta, B = unpack_inputs(x)
    for p, (i, j) in enumerate(PAIRS):
        # the per-component loop of Listing 1 with db(i,j) = d_j beta_i
        ref = (-2.0 * alpha * K[i, j] + B[j, i]) + B[i, j]
        assert np.array_equal(y[33 + p], ref)


def _conformal_reference(side):
    a = -4.0 + 8.0 * np.arange(side) / (side - 1)
    X0 = np.tile(a, side * side)
    X1 = np.tile(np.repeat(a, side), side)
    X2 = np.repeat(a, side * side)
    X = np.stack([X0, X1, X2])
    e = np.exp(-(X ** 2).sum(0))
    psi = 1 + 0.5 * e
    dpsi = -X * e
    return psi, dpsi


def test_conformally_flat_closed_form():
    side = 16
    x = gridgen.conformal_grid(side)
    y = oracle.forward(x)
    psi, dpsi = _conformal_reference(side)
    _, Gam, Nb, _ = unpack_outputs(y)
    d = np.eye(3)
    for i in range(3):
        for j in range(3):
            for k in range(3):
                ref = 2.0 * (d[i, j] * dpsi[k] + d[i, k] * dpsi[j] - d[j, k] * dpsi[i]) / psi
                assert normwise(Gam[i, j, k], ref) <= 1e-14 or np.abs(Gam[i, j, k] - ref).max() <= 1e-15
    assert np.all(y[24:33] == 0.0) and np.all(y[33:39] == 0.0)  # beta = K = 0 => exact zeros


def test_diagonal_metric_hand_formula():
    n = 1024
    rng = np.random.default_rng(3)
    x = gridgen.random_grid(n, 12)
    gd = rng.uniform(0.5, 2.0, size=(3, n))
    x[0:6] = 0.0
    x[0], x[3], x[5] = gd
    y = oracle.forward(x)
    _, D, _, _, _, _ = unpack_inputs(x)
    _, Gam, _, _ = unpack_outputs(y)
    for i in range(3):
        for j in range(3):
            for k in range(3):
                ref = (D[j, i, k] + D[i, k, j] - D[j, k, i]) / (2.0 * gd[i])
                assert np.abs(Gam[i, j, k] - ref).max() <= 2e-15 * np.abs(ref).max() + 1e-17


def test_spherical_coordinates_textbook():
    """Euclidean space in spherical coordinates (r, theta, phi): g = diag(1, r^2, r^2 sin^2 theta) and the
    standard non-zero symbols G^r_tt = -r, G^r_pp = -r sin^2, G^t_rt = 1/r, G^t_pp = -sin cos,
    G^p_rp = 1/r, G^p_tp = cot theta."""
    r = np.array([0.5, 1.0, 2.0, 3.7])
    th = np.array([0.3, 1.0, 1.2, 2.5])
    n = r.size
    s, c = np.sin(th), np.cos(th)
    G = np.zeros((3, 3, n)); D = np.zeros((3, 3, 3, n))
    G[0, 0] = 1; G[1, 1] = r ** 2; G[2, 2] = (r * s) ** 2
    D[1, 1, 0] = 2 * r; D[2, 2, 0] = 2 * r * s * s; D[2, 2, 1] = 2 * r * r * s * c
    x = pack_inputs(G, D, np.zeros((3, 3, n)), np.ones(n), np.zeros((3, n)), np.zeros((3, 3, n)))
    _, Gam, _, _ = unpack_outputs(oracle.forward(x))
    ref = np.zeros((3, 3, 3, n))
    ref[0, 1, 1] = -r; ref[0, 2, 2] = -r * s * s
    ref[1, 0, 1] = ref[1, 1, 0] = 1 / r; ref[1, 2, 2] = -s * c
    ref[2, 0, 2] = ref[2, 2, 0] = 1 / r; ref[2, 1, 2] = ref[2, 2, 1] = c / s
    assert np.abs(Gam - ref).max() <= 1e-14


def _curvilinear_flat(n, seed):
    """Flat space in the coordinates y with Cartesian x = y + 1/2 C(y, y) (C symmetric in its lower
    pair).  J^a_i = d x^a / d y^i, g_ij = J^a_i J^a_j, d_k g_ij = C^a_ik J^a_j + J^a_i C^a_jk and the
    Christoffel symbols are Gamma^i_jk = (J^-1)^i_a C^a_jk.  A Cartesian affine covector field
    b_a + M_ab x^b (M not symmetric) has, in y, beta_i = J^a_i (b + M x)_a,
    d_j beta_i = C^a_ij (b + M x)_a + J^a_i M_ab J^b_j and covariant derivative nabla_j beta_i =
    J^a_i M_ab J^b_j."""
    rng = np.random.default_rng(seed)
    C = rng.uniform(-0.05, 0.05, size=(3, 3, 3, n))
    C = 0.5 * (C + C.transpose(0, 2, 1, 3))
    y = rng.uniform(-1, 1, size=(3, n))
    J = np.eye(3)[:, :, None] + np.einsum("aikn,kn->ain", C, y)
    xc = y + 0.5 * np.einsum("ajkn,jn,kn->an", C, y, y)
    G = np.einsum("ain,ajn->ijn", J, J)
    D = np.einsum("aikn,ajn->ijkn", C, J) + np.einsum("ain,ajkn->ijkn", J, C)
    Jinv = np.linalg.inv(J.transpose(2, 0, 1)).transpose(1, 2, 0)
    Gam = np.einsum("ian,ajkn->ijkn", Jinv, C)
    b = rng.normal(0, 0.3, size=(3, n))
    M = rng.normal(0, 0.3, size=(3, 3, n))
    cov = b + np.einsum("abn,bn->an", M, xc)
    beta = np.einsum("ain,an->in", J, cov)
    B = np.einsum("aijn,an->ijn", C, cov) + np.einsum("ain,abn,bjn->ijn", J, M, J)
    Nb = np.einsum("ain,abn,bjn->ijn", J, M, J)
    K = rng.normal(0, 0.1, size=(3, 3, n)); K = 0.5 * (K + K.transpose(1, 0, 2))
    alpha = rng.uniform(0.5, 1.5, size=n)
    dtg = -2 * alpha * K + Nb + Nb.transpose(1, 0, 2)
    return pack_inputs(G, D, K, alpha, beta, B), Gam, Nb, dtg


def test_curvilinear_flat_space_closed_forms():
    x, Gam_ref, Nb_ref, dtg_ref = _curvilinear_flat(2000, 5)
    _, Gam, Nb, dtg = unpack_outputs(oracle.forward(x))
    assert normwise(Gam, Gam_ref) <= 1e-13
    assert np.abs(Nb - Nb_ref).max() <= 1e-13        # dbcov[i][j] = nabla_j beta_i (M not symmetric)
    assert np.abs(dtg - dtg_ref).max() <= 1e-13


def test_killing_field_rotation():
    """A rigid rotation of flat space is a Killing field: nabla_i beta_j + nabla_j beta_i = 0, so
    d_t g_ij = -2 alpha K_ij (Eq. 5)."""
    n = 300
    rng = np.random.default_rng(9)
    C = rng.uniform(-0.05, 0.05, size=(3, 3, 3, n)); C = 0.5 * (C + C.transpose(0, 2, 1, 3))
    yv = rng.uniform(-1, 1, size=(3, n))
    J = np.eye(3)[:, :, None] + np.einsum("aikn,kn->ain", C, yv)
    xc = yv + 0.5 * np.einsum("ajkn,jn,kn->an", C, yv, yv)
    w = rng.normal(0, 0.5, size=(3, n))
    M = np.zeros((3, 3, n))
    M[0, 1], M[1, 0], M[0, 2], M[2, 0], M[1, 2], M[2, 1] = -w[2], w[2], w[1], -w[1], -w[0], w[0]
    cov = np.einsum("abn,bn->an", M, xc)
    G = np.einsum("ain,ajn->ijn", J, J)
    D = np.einsum("aikn,ajn->ijkn", C, J) + np.einsum("ain,ajkn->ijkn", J, C)
    beta = np.einsum("ain,an->in", J, cov)
    B = np.einsum("aijn,an->ijn", C, cov) + np.einsum("ain,abn,bjn->ijn", J, M, J)
    K = rng.normal(0, 0.1, size=(3, 3, n)); K = 0.5 * (K + K.transpose(1, 0, 2))
    alpha = rng.uniform(0.5, 1.5, size=n)
    y = oracle.forward(pack_inputs(G, D, K, alpha, beta, B))
    _, _, _, dtg = unpack_outputs(y)
    assert np.abs(dtg - (-2 * alpha * K)).max() <= 1e-13


@pytest.mark.parametrize("seed,stretch", [(17, 1.0), (18, 1.0), (19, 25.0)])
def test_shift_derivative_and_eq5_from_the_lie_derivative(seed, stretch):
    """Christoffel-free closed forms on a generic curved grid.  With the vector beta^k = g^kl beta_l,
    the symmetric part of nabla_j beta_i is half the Lie derivative of the metric along beta^k,
        L_beta g_ij = beta^k d_k g_ij + g_kj d_i beta^k + g_ik d_j beta^k,
    with d_i beta^k = -g^ka (d_i g_ab) g^bl beta_l + g^kl d_i beta_l, and its antisymmetric part is that
    of d_j beta_i (Gamma^k_ij is symmetric in ij).  So nabla_j beta_i = L_ij / 2 + (d_j beta_i -
    d_i beta_j) / 2 and Eq. 5 gives d_t g_ij = -2 alpha K_ij + L_ij.  The inverse here is numpy's.
    stretch > 1 scales the metric's z row and column (and their derivatives) into a stretched,
    anisotropic metric with condition number ~stretch^2."""
    x = gridgen.random_grid(4096, seed)
    G, D, K, alpha, beta, B = unpack_inputs(x)
    s3 = np.array([1.0, 1.0, stretch])
    G = G * s3[:, None, None] * s3[None, :, None]
    D = D * s3[:, None, None, None] * s3[None, :, None, None]
    x = pack_inputs(G, D, K, alpha, beta, B)
    H = np.linalg.inv(G.transpose(2, 0, 1)).transpose(1, 2, 0)
    bu = np.einsum("kln,ln->kn", H, beta)
    dbu = -np.einsum("kan,abin,bln,ln->kin", H, D, H, beta) + np.einsum("kln,lin->kin", H, B)
    L = np.einsum("kn,ijkn->ijn", bu, D) + np.einsum("kjn,kin->ijn", G, dbu) + np.einsum("ikn,kjn->ijn", G, dbu)
    _, _, Nb, dtg = unpack_outputs(oracle.forward(x))
    Nb_ref = 0.5 * L + 0.5 * (B - B.transpose(1, 0, 2))
    dtg_ref = -2.0 * alpha * K + L
    for i in range(3):
        for j in range(3):
            assert normwise(Nb[i, j], Nb_ref[i, j]) <= 1e-14, (i, j)
            assert normwise(dtg[i, j], dtg_ref[i, j]) <= 1e-14, (i, j)


def test_metric_compatibility():
    """nabla_k g_ij = 0:  g_lj Gamma^l_ki + g_il Gamma^l_kj = d_k g_ij for any metric."""
    x = gridgen.random_grid(4096, 0)
    G, D, *_ = unpack_inputs(x)
    _, Gam, _, _ = unpack_outputs(oracle.forward(x))
    lhs = np.einsum("ljn,lkin->ijkn", G, Gam) + np.einsum("iln,lkjn->ijkn", G, Gam)
    assert np.abs(lhs - D).max() <= 2e-15


def test_packing_convention():
    """g stored as (00, 01, 02, 11, 12, 22): a metric whose only off-diagonal entry is g_12 has an
    inverse whose (0,1) and (0,2) entries vanish; Gamma^i_jk lands at gamma[6 i + p(j,k)]."""
    x = np.zeros((43, 1)); x[30] = 1.0
    x[0:6, 0] = [1, 0, 0, 2, 0.5, 3]
    x[6 + 3 * 4 + 0, 0] = 1.0                 # d_0 g_12 = 1, all other derivatives 0
    y = oracle.forward(x)
    assert y[1, 0] == 0 and y[2, 0] == 0 and y[4, 0] != 0
    G, D, *_ = unpack_inputs(x)
    H = np.linalg.inv(G[:, :, 0])
    # Gamma^i_jk = 1/2 g^il (d_k g_jl + d_j g_lk - d_l g_jk) with only d_0 g_12 = d_0 g_21 = 1
    for i in range(3):
        for j in range(3):
            for k in range(j, 3):
                ref = 0.5 * sum(H[i, l] * (D[j, l, k, 0] + D[l, k, j, 0] - D[j, k, l, 0]) for l in range(3))
                assert abs(y[6 + 6 * i + P[(j, k)], 0] - ref) <= 1e-15


@pytest.mark.parametrize("n,threads", [(10007, 4), (5, 8), (1, 3)])
def test_threaded_forward_is_the_same_loop(n, threads):
    """The host-thread split the CPU baseline times (disjoint point ranges, the C loop unchanged on
    each) gives the single call's outputs bit for bit, including ranges left empty."""
    x = gridgen.random_grid(n, 23)
    out = np.full((39, n), np.nan)
    oracle.forward_threaded(x, out, threads)
    assert np.array_equal(out, oracle.forward(x))


def test_argument_errors_and_empty():
    assert oracle.forward(np.zeros((43, 0))).shape == (39, 0)
    with pytest.raises(AssertionError):
        oracle.forward(np.zeros((42, 3)))


# ------------------------------------------------------------------------------------------------ adjoint

def _upstream(n, seed):
    W = gridgen.normal_fields(6, n, seed, 1000)
    V = gridgen.normal_fields(18, n, seed, 1100)
    return [None] * 6 + list(V) + [None] * 9 + list(W)


def _loss_per_point(x, gout):
    y = oracle.forward(x)
    s = np.zeros(x.shape[1])
    for c, g in enumerate(gout):
        if g is not None:
            s += g * y[c]
    return s


def test_adjoint_central_differences():
    n = 512
    x = gridgen.random_grid(n, 3)
    gout = _upstream(n, 3)
    gin = oracle.backward(x, gout)
    h = 1e-6
    for s in range(43):
        xp = x.copy(); xp[s] += h
        xm = x.copy(); xm[s] -= h
        fd = (_loss_per_point(xp, gout) - _loss_per_point(xm, gout)) / (2 * h)
        err = np.abs(fd - gin[s]) / np.maximum(1.0, np.abs(gin[s]))
        assert err.max() <= 1e-7, (s, err.max())


def test_adjoint_all_outputs_and_dot_product_identity():
    """With upstream gradients on all 39 outputs (ginv and dbcov too): <J v, w> = <v, J^T w> per point,
    J v by central differences of the forward along a random direction v."""
    n = 400
    x = gridgen.random_grid(n, 21)
    w = gridgen.normal_fields(39, n, 21, 2000)
    v = gridgen.normal_fields(43, n, 21, 3000)
    gin = oracle.backward(x, list(w))
    h = 1e-6
    Jv = (oracle.forward(x + h * v) - oracle.forward(x - h * v)) / (2 * h)
    lhs = (Jv * w).sum(0)
    rhs = (v * gin).sum(0)
    assert np.abs(lhs - rhs).max() <= 1e-7 * max(1.0, np.abs(rhs).max())


def test_adjoint_against_torch_autograd():
    torch = pytest.importorskip("torch")
    n = 64
    x = gridgen.random_grid(n, 3)
    gout = _upstream(n, 3)
    gin = oracle.backward(x, gout)

    # An independent transcription of the forward chain in plain torch (float64), differentiated by
    # autograd.  Symmetric inputs are expanded from their packed storage so autograd folds both index
    # orders onto the stored element.
    X = torch.tensor(x, dtype=torch.float64, requires_grad=True)
    idx = torch.tensor([[P[(a, b)] for b in range(3)] for a in range(3)])
    Gm = X[0:6][idx]                                        # [3,3,n]
    Dm = X[6:24].reshape(6, 3, n)[idx]                      # [3,3,3,n]: D[a,b,c] = d_c g_ab
    Km = X[24:30][idx]
    al = X[30]
    be = X[31:34]
    Bm = X[34:43].reshape(3, 3, n)
    H = torch.linalg.inv(Gm.permute(2, 0, 1)).permute(1, 2, 0)
    Tm = Dm.permute(1, 0, 2, 3) + Dm.permute(0, 2, 1, 3) - Dm.permute(2, 0, 1, 3)  # T[l,j,k]
    # check the bracket's index placement: T[l,j,k] = D[j,l,k] + D[l,k,j] - D[j,k,l]
    Gam = 0.5 * torch.einsum("iln,ljkn->ijkn", H, Tm)
    Nb = Bm - torch.einsum("kijn,kn->ijn", Gam, be)
    dtg = -2 * al * Km + Nb.permute(1, 0, 2) + Nb
    L = 0.0
    for p, (a, b) in enumerate(PAIRS):
        L = L + (torch.tensor(gout[33 + p]) * dtg[a, b]).sum()
        for i in range(3):
            L = L + (torch.tensor(gout[6 + 6 * i + p]) * Gam[i, a, b]).sum()
    L.backward()
    g_auto = X.grad.numpy()
    for s in range(43):
        assert normwise(gin[s], g_auto[s]) <= 1e-12, s


def test_tensor_bracket_index_placement():
    """The torch transcription's permutes give T[l,j,k] = D[j,l,k] + D[l,k,j] - D[j,k,l]."""
    torch = pytest.importorskip("torch")
    D = torch.randn(3, 3, 3, 1, dtype=torch.float64)
    T = D.permute(1, 0, 2, 3) + D.permute(0, 2, 1, 3) - D.permute(2, 0, 1, 3)
    for l in range(3):
        for j in range(3):
            for k in range(3):
                ref = D[j, l, k] + D[l, k, j] - D[j, k, l]
                assert torch.allclose(T[l, j, k], ref, rtol=0, atol=1e-15)
