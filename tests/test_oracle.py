"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Nothing here re-types the oracle's own formulas: every expected value comes
from a closed form, an invariant, a planted spectrum, a hand computation,
brute force, or LAPACK run on the oracle's covariance.  A final test compiles
deliberately broken copies of the oracle and checks that these pins catch
each one.
"""
import math
import os
import tempfile

import numpy as np
import pytest

import oracle


def sign_normalise(V):
    """Largest-magnitude entry of each column positive (lowest row on ties)."""
    V = np.array(V, dtype=np.float64, copy=True)
    idx = np.argmax(np.abs(V), axis=0)
    sg = np.sign(V[idx, np.arange(V.shape[1])])
    sg[sg == 0] = 1
    return V * sg[None, :]


def rand_sym(rng, B, spread=1.0):
    Wq, _ = np.linalg.qr(rng.standard_normal((B, B)))
    lam = np.sort(rng.uniform(0.1, 10.0, B) ** spread)[::-1]
    return (Wq * lam) @ Wq.T, lam


# ---------------------------------------------------------------- 2x2 (Eqs. 1-5)

CASES_2X2 = [
    (2.0, 1.0, 3.0), (3.0, 1.0, 2.0), (1.0, 0.0, 5.0), (4.0, 2.5, 4.0),
    (1.0, 1e-9, 1.0 + 1e-3), (1e6, -3.0, 1e-6), (-2.0, 7.0, 0.5), (5.0, -1e-12, 5.0),
]


@pytest.mark.parametrize("a,b,c", CASES_2X2)
def test_rotation_zeroes_offdiag_and_gives_closed_form_eigenvalues(a, b, c):
    cs, sn = oracle.rotation(a, c, b)
    assert abs(cs * cs + sn * sn - 1.0) < 4e-16
    # the angle of Eq. 3 is the small root: |t| <= 1, |alpha| <= pi/4
    assert abs(sn) <= cs + 1e-15
    P = np.array([[cs, sn], [-sn, cs]])          # Eq. 1 / Eq. 6 layout
    A = np.array([[a, b], [b, c]])
    Bm = P.T @ A @ P                              # Eq. 1 with P^-1 = P^T
    scale = max(abs(a), abs(b), abs(c))
    assert abs(Bm[0, 1]) <= 4e-16 * scale
    mid, rad = (a + c) / 2.0, math.hypot((a - c) / 2.0, b)
    got = sorted([Bm[0, 0], Bm[1, 1]])
    assert got[0] == pytest.approx(mid - rad, rel=1e-14, abs=1e-15 * scale)
    assert got[1] == pytest.approx(mid + rad, rel=1e-14, abs=1e-15 * scale)


def test_rotation_matches_eq3_where_eq3_is_well_conditioned():
    # Eq. 2-5 literally: m = 2b/(c-a), t = (-1 + sqrt(1+m^2))/m
    for a, b, c in [(2.0, 1.0, 3.0), (1.0, 0.7, 4.0), (3.0, -2.0, 1.0), (0.5, 3.0, 0.25)]:
        m = 2 * b / (c - a)
        t = (-1.0 + math.sqrt(1.0 + m * m)) / m
        cs_expect = 1.0 / math.sqrt(1.0 + t * t)
        cs, sn = oracle.rotation(a, c, b)
        assert cs == pytest.approx(cs_expect, rel=1e-14)
        assert sn == pytest.approx(t * cs_expect, rel=1e-13)


def test_rotation_equal_diagonal_is_45_degrees_and_zero_offdiag_is_identity():
    cs, sn = oracle.rotation(3.0, 3.0, 2.0)
    assert cs == pytest.approx(math.sqrt(0.5), rel=1e-15)
    assert sn == pytest.approx(math.sqrt(0.5), rel=1e-15)
    assert oracle.rotation(1.0, 2.0, 0.0) == (1.0, 0.0)


def test_jacobi_2x2_single_rotation():
    A = np.array([[4.0, 9.0], [9.0, 21.0]])
    Ak, V, info = oracle.jacobi(A)
    assert info["rotations"] == 1 and info["sweeps"] == 1
    lam = sorted(np.diag(Ak))
    assert lam[0] == pytest.approx((25 - math.sqrt(613)) / 2, rel=1e-14)
    assert lam[1] == pytest.approx((25 + math.sqrt(613)) / 2, rel=1e-14)


# ---------------------------------------------------------------- tiny cube by hand

def test_tiny_cube_by_hand():
    # N = 3 pixels, B = 2 bands.  mu = (3, 6); X = [[-2,-4],[0,-1],[2,5]];
    # C = X^T X / 2 = [[4, 9], [9, 21]]; eigenvalues (25 +- sqrt(613)) / 2.
    Y = np.array([[1.0, 2.0], [3.0, 5.0], [5.0, 11.0]])
    r = oracle.pca_fit(Y, 2)
    assert np.allclose(r["mu"], [3.0, 6.0], rtol=0, atol=1e-15)
    C = oracle.covariance(Y)
    assert np.array_equal(C, np.array([[4.0, 9.0], [9.0, 21.0]]))
    l1, l2 = (25 + math.sqrt(613)) / 2, (25 - math.sqrt(613)) / 2
    assert r["lam"][0] == pytest.approx(l1, rel=1e-14)
    assert r["lam"][1] == pytest.approx(l2, rel=1e-13)
    # eigenvector of l1: (9, l1 - 4) normalised, positive largest entry
    v = np.array([9.0, l1 - 4.0])
    v /= np.linalg.norm(v)
    assert np.allclose(r["V"][:, 0], v, atol=1e-14)
    X = Y - np.array([3.0, 6.0])
    assert np.allclose(r["Q"][:, 0], X @ v, atol=1e-13)


# ---------------------------------------------------------------- 3x3 brute force

def cubic_eigs(A):
    """Eigenvalues of a symmetric 3x3 by the trigonometric solution of the
    characteristic cubic (closed form, independent of any iteration)."""
    p1 = A[0, 1] ** 2 + A[0, 2] ** 2 + A[1, 2] ** 2
    q = np.trace(A) / 3.0
    p2 = (A[0, 0] - q) ** 2 + (A[1, 1] - q) ** 2 + (A[2, 2] - q) ** 2 + 2 * p1
    p = math.sqrt(p2 / 6.0)
    Bm = (A - q * np.eye(3)) / p
    r = np.clip(np.linalg.det(Bm) / 2.0, -1.0, 1.0)
    phi = math.acos(r) / 3.0
    l1 = q + 2 * p * math.cos(phi)
    l3 = q + 2 * p * math.cos(phi + 2 * math.pi / 3)
    return sorted([l1, 3 * q - l1 - l3, l3], reverse=True)


def charpoly(A, lam):
    M = A - lam * np.eye(3)
    return (M[0, 0] * (M[1, 1] * M[2, 2] - M[1, 2] * M[2, 1])
            - M[0, 1] * (M[1, 0] * M[2, 2] - M[1, 2] * M[2, 0])
            + M[0, 2] * (M[1, 0] * M[2, 1] - M[1, 1] * M[2, 0]))


def bisect_eigs(A, grid=20001):
    r = np.max(np.sum(np.abs(A), axis=1))
    xs = np.linspace(-r - 1, r + 1, grid)
    fs = np.array([charpoly(A, x) for x in xs])
    roots = []
    for i in range(grid - 1):
        if fs[i] == 0:
            roots.append(xs[i])
        elif fs[i] * fs[i + 1] < 0:
            lo, hi, flo = xs[i], xs[i + 1], fs[i]
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                fm = charpoly(A, mid)
                if (fm < 0) == (flo < 0):
                    lo, flo = mid, fm
                else:
                    hi = mid
            roots.append(0.5 * (lo + hi))
    return sorted(roots, reverse=True)


@pytest.mark.parametrize("seed", range(6))
def test_3x3_against_characteristic_polynomial(seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((3, 3))
    A = G + G.T
    Ak, V, info = oracle.jacobi(A)
    lam = np.sort(np.diag(Ak))[::-1]
    ref1 = cubic_eigs(A)
    ref2 = bisect_eigs(A)
    scale = np.abs(A).max()
    assert np.allclose(lam, ref1, atol=1e-13 * scale)
    assert len(ref2) == 3 and np.allclose(lam, ref2, atol=1e-12 * scale)


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("B", [5, 16, 33, 64])
@pytest.mark.parametrize("ordering", [oracle.ROW_CYCLIC, oracle.ROUND_ROBIN, oracle.ODD_EVEN,
                                      oracle.CLASSICAL, oracle.GREEDY])
def test_jacobi_invariants(B, ordering):
    rng = np.random.default_rng(100 + B)
    A, lam_true = rand_sym(rng, B)
    Ak, V, info = oracle.jacobi(A, tol=1e-15, ordering=ordering)
    assert info["status"] == oracle.OK
    lam = np.diag(Ak)
    nA = np.linalg.norm(A)
    assert abs(np.trace(A) - lam.sum()) <= 1e-13 * nA
    assert abs(nA ** 2 - (lam ** 2).sum()) <= 1e-13 * nA ** 2
    assert np.linalg.norm(V.T @ V - np.eye(B)) <= 1e-13
    assert np.linalg.norm(A @ V - V * lam[None, :]) <= 1e-12 * nA
    assert np.allclose(np.sort(lam)[::-1], lam_true, rtol=1e-12)


def test_orderings_agree():
    rng = np.random.default_rng(7)
    Y = rng.standard_normal((400, 21)) @ rng.standard_normal((21, 21))
    r0 = oracle.pca_fit(Y, 5)
    for o in (oracle.ROUND_ROBIN, oracle.ODD_EVEN, oracle.CLASSICAL, oracle.GREEDY):
        r = oracle.pca_fit(Y, 5, ordering=o)
        assert np.allclose(r["lam"], r0["lam"], rtol=1e-12, atol=1e-13 * r0["lam"][0])
        assert np.allclose(r["V"], r0["V"], atol=1e-10)


def test_classical_rotation_zeroes_the_largest_element_and_off_drops_by_twice_its_square():
    """Classical pivot (Sec. 4.2 stage 4.1): each rotation zeroes the largest
    off-diagonal element, and a Jacobi rotation lowers off(A)^2 by exactly 2 a_pq^2
    (the textbook identity of the Jacobi method)."""
    rng = np.random.default_rng(31)
    A, _ = rand_sym(rng, 9)
    cur = A.copy()
    off2 = lambda M: float((M ** 2).sum() - (np.diag(M) ** 2).sum())
    for step in range(6):
        iu = np.triu_indices(9, 1)
        k = int(np.argmax(np.abs(cur[iu])))
        p, q = iu[0][k], iu[1][k]
        big = cur[p, q]
        nxt, V, nrot = oracle.jacobi_steps(cur, oracle.CLASSICAL, 1)
        assert nrot == 1
        assert nxt[p, q] == 0.0 and nxt[q, p] == 0.0
        assert abs(off2(cur) - off2(nxt) - 2 * big * big) <= 1e-13 * (A ** 2).sum()
        assert np.linalg.norm(V.T @ V - np.eye(9)) <= 1e-14
        cur = nxt


def test_greedy_iteration_takes_row_wise_disjoint_pairs_above_threshold():
    """Greedy selection (Code 5.3.1): one iteration takes, row by row, the pairs
    above the threshold whose indices are still free -- here (0,1), (2,3), (4,5) --
    and leaves rows and columns 6, 7 untouched; the next iteration may take a
    pair it skipped, but never a pair zeroed earlier in the sweep."""
    B = 8
    A = np.diag(np.arange(1.0, B + 1.0)) + 0.01
    for (i, j, v) in [(0, 1, 5.0), (0, 2, 4.0), (2, 3, 3.0), (4, 5, 2.0), (1, 3, 1.5)]:
        A[i, j] = A[j, i] = v
    A1, V, nrot = oracle.jacobi_steps(A, oracle.GREEDY, 1, thr=1.0)
    assert nrot == 3
    for (i, j) in [(0, 1), (2, 3), (4, 5)]:
        assert A1[i, j] == 0.0
    assert A1[6, 7] == A[6, 7] and A1[6, 6] == A[6, 6] and A1[7, 7] == A[7, 7]
    assert abs(A1[0, 2]) > 1.0                      # rotated, not yet taken
    A2, _, nrot2 = oracle.jacobi_steps(A, oracle.GREEDY, 2, thr=1.0)
    assert nrot2 > 3
    assert A2[6, 7] == A[6, 7]


# ---------------------------------------------------------------- planted spectrum

def planted_cube(rng, N, B, s, offset_scale=10.0):
    G = rng.standard_normal((N, B))
    G -= G.mean(axis=0, keepdims=True)
    U, _ = np.linalg.qr(G)                       # centred, orthonormal columns
    Wq, _ = np.linalg.qr(rng.standard_normal((B, B)))
    m = rng.uniform(0.0, offset_scale, B)
    Y = (U * s[None, :]) @ Wq.T + m[None, :]
    return Y, Wq, m


def test_planted_spectrum_recovered_exactly():
    rng = np.random.default_rng(11)
    N, B = 3000, 24
    s = 3.0 * 0.8 ** np.arange(B)
    Y, W, m = planted_cube(rng, N, B, s)
    r = oracle.pca_fit(Y, 6)
    assert np.allclose(r["mu"], m, atol=1e-13)
    lam_true = s ** 2 / (N - 1)
    assert np.allclose(r["lam"], lam_true, rtol=1e-11)
    assert np.allclose(r["V"], sign_normalise(W), atol=1e-9)


# ---------------------------------------------------------------- LAPACK / numpy

@pytest.mark.parametrize("N,B", [(500, 7), (2000, 48), (300, 103)])
def test_covariance_and_eigs_vs_lapack(N, B):
    rng = np.random.default_rng(N + B)
    Y = rng.standard_normal((N, B)) @ rng.uniform(0, 1, (B, B)) + 5.0
    mu = oracle.band_means(Y)
    assert np.allclose(mu, Y.mean(axis=0), rtol=0, atol=1e-13 * np.abs(Y).max())
    C = oracle.covariance(Y, mu)
    Cn = np.cov(Y, rowvar=False)
    assert np.allclose(C, Cn, rtol=0, atol=1e-12 * np.abs(Cn).max())
    r = oracle.pca_fit(Y, 3)
    w, v = np.linalg.eigh(C)
    w, v = w[::-1], v[:, ::-1]
    assert np.allclose(r["lam"], w, rtol=0, atol=1e-12 * w[0])
    gaps = np.abs(np.diff(w)) / w[0]
    ok = np.concatenate([[gaps[0]], np.minimum(gaps[:-1], gaps[1:]), [gaps[-1]]]) > 1e-6
    assert np.allclose(r["V"][:, ok], sign_normalise(v)[:, ok], atol=1e-8)


# ---------------------------------------------------------------- projection

def test_projection_properties():
    rng = np.random.default_rng(5)
    Y = rng.standard_normal((1500, 12)) @ rng.standard_normal((12, 12)) + 3.0
    r = oracle.pca_fit(Y, 5)
    Q = r["Q"]
    assert np.abs(Q.mean(axis=0)).max() <= 1e-12 * np.abs(Q).max()
    G = Q.T @ Q / (Y.shape[0] - 1)
    assert np.allclose(G, np.diag(r["lam"][:5]), rtol=0, atol=1e-11 * r["lam"][0])


# ---------------------------------------------------------------- special cases

def test_diagonal_input_needs_no_rotation():
    A = np.diag([3.0, 1.0, 7.0, 2.0])
    Ak, V, info = oracle.jacobi(A, tol=1e-14)
    assert info["sweeps"] == 0 and info["rotations"] == 0
    assert np.array_equal(V, np.eye(4))
    lam, Vs = oracle.sort_sign(np.diag(Ak), V)
    assert list(lam) == [7.0, 3.0, 2.0, 1.0]
    assert np.array_equal(Vs[:, 0], [0, 0, 1, 0]) and np.array_equal(Vs[:, 3], [0, 1, 0, 0])


def test_constant_cube_is_all_zero():
    Y = np.full((50, 6), 2.5)
    r = oracle.pca_fit(Y, 2)
    assert np.all(r["lam"] == 0.0) and r["sweeps"] == 0 and np.all(r["Q"] == 0.0)
    assert np.array_equal(r["V"], np.eye(6))


def test_rank_one_cube():
    rng = np.random.default_rng(2)
    u = rng.standard_normal(400)
    w = rng.standard_normal(9)
    w /= np.linalg.norm(w)
    Y = np.outer(u, w) + 1.0
    r = oracle.pca_fit(Y, 1)
    uc = u - u.mean()
    assert r["lam"][0] == pytest.approx(uc @ uc / 399, rel=1e-12)
    assert np.all(np.abs(r["lam"][1:]) <= 1e-13 * r["lam"][0])
    assert np.allclose(r["V"][:, 0], sign_normalise(w[:, None])[:, 0], atol=1e-12)


def test_band_permutation_and_pixel_permutation_and_scaling():
    rng = np.random.default_rng(9)
    Y = rng.standard_normal((800, 10)) @ rng.standard_normal((10, 10))
    r = oracle.pca_fit(Y, 4)
    perm = rng.permutation(10)
    rp = oracle.pca_fit(Y[:, perm], 4)
    assert np.allclose(rp["lam"], r["lam"], rtol=1e-12)
    assert np.allclose(rp["V"], r["V"][perm, :], atol=1e-10)
    px = rng.permutation(800)
    rx = oracle.pca_fit(Y[px], 4)
    assert np.allclose(rx["lam"], r["lam"], rtol=1e-12)
    assert np.allclose(rx["Q"], r["Q"][px], atol=1e-10)
    rs = oracle.pca_fit(3.0 * Y, 4)
    assert np.allclose(rs["lam"], 9.0 * r["lam"], rtol=1e-12)
    assert np.allclose(rs["V"], r["V"], atol=1e-10)


def test_sort_is_descending_with_ties_by_index_and_sign_rule():
    lam = np.array([1.0, 5.0, 1.0, 5.0, 3.0])
    V = np.eye(5)
    V[:, 2] = [0.0, -0.6, -0.8, 0.0, 0.0]        # largest |.| negative -> flipped
    V[:, 4] = [0.5, 0.0, 0.0, -0.5, 0.0]          # tie in |.|: lowest row decides (positive)
    l2, V2 = oracle.sort_sign(lam, V)
    assert list(l2) == [5.0, 5.0, 3.0, 1.0, 1.0]
    assert np.array_equal(V2[:, 0], np.eye(5)[:, 1])
    assert np.array_equal(V2[:, 1], np.eye(5)[:, 3])
    assert np.array_equal(V2[:, 2], [0.5, 0.0, 0.0, -0.5, 0.0])
    assert np.array_equal(V2[:, 3], np.eye(5)[:, 0])
    assert np.array_equal(V2[:, 4], [0.0, 0.6, 0.8, 0.0, 0.0])


def test_stop_rule_is_relative_to_the_norm():
    # Jacobi angles depend only on ratios, so scaling A by a power of two
    # scales every iterate exactly; a stop rule relative to ||A||_F must then
    # take the same sweeps and reach the same off(A)/||A||_F (reading of the
    # paper's "all off-diagonal elements smaller than the stop factor").
    rng = np.random.default_rng(4)
    A, _ = rand_sym(rng, 20)
    ref = oracle.jacobi(A, tol=1e-12, sweeps_max=40)[2]
    assert ref["status"] == oracle.OK
    for c in (2.0 ** 30, 2.0 ** -30):
        info = oracle.jacobi(c * A, tol=1e-12, sweeps_max=40)[2]
        assert info["status"] == oracle.OK
        assert info["sweeps"] == ref["sweeps"]
        assert info["off_rel"] == ref["off_rel"]


def test_nonconvergence_returns_last_iterate():
    rng = np.random.default_rng(3)
    A, _ = rand_sym(rng, 30)
    Ak, V, info = oracle.jacobi(A, tol=1e-15, sweeps_max=1)
    assert info["status"] == oracle.ERR_NOCONV and info["sweeps"] == 1
    assert info["off_rel"] > 1e-15
    assert np.linalg.norm(V.T @ V - np.eye(30)) < 1e-13
    assert np.linalg.norm(V.T @ A @ V - Ak) < 1e-12 * np.linalg.norm(A)


def test_nonfinite_input_is_reported():
    Y = np.ones((10, 3))
    Y[4, 1] = np.nan
    with pytest.raises(oracle.OracleError):
        oracle.pca_fit(Y, 1)
    Y[4, 1] = np.inf
    with pytest.raises(oracle.OracleError):
        oracle.band_means(Y)


# ---------------------------------------------------------------- the pins catch mistakes

MUTANTS = {
    "classical pivot takes the smallest element": (
        "if (a > best) { best = a; *pp = i; *pq = j; found = 1; }",
        "if (a > 0.0 && (!found || a < best)) { best = a; *pp = i; *pq = j; found = 1; }"),
    "greedy ignores used indices": (
        "if (used[i] || used[j] || zeroed[(size_t)i * B + j]) continue;",
        "if (zeroed[(size_t)i * B + j]) continue;"),
    "row update sign": ("A[(size_t)p * B + k] = c * apk - s * aqk;",
                        "A[(size_t)p * B + k] = c * apk + s * aqk;"),
    "column update sign": ("A[(size_t)k * B + q] = s * akp + c * akq;",
                           "A[(size_t)k * B + q] = -s * akp + c * akq;"),
    "eigenvector transposed": ("double vkp = V[(size_t)k * B + p], vkq = V[(size_t)k * B + q];",
                               "double vkp = V[(size_t)p * B + k], vkq = V[(size_t)q * B + k];"),
    "angle sign": ("double tau = (aqq - app) / (2.0 * apq);",
                   "double tau = (app - aqq) / (2.0 * apq);"),
    "normalise by N": ("const double inv = 1.0 / (double)(N - 1);",
                       "const double inv = 1.0 / (double)(N);"),
    "mean dropped": ("for (int b = 0; b < B; ++b) x[b] = Y[n * B + b] - mu[b];",
                     "for (int b = 0; b < B; ++b) x[b] = Y[n * B + b];"),
    "ascending sort": ("while (j >= 0 && lam[idx[j]] < lam[v])",
                       "while (j >= 0 && lam[idx[j]] > lam[v])"),
    "projection index": ("s += (Y[n * B + b] - mu[b]) * V[(size_t)b * B + j];",
                         "s += (Y[n * B + b] - mu[b]) * V[(size_t)j * B + b];"),
    "stop rule absolute": ("if (fro == 0.0 || off <= tol * fro)",
                           "if (fro == 0.0 || off <= tol)"),
    "adjoint gap sign": ("M[(size_t)i * B + j] / gap : 0.0;", "M[(size_t)i * B + j] / -gap : 0.0;"),
    "adjoint dQ not centred": ("s += (dQ[n * k + j] - mdq[j]) * V[(size_t)c * B + j];",
                               "s += dQ[n * k + j] * V[(size_t)c * B + j];"),
    "adjoint covariance factor": ("const double f = 2.0 / (double)(N - 1);",
                                  "const double f = 1.0 / (double)(N - 1);"),
    "adjoint M transposed": ("s += V[(size_t)b * B + i] * dVk[(size_t)b * k + j];",
                             "s += V[(size_t)i * B + b] * dVk[(size_t)b * k + j];"),
}


# ---------------------------------------------------------------- adjoint of the path

FD_SIDE, FD_BANDS, FD_K = 32, 48, 10      # the separately generated FD sub-cube


def _adjoint_case(seed=5):
    """A 32 x 32 pixel x 48 band planted cube (s_i = 0.9^(i-1) over 11
    components above a 0.05 floor) with its upstream gradients.  Central
    differences only pin the adjoint where the eigen-pairs it differentiates
    are simple, so the realised gaps of the top k + 1 eigenvalues are asserted
    to be at least 1e-3 of lambda_1 (first-order perturbation theory divides
    by them)."""
    import synth
    c = synth.gradient_cube(seed=seed, side=FD_SIDE, bands=FD_BANDS, comps=FD_K + 1, k=FD_K)
    Y = c.Y.astype(np.float64)
    lam = oracle.pca_fit(Y, c.k, tol=1e-14, project_q=False)["lam"]
    gaps = (lam[:c.k + 1] - lam[1:c.k + 2]) / lam[0]
    assert gaps.min() >= 1e-3, gaps
    rng = np.random.default_rng(seed + 100)
    dQ = rng.standard_normal((c.N, c.k))
    dl = rng.standard_normal(c.B)
    return Y, c.k, dQ, dl


def _loss(Y, k, dQ, dl):
    r = oracle.pca_fit(Y, k, tol=1e-14)
    return float(np.sum(dQ * r["Q"]) + np.dot(dl, r["lam"]))


def _fd_check(entries, directions, seed=5):
    """dL/dY of L = <dQ, Q(Y)> + <dlam, lam(Y)> against central finite
    differences (h = 1e-6, FP64) at `entries` distinct random entries and along
    `directions` random directions.  The forward pass's sign rule is the same
    on both sides of every difference (no column's largest entry changes rank
    at this step size), so the differences see one smooth branch."""
    Y, k, dQ, dl = _adjoint_case(seed)
    r = oracle.pca_fit(Y, k, tol=1e-14)
    adj = oracle.backward(Y, k, r["mu"], r["lam"], r["V"], dQ, dl, gap_eps=1e-9)
    scale = np.abs(adj).max()
    h = 1e-6
    rng = np.random.default_rng(7)
    N, B = Y.shape
    flat = rng.choice(N * B, size=entries, replace=False)
    worst = 0.0
    for e in flat:
        n, b = divmod(int(e), B)
        Yp, Ym = Y.copy(), Y.copy()
        Yp[n, b] += h
        Ym[n, b] -= h
        fd = (_loss(Yp, k, dQ, dl) - _loss(Ym, k, dQ, dl)) / (2 * h)
        worst = max(worst, abs(fd - adj[n, b]) / scale)
        assert abs(fd - adj[n, b]) <= 2e-7 * scale, (n, b, fd, adj[n, b])
    for _ in range(directions):
        D = rng.standard_normal(Y.shape)
        fd = (_loss(Y + h * D, k, dQ, dl) - _loss(Y - h * D, k, dQ, dl)) / (2 * h)
        # error bound on the scale of |<adj, D>| <= ||adj|| ||D|| (Cauchy-Schwarz)
        assert abs(fd - np.sum(adj * D)) <= 1e-6 * np.linalg.norm(adj) * np.linalg.norm(D), fd
    return worst


def test_adjoint_matches_central_differences():
    """The adjoint pin at full size: 256 entries and 8 directional derivatives
    of the 32 x 32 x 48 sub-cube."""
    worst = _fd_check(entries=256, directions=8)
    print(f"largest entry error / max|dY|: {worst:.2e}")


def test_adjoint_special_cases():
    """dQ = 0 and dlam = e_i: dlam_i/dY = 2/(N-1) X v_i v_i^T (the derivative of
    a simple eigenvalue of C = X^T X/(N-1)); all-zero gradients give zero."""
    Y, k, dQ, dl = _adjoint_case(6)
    r = oracle.pca_fit(Y, k, tol=1e-14)
    N, B = Y.shape
    X = Y - r["mu"][None, :]
    for i in (0, 3):
        e = np.zeros(B)
        e[i] = 1.0
        adj = oracle.backward(Y, k, r["mu"], r["lam"], r["V"], np.zeros((N, k)), e)
        v = r["V"][:, i]
        expect = 2.0 / (N - 1) * np.outer(X @ v, v)
        assert np.abs(adj - expect).max() <= 1e-12 * np.abs(expect).max()
    z = oracle.backward(Y, k, r["mu"], r["lam"], r["V"], np.zeros((N, k)))
    assert np.all(z == 0.0)
    # a gradient of Q only: the centring makes every column of dY sum to what
    # X S contributes, and the V_k^T term has zero column sums
    adj = oracle.backward(Y, k, r["mu"], r["lam"], r["V"], dQ)
    assert np.abs(adj.sum(axis=0)).max() <= 1e-10 * np.abs(adj).max() * N


def _pins_pass() -> bool:
    """The cheapest pins, run against whatever oracle build is current."""
    try:
        test_tiny_cube_by_hand()
        for a, b, c in CASES_2X2[:4]:
            test_rotation_zeroes_offdiag_and_gives_closed_form_eigenvalues(a, b, c)
        for seed in range(2):
            test_3x3_against_characteristic_polynomial(seed)
        test_jacobi_invariants(16, oracle.ROW_CYCLIC)
        test_jacobi_invariants(16, oracle.CLASSICAL)
        test_jacobi_invariants(16, oracle.GREEDY)
        test_classical_rotation_zeroes_the_largest_element_and_off_drops_by_twice_its_square()
        test_greedy_iteration_takes_row_wise_disjoint_pairs_above_threshold()
        test_planted_spectrum_recovered_exactly()
        test_projection_properties()
        test_sort_is_descending_with_ties_by_index_and_sign_rule()
        test_nonconvergence_returns_last_iterate()
        test_covariance_and_eigs_vs_lapack(500, 7)
        test_rank_one_cube()
        test_stop_rule_is_relative_to_the_norm()
        test_adjoint_special_cases()
        _fd_check(entries=24, directions=2)
    except (AssertionError, oracle.OracleError):
        return False
    return True


def test_pins_pass_on_the_real_oracle():
    assert _pins_pass()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name):
    old, new = MUTANTS[name]
    src = oracle.source()
    assert src.count(old) == 1, f"mutation anchor for {name!r} not found exactly once"
    with tempfile.TemporaryDirectory() as d:
        so = oracle.compile_variant(src.replace(old, new), os.path.join(d, "mutant.so"))
        with oracle.using(so):
            assert not _pins_pass(), f"no pin failed with planted mistake: {name}"
