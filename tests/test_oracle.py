"""Pins for the CPU oracle against things other than itself: hand-derived
values, closed forms, library routines (numpy / scipy LAPACK), invariants and
brute force.  No GPU needed."""
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_1811_01277_gb300 import inputs

U = 2.0 ** -53
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = np.array([float(v) for v in vals])
    return out


def _dense_reflector(n, r0, v, tau):
    """I - tau v v^H embedded at 0-based row r0 (numpy, for brute force)."""
    H = np.eye(n, dtype=np.result_type(v, tau))
    m = len(v)
    H[r0:r0 + m, r0:r0 + m] -= tau * np.outer(v, v.conj())
    return H


def _q2_brute(n, b, hv, ht):
    """Q2 = H(1,0) H(1,1) ... H(n-1, 0) as an explicit product of dense
    reflectors, each placed at rows s+1+k*b .. (1-based), in generation order."""
    Q = np.eye(n, dtype=hv.dtype)
    idx = 0
    for s in range(1, n):
        for k in range((n - s + b - 1) // b):
            r0 = s + k * b
            ln = min(b, n - r0)
            v = hv[idx * b: idx * b + ln]
            Q = Q @ _dense_reflector(n, r0, v, ht[idx])
            idx += 1
    return Q


# --------------------------------------------------------------------- layout
@pytest.mark.parametrize("n,b", [(1, 1), (2, 1), (2, 5), (3, 2), (10, 3), (64, 64), (100, 7), (257, 32)])
def test_layout_counts_match_enumeration(n, b):
    cnt = 0
    for s in range(1, n):
        r = s + 1
        while r <= n:          # one reflector per block of b rows below s
            assert oracle.hh_index(n, b, s, (r - s - 1) // b) == cnt
            cnt += 1
            r += b
    assert oracle.hh_count(n, b) == cnt
    nk, first = inputs.hh_layout(n, b)
    assert int(nk.sum()) == cnt
    lens = inputs.hh_lengths(n, b)
    # the reflectors of one sweep partition rows s+1..n
    assert int(lens.sum()) == n * (n - 1) // 2
    assert lens.min(initial=1) >= 1 and lens.max(initial=1) <= b


# ---------------------------------------------------------------------- larfg
@pytest.mark.parametrize("m", [0, 1, 3, 17])
@pytest.mark.parametrize("cplx", [False, True])
def test_larfg_annihilates(m, cplx):
    g = np.random.default_rng(11 + m)
    x = g.standard_normal(m) + (1j * g.standard_normal(m) if cplx else 0)
    alpha = g.standard_normal() + (1j * g.standard_normal() if cplx else 0)
    beta, v, tau = oracle.larfg(alpha, x)
    H = np.eye(m + 1, dtype=v.dtype) - tau * np.outer(v, v.conj())
    y = H.conj().T @ np.concatenate([[alpha], x])
    assert abs(np.imag(beta)) == 0.0
    nrm = np.linalg.norm(np.concatenate([[alpha], x]))
    if m == 0 and not cplx:
        assert tau == 0.0 and beta == alpha
    else:
        assert abs(abs(beta) - nrm) <= 8 * U * nrm
        assert np.abs(y - np.concatenate([[beta], np.zeros(m)])).max() <= 16 * U * nrm
    assert np.abs(H.conj().T @ H - np.eye(m + 1)).max() <= 16 * U * (m + 1)
    if not cplx and m > 0:
        assert 1.0 <= tau <= 2.0
    if cplx and m > 0:
        assert 1.0 <= tau.real <= 2.0 and abs(tau - 1.0) <= 1.0 + 1e-15


def test_larfg_special_cases():
    beta, v, tau = oracle.larfg(3.0, [0.0, 0.0])
    assert tau == 0.0 and beta == 3.0
    beta, v, tau = oracle.larfg(0.0, [4.0])      # sign(0) = +1: beta = -||x||
    assert beta == -4.0 and tau == 1.0 and v[1] == 1.0  # v = [1, 4/(0+4)]
    beta, v, tau = oracle.larfg(2.0 + 0j, np.zeros(2, complex))
    assert tau == 0.0
    beta, v, tau = oracle.larfg(1j, np.zeros(0, complex))  # only makes alpha real
    assert beta == -1.0 and abs(tau - (1 + 1j)) < 1e-15


# ----------------------------------------------------------- golden n=3 case
def test_golden_bulge_chase_n3():
    g = _load_golden("bulge_n3_b2.txt")
    n, b = int(g["n"][0]), int(g["b"][0])
    B = g["B"].reshape(n, n, order="F")
    d, e, hv, ht, T = oracle.bulge_chase(B, b)
    assert np.allclose(hv, g["hh_v"], rtol=0, atol=4 * U)
    assert np.allclose(ht, g["hh_tau"], rtol=0, atol=4 * U)
    assert np.allclose(d, g["d"], rtol=0, atol=8 * U)
    assert np.allclose(e, g["e"], rtol=0, atol=8 * U)
    w, V = oracle.tridiag_ql(d, e)
    assert np.allclose(w, g["lambda"], rtol=0, atol=16 * U)
    Q = oracle.trans_ev(n, b, hv, ht, np.eye(n))
    assert np.allclose(Q, g["Q2"].reshape(n, n, order="F"), rtol=0, atol=8 * U)


# --------------------------------------------------------------- bulge chase
CASES = [(5, 2), (17, 3), (40, 8), (64, 16), (33, 32), (70, 9), (31, 1)]


@pytest.mark.parametrize("n,b", CASES)
@pytest.mark.parametrize("cplx", [False, True])
def test_bulge_chase_similarity(n, b, cplx):
    B = inputs.band_symmetric(n, b, seed=n * 31 + b, cplx=cplx)
    d, e, hv, ht, T = oracle.bulge_chase(B, b)
    nrm = np.linalg.norm(B, 2)
    # result is exactly tridiagonal with a real sub-diagonal
    assert np.all(np.tril(T, -2) == 0) and np.all(np.triu(T, 2) == 0)
    Tt = np.diag(d) + np.diag(e, -1) + np.diag(e, 1)
    # eigenvalues preserved (LAPACK via numpy, independent of the oracle)
    lam_B = np.linalg.eigvalsh(B)
    lam_T = np.linalg.eigvalsh(Tt)
    assert np.abs(lam_B - lam_T).max() <= 50 * n * U * nrm
    # Q2 from the back-transformation of I: unitary and Q2^H B Q2 = T
    Q = oracle.trans_ev(n, b, hv, ht, np.eye(n, dtype=B.dtype))
    assert np.abs(Q.conj().T @ Q - np.eye(n)).max() <= 50 * n * U
    assert np.abs(Q.conj().T @ B @ Q - Tt).max() <= 50 * n * U * nrm
    # brute force: explicit product in generation order with the documented rows
    Qb = _q2_brute(n, b, hv, ht)
    assert np.abs(Q - Qb).max() <= 50 * n * U
    if not cplx:
        assert np.all((ht == 0) | ((ht >= 1) & (ht <= 2)))


def test_bulge_chase_b1_is_identity():
    n = 12
    B = inputs.band_symmetric(n, 1, seed=5)
    d, e, hv, ht, T = oracle.bulge_chase(B, 1)
    assert np.all(ht == 0)
    Z = inputs.z_gaussian(n, 5, seed=1)
    assert np.array_equal(oracle.trans_ev(n, 1, hv, ht, Z), Z)
    assert np.array_equal(d, np.diag(B)) and np.array_equal(e, np.diag(B, -1))


@pytest.mark.parametrize("cplx", [False, True])
def test_bulge_chase_tridiagonal_input_gives_identity(cplx):
    n, b = 20, 4
    B = inputs.toeplitz_band(n, b, cplx=cplx)
    d, e, hv, ht, T = oracle.bulge_chase(B, b)
    assert np.all(ht == 0)
    Z = inputs.z_gaussian(n, 3, seed=2, cplx=cplx)
    assert np.array_equal(oracle.trans_ev(n, b, hv, ht, Z), Z)


# ------------------------------------------------------------------ trans_ev
@pytest.mark.parametrize("cplx", [False, True])
def test_trans_ev_single_reflector_closed_form(cplx):
    # n = 3, b = 2: sweep 1 holds one reflector on rows 2..3, sweep 2 one of length 1
    n, b = 3, 2
    g = np.random.default_rng(3)
    v = np.array([1.0, 0.3 + (0.2j if cplx else 0)])
    tau = 1.4 - (0.3j if cplx else 0)
    hv = np.array([v[0], v[1], 1.0, 0.0], dtype=v.dtype)
    ht = np.array([tau, 0.0], dtype=v.dtype)
    Z = g.standard_normal((n, 4)) + (1j * g.standard_normal((n, 4)) if cplx else 0)
    out = oracle.trans_ev(n, b, hv, ht, Z)
    ref = Z.copy()
    ref[1:3] = Z[1:3] - tau * np.outer(v, v.conj() @ Z[1:3])
    assert np.abs(out - ref).max() <= 8 * U


@pytest.mark.parametrize("n,b", [(9, 2), (23, 5), (41, 6)])
@pytest.mark.parametrize("cplx", [False, True])
def test_trans_ev_matches_brute_force_product(n, b, cplx):
    hv, ht = inputs.synthetic_reflectors(n, b, seed=n + b, cplx=cplx)
    Z = inputs.z_gaussian(n, 7, seed=3, cplx=cplx)
    out = oracle.trans_ev(n, b, hv, ht, Z)
    ref = _q2_brute(n, b, hv, ht) @ Z
    assert np.abs(out - ref).max() <= 50 * n * U
    # columns are independent: any subset gives the same columns
    sub = oracle.trans_ev(n, b, hv, ht, Z[:, [5, 1]])
    assert np.array_equal(sub, out[:, [5, 1]])


def test_trans_ev_ldz_larger_than_n():
    n, b, nev = 30, 4, 5
    hv, ht = inputs.synthetic_reflectors(n, b, seed=9)
    Zpad = inputs.z_gaussian(n, nev, seed=4, ldz=n + 3)
    out = oracle.trans_ev(n, b, hv, ht, Zpad)    # passes ldz = n + 3
    ref = oracle.trans_ev(n, b, hv, ht, np.asfortranarray(Zpad[:n]))
    assert np.array_equal(out[:n], ref)
    assert np.array_equal(out[n:], Zpad[n:])     # padding rows untouched


# ------------------------------------------------------------------------ QL
@pytest.mark.parametrize("n", [1, 2, 7, 50, 200])
def test_ql_toeplitz_closed_form(n):
    d = 2.0 * np.ones(n)
    e = -np.ones(n - 1)
    w, V = oracle.tridiag_ql(d, e)
    k = np.arange(1, n + 1)
    lam = 2.0 - 2.0 * np.cos(k * np.pi / (n + 1))
    assert np.abs(w - np.sort(lam)).max() <= 50 * n * U * 4
    j = np.arange(1, n + 1)[:, None]
    Vc = np.sqrt(2.0 / (n + 1)) * np.sin(j * k[None, :] * np.pi / (n + 1))  # columns ascend in lam
    assert np.abs(np.abs(np.sum(V * Vc, axis=0)) - 1.0).max() <= 1e-12


def test_ql_diagonal_and_2x2():
    d = np.array([3.0, -1.0, 2.0, 0.5])
    w, V = oracle.tridiag_ql(d, np.zeros(3))
    assert np.array_equal(w, np.sort(d))
    assert np.array_equal(np.abs(V), np.eye(4)[:, np.argsort(d)])
    a, c, bb = 1.0, 4.0, 2.0
    w, V = oracle.tridiag_ql(np.array([a, c]), np.array([bb]))
    disc = np.sqrt(((a - c) / 2) ** 2 + bb ** 2)
    assert np.allclose(w, [(a + c) / 2 - disc, (a + c) / 2 + disc], rtol=0, atol=8 * U * 5)


@pytest.mark.parametrize("n", [10, 100, 300])
def test_ql_random_against_lapack(n):
    g = np.random.default_rng(n)
    d, e = g.standard_normal(n), g.standard_normal(n - 1)
    w, V = oracle.tridiag_ql(d, e)
    wl = scipy.linalg.eigh_tridiagonal(d, e, eigvals_only=True)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    nrm = np.linalg.norm(T, 2)
    assert np.abs(w - wl).max() <= 50 * n * U * nrm
    assert np.linalg.norm(T @ V - V * w) / np.linalg.norm(T) <= 50 * n * U
    assert np.abs(V.T @ V - np.eye(n)).max() <= 50 * n * U


# -------------------------------------------------------------------- Jacobi
@pytest.mark.parametrize("n", [1, 2, 9, 32])
def test_jacobi_against_lapack(n):
    A = inputs.band_symmetric(n, n, seed=100 + n)
    w, V = oracle.jacobi(A)
    nrm = max(np.linalg.norm(A, 2), 1e-300)
    assert np.abs(w - np.linalg.eigvalsh(A)).max() <= 50 * n * U * nrm
    assert np.linalg.norm(A @ V - V * w) <= 50 * n * U * np.linalg.norm(A)
    assert np.abs(V.T @ V - np.eye(n)).max() <= 50 * n * U


# ---------------------------------------------- full solve: one-stage oracle
def test_sytrd_ql_prescribed_spectrum():
    n = 120
    g = np.random.default_rng(7)
    lam = np.sort(g.uniform(-50, 50, n))
    Q, _ = np.linalg.qr(g.standard_normal((n, n)))
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    d, e, v, tau = oracle.sytrd(A)
    w, Vt = oracle.tridiag_ql(d, e)
    Z = oracle.sytrd_apply(v, tau, Vt)
    nrm = np.linalg.norm(A, 2)
    assert np.abs(w - lam).max() / nrm <= 1e-11
    assert np.linalg.norm(A @ Z - Z * w) / np.linalg.norm(A) <= 50 * n * U
    assert np.abs(Z.T @ Z - np.eye(n)).max() <= 50 * n * U


# --------------------------------------------- two-stage: chase + QL + back
@pytest.mark.parametrize("n,b,cplx", [(16, 3, False), (30, 4, False), (32, 8, False), (28, 5, True)])
def test_two_stage_brute_force_small(n, b, cplx):
    B = inputs.band_symmetric(n, b, seed=900 + n, cplx=cplx)
    d, e, hv, ht, _ = oracle.bulge_chase(B, b)
    w, Vt = oracle.tridiag_ql(d, e)
    Z = oracle.trans_ev(n, b, hv, ht, Vt.astype(B.dtype))
    nrm = np.linalg.norm(B, 2)
    if not cplx:
        wj, Vj = oracle.jacobi(B)
    else:
        wj, Vj = np.linalg.eigh(B)
    assert np.abs(w - wj).max() <= 50 * n * U * nrm
    assert np.linalg.norm(B @ Z - Z * w) / np.linalg.norm(B) <= 50 * n * U
    assert np.abs(Z.conj().T @ Z - np.eye(n)).max() <= 50 * n * U
    # eigenvectors agree with the brute-force ones up to phase (spectrum is simple here)
    assert np.min(np.diff(w)) > 1e-6
    assert np.abs(np.abs(np.sum(Z.conj() * Vj, axis=0)) - 1.0).max() <= 1e-9


def test_two_stage_config_size_n1024():
    n, b = 1024, 32
    B = inputs.band_symmetric(n, b, seed=1)
    d, e, hv, ht, _ = oracle.bulge_chase(B, b)
    w, Vt = oracle.tridiag_ql(d, e)
    Z = oracle.trans_ev(n, b, hv, ht, Vt)
    assert np.abs(w - np.linalg.eigvalsh(B)).max() / np.linalg.norm(B, 2) <= 1e-11
    assert np.linalg.norm(B @ Z - Z * w) / np.linalg.norm(B) <= 50 * n * U
    assert np.abs(Z.T @ Z - np.eye(n)).max() <= 50 * n * U


def test_two_stage_toeplitz_closed_form():
    n, b = 64, 8
    B = inputs.toeplitz_band(n, b)
    d, e, hv, ht, _ = oracle.bulge_chase(B, b)
    w, Vt = oracle.tridiag_ql(d, e)
    Z = oracle.trans_ev(n, b, hv, ht, Vt)
    k = np.arange(1, n + 1)
    assert np.abs(w - np.sort(2 - 2 * np.cos(k * np.pi / (n + 1)))).max() <= 50 * n * U * 4
    assert np.linalg.norm(B @ Z - Z * w) / np.linalg.norm(B) <= 50 * n * U


def test_gapped_uniform_spectrum():
    """The n = 32768 workload's spectrum: in [-1, 1], sorted, n values, and
    10% of them in runs of 8 whose neighbours are 1e-6 apart."""
    lam = inputs.gapped_uniform_spectrum(4096, seed=3)
    assert lam.shape == (4096,) and np.all(np.diff(lam) >= 0)
    assert lam.min() >= -1.0 and lam.max() <= 1.0
    gaps = np.diff(lam)
    close = np.isclose(gaps, 1e-6, rtol=1e-6, atol=0)
    assert close.sum() >= 51 * 7 * 0.95   # 51 clusters x 7 inner gaps (a few may merge with free values)
