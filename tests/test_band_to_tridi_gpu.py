"""Device band -> tridiagonal bulge chase (gb_band_to_tridi_d) through the C ABI.

Checks: the tridiagonal's eigenvalues equal the band matrix's (LAPACK via
numpy/scipy) within 50 n u ||B||; the emitted reflectors reproduce T, i.e.
Q2^T B Q2 = T with Q2 formed by the oracle's back-transformation; outputs
agree with the oracle's bulge chase entry by entry (to 1e-9 ||B||: the two
run the same steps with different summation orders, and the reduction is
backward, not forward, stable); exact identities for b = 1 and tridiagonal
input; and the whole two-stage tail on the GPU: chase -> QL (oracle, CPU) ->
gb_trans_ev_tridi_to_band_d gives eigenvectors of B.
"""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_1811_01277_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_01277_gb300 as m
    from paper_1811_01277_gb300 import build
    build.build()
    m.load()
    return m


def lower_band(B, b):
    n = B.shape[0]
    AB = np.zeros((b + 1, n), order="F")
    for d in range(b + 1):
        AB[d, :n - d] = np.diag(B, -d)
    return AB


def chase_gpu(gb, B, b):
    n = B.shape[0]
    dev = torch.device("cuda")
    AB = lower_band(B, b)
    AB_d = torch.from_numpy(np.ascontiguousarray(AB.T)).to(dev)      # (n, b+1) row-major = column-major AB
    cnt = gb.gb_hh_count(n, b)
    d = torch.zeros(n, dtype=torch.float64, device=dev)
    e = torch.zeros(max(n - 1, 1), dtype=torch.float64, device=dev)
    hv = torch.full((max(cnt * b, 1),), np.nan, dtype=torch.float64, device=dev)
    ht = torch.full((max(cnt, 1),), np.nan, dtype=torch.float64, device=dev)
    wsb = gb.gb_band_to_tridi_workspace_bytes(n, b)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream()
    gb.gb_band_to_tridi_d(n, b, AB_d, b + 1, d, e, hv, ht, ws, wsb, st)
    assert gb.gb_trans_ev_query(ws, wsb, st) == 0
    return (d.cpu().numpy(), e.cpu().numpy()[:n - 1], hv.cpu().numpy()[:cnt * b], ht.cpu().numpy()[:cnt])


CASES = [(2, 1), (3, 2), (5, 2), (17, 3), (40, 8), (64, 16), (100, 7), (130, 33), (200, 64), (257, 16), (300, 64)]


@pytest.mark.parametrize("n,b", CASES)
def test_chase_matches_oracle_and_invariants(gb, n, b):
    B = inputs.band_symmetric(n, b, seed=n * 7 + b)
    d, e, hv, ht = chase_gpu(gb, B, b)
    d0, e0, hv0, ht0, _ = oracle.bulge_chase(B, b)
    nrm = np.linalg.norm(B, 2)
    assert np.all(np.isfinite(hv)) and np.all(np.isfinite(ht))
    # eigenvalues preserved (library routines only)
    lam_B = np.linalg.eigvalsh(B)
    lam_T = scipy.linalg.eigvalsh_tridiagonal(d, e) if n > 1 else d
    assert np.abs(np.sort(lam_T) - lam_B).max() <= 50 * n * U * nrm
    # the emitted reflectors reproduce T
    Q = oracle.trans_ev(n, b, hv, ht, np.eye(n))
    T = np.diag(d) + np.diag(e, -1) + np.diag(e, 1)
    assert np.abs(Q.T @ Q - np.eye(n)).max() <= 50 * n * U
    assert np.abs(Q.T @ B @ Q - T).max() <= 50 * n * U * nrm
    # entry by entry against the oracle's chase
    assert np.abs(d - d0).max() <= 1e-9 * nrm
    assert np.abs(e - e0).max() <= 1e-9 * nrm
    assert np.abs(ht - ht0).max() <= 1e-9
    assert np.abs(hv - hv0).max() <= 1e-9


def test_chase_identity_cases(gb):
    n = 50
    B = inputs.band_symmetric(n, 1, seed=2)
    d, e, hv, ht = chase_gpu(gb, B, 1)
    assert np.all(ht == 0) and np.array_equal(d, np.diag(B)) and np.array_equal(e, np.diag(B, -1))
    B = inputs.toeplitz_band(n, 5)
    d, e, hv, ht = chase_gpu(gb, B, 5)
    assert np.all(ht == 0) and np.array_equal(d, np.diag(B)) and np.array_equal(e, np.diag(B, -1))


def test_two_stage_tail_on_gpu(gb):
    """band B -> (GPU chase) -> T -> (oracle QL) -> Z_tri -> (GPU trans_ev) -> eigenvectors of B."""
    n, b = 1024, 32
    B = inputs.band_symmetric(n, b, seed=1)
    d, e, hv, ht = chase_gpu(gb, B, b)
    w, V = oracle.tridiag_ql(d, e)
    dev = torch.device("cuda")
    Zt = torch.from_numpy(np.ascontiguousarray(V.T)).to(dev)
    hv_d, ht_d = torch.from_numpy(hv).to(dev), torch.from_numpy(ht).to(dev)
    wsb = gb.gb_trans_ev_workspace_bytes(n, b, n, 0)
    ws = torch.zeros(max(wsb, 256), dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream()
    gb.gb_trans_ev_tridi_to_band_d(n, b, n, hv_d, ht_d, Zt, n, ws, wsb, st)
    assert gb.gb_trans_ev_query(ws, wsb, st) == 0
    Z = Zt.cpu().numpy().T
    assert np.abs(w - np.linalg.eigvalsh(B)).max() / np.linalg.norm(B, 2) <= 1e-11
    assert np.linalg.norm(B @ Z - Z * w) / np.linalg.norm(B) <= 50 * n * U
    assert np.abs(Z.T @ Z - np.eye(n)).max() <= 50 * n * U


def test_chase_large_eigenvalues(gb):
    """n = 4096, b = 64: eigenvalues of the GPU tridiagonal against LAPACK's
    banded eigensolver on B."""
    n, b = 4096, 64
    B = inputs.band_symmetric(n, b, seed=4096)
    d, e, hv, ht = chase_gpu(gb, B, b)
    lam_T = scipy.linalg.eigvalsh_tridiagonal(d, e)
    lam_B = scipy.linalg.eig_banded(lower_band(B, b), lower=True, eigvals_only=True)
    nrm = np.abs(lam_B).max()
    assert np.abs(np.sort(lam_T) - np.sort(lam_B)).max() <= 50 * n * U * nrm


def chase_gpu_z(gb, B, b):
    n = B.shape[0]
    dev = torch.device("cuda")
    AB = np.zeros((b + 1, n), dtype=np.complex128, order="F")
    for dd in range(b + 1):
        AB[dd, :n - dd] = np.diag(B, -dd)
    AB_d = torch.from_numpy(np.ascontiguousarray(AB.T)).to(dev)
    cnt = gb.gb_hh_count(n, b)
    d = torch.zeros(n, dtype=torch.float64, device=dev)
    e = torch.zeros(max(n - 1, 1), dtype=torch.float64, device=dev)
    hv = torch.full((max(cnt * b, 1),), complex(np.nan, np.nan), dtype=torch.complex128, device=dev)
    ht = torch.full((max(cnt, 1),), complex(np.nan, np.nan), dtype=torch.complex128, device=dev)
    wsb = gb.gb_band_to_tridi_workspace_bytes_z(n, b)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream()
    gb.gb_band_to_tridi_z(n, b, AB_d, b + 1, d, e, hv, ht, ws, wsb, st)
    assert gb.gb_trans_ev_query(ws, wsb, st) == 0
    return (d.cpu().numpy(), e.cpu().numpy()[:n - 1], hv.cpu().numpy()[:cnt * b], ht.cpu().numpy()[:cnt])


@pytest.mark.parametrize("n,b", [(2, 1), (5, 2), (17, 3), (60, 7), (130, 33), (200, 64)])
def test_chase_complex_matches_oracle(gb, n, b):
    B = inputs.band_symmetric(n, b, seed=n + 3 * b, cplx=True)
    d, e, hv, ht = chase_gpu_z(gb, B, b)
    d0, e0, hv0, ht0, _ = oracle.bulge_chase(B, b)
    nrm = np.linalg.norm(B, 2)
    lam_T = scipy.linalg.eigvalsh_tridiagonal(d, e) if n > 1 else d
    assert np.abs(np.sort(lam_T) - np.linalg.eigvalsh(B)).max() <= 50 * n * U * nrm
    Q = oracle.trans_ev(n, b, hv, ht, np.eye(n, dtype=np.complex128))
    T = np.diag(d) + np.diag(e, -1) + np.diag(e, 1)
    assert np.abs(Q.conj().T @ Q - np.eye(n)).max() <= 50 * n * U
    assert np.abs(Q.conj().T @ B @ Q - T).max() <= 50 * n * U * nrm
    assert np.abs(d - d0).max() <= 1e-9 * nrm and np.abs(e - e0).max() <= 1e-9 * nrm
    assert np.abs(hv - hv0).max() <= 1e-9 and np.abs(ht - ht0).max() <= 1e-9


def test_two_stage_tail_complex_on_gpu(gb):
    n, b = 512, 32
    B = inputs.band_symmetric(n, b, seed=2, cplx=True)
    d, e, hv, ht = chase_gpu_z(gb, B, b)
    w, V = oracle.tridiag_ql(d, e)
    dev = torch.device("cuda")
    Zt = torch.from_numpy(np.ascontiguousarray(V.T.astype(np.complex128))).to(dev)
    st = torch.cuda.current_stream()
    wsb = gb.gb_trans_ev_workspace_bytes(n, b, n, 1, None)      # the tensor-core path needs one at n >= 512
    ws = torch.zeros(max(wsb, 256), dtype=torch.uint8, device=dev)
    gb.gb_trans_ev_tridi_to_band_z(n, b, n, torch.from_numpy(hv).to(dev), torch.from_numpy(ht).to(dev), Zt, n,
                                   ws, wsb, st)
    assert gb.gb_trans_ev_query(ws, wsb, st) == 0
    torch.cuda.synchronize()
    Z = Zt.cpu().numpy().T
    assert np.linalg.norm(B @ Z - Z * w) / np.linalg.norm(B) <= 50 * n * U
    assert np.abs(Z.conj().T @ Z - np.eye(n)).max() <= 50 * n * U
