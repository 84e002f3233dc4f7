"""FP64 products of the solver (gb_dgemm, gb_dsymm, gb_dsyr2k, gb_dsyrk:
DFMA-tiled kernels) against numpy's float64 products on ragged shapes,
with padded leading dimensions, the split-K path (workspace given) and the
unsplit path, and the triangle / beta = 0 contracts (entries the call must
not read are NaN, entries it must not write keep a sentinel)."""
import numpy as np
import pytest

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


def dev_cm(X, ld=None):
    """Column-major device copy of X (rows x cols) with leading dimension ld,
    padding rows filled with NaN."""
    r, c = X.shape
    ld = ld or max(r, 1)
    buf = np.full((max(c, 1), ld), np.nan)
    buf[:c, :r] = X.T
    return torch.from_numpy(buf).cuda(), ld


def host_cm(T, rows, cols):
    return T.cpu().numpy()[:cols, :rows].T


def bound(k, absprod, absc=0.0):
    """Elementwise rounding-error bound of a length-k dot product plus the
    scaled C term, gamma_{k+2} (|alpha| |opA||opB| + |beta| |C|), times 2."""
    g = (k + 2) * U / (1 - (k + 2) * U)
    return 2 * g * (absprod + absc) + 1e-300


SHAPES = [(1, 1, 1), (37, 29, 13), (64, 64, 64), (65, 63, 70), (200, 77, 131), (513, 64, 1000), (64, 300, 2500)]


@pytest.mark.parametrize("m,n,k", SHAPES)
@pytest.mark.parametrize("ta", "NT")
@pytest.mark.parametrize("tb", "NT")
@pytest.mark.parametrize("split", [False, True])
def test_dgemm(gb, m, n, k, ta, tb, split):
    g = np.random.default_rng(m * 1000 + n * 10 + k)
    A = g.uniform(-1, 1, (k, m) if ta == "T" else (m, k))
    B = g.uniform(-1, 1, (n, k) if tb == "T" else (k, n))
    C0 = g.uniform(-1, 1, (m, n))
    alpha, beta = 0.75, -1.25
    Ad, lda = dev_cm(A, A.shape[0] + 3)
    Bd, ldb = dev_cm(B, B.shape[0] + 1)
    Cd, ldc = dev_cm(C0, m + 2)
    wsb = gb.gb_dgemm_workspace_bytes(m, n) if split else 0
    ws = torch.empty(max(wsb, 8), dtype=torch.uint8, device="cuda") if split else None
    gb.gb_dgemm(ta, tb, m, n, k, alpha, Ad, lda, Bd, ldb, beta, Cd, ldc, ws, wsb, torch.cuda.current_stream())
    opA = A.T if ta == "T" else A
    opB = B.T if tb == "T" else B
    ref = alpha * (opA @ opB) + beta * C0
    got = host_cm(Cd, m, n)
    assert np.all(np.abs(got - ref) <= bound(k, abs(alpha) * (np.abs(opA) @ np.abs(opB)), abs(beta) * np.abs(C0)))
    # padding rows of C untouched (still NaN)
    assert np.all(np.isnan(Cd.cpu().numpy()[:n, m:ldc]))


def test_dgemm_beta_zero_does_not_read_c(gb):
    m, n, k = 70, 90, 33
    g = np.random.default_rng(3)
    A, B = g.uniform(-1, 1, (m, k)), g.uniform(-1, 1, (k, n))
    Ad, lda = dev_cm(A)
    Bd, ldb = dev_cm(B)
    Cd = torch.full((n, m), float("nan"), dtype=torch.float64, device="cuda")
    gb.gb_dgemm("N", "N", m, n, k, 1.0, Ad, lda, Bd, ldb, 0.0, Cd, m, None, 0, torch.cuda.current_stream())
    assert np.all(np.abs(host_cm(Cd, m, n) - A @ B) <= bound(k, np.abs(A) @ np.abs(B)))


@pytest.mark.parametrize("side", "LR")
@pytest.mark.parametrize("m,n", [(1, 1), (45, 17), (64, 64), (130, 70), (700, 64), (64, 700)])
def test_dsymm_reads_lower_only(gb, side, m, n):
    g = np.random.default_rng(m + 7 * n)
    s = m if side == "L" else n
    S = g.uniform(-1, 1, (s, s))
    S = S + S.T
    S_lower = np.tril(S) + np.triu(np.full((s, s), np.nan), 1)
    B = g.uniform(-1, 1, (m, n))
    C0 = g.uniform(-1, 1, (m, n))
    Sd, lds = dev_cm(S_lower, s + 1)
    Bd, ldb = dev_cm(B, m + 3)
    Cd, ldc = dev_cm(C0, m)
    wsb = gb.gb_dgemm_workspace_bytes(m, n)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    gb.gb_dsymm(side, m, n, -0.5, Sd, lds, Bd, ldb, 2.0, Cd, ldc, ws, wsb, torch.cuda.current_stream())
    ref = -0.5 * (S @ B if side == "L" else B @ S) + 2.0 * C0
    absprod = 0.5 * (np.abs(S) @ np.abs(B) if side == "L" else np.abs(B) @ np.abs(S))
    assert np.all(np.abs(host_cm(Cd, m, n) - ref) <= bound(s, absprod, 2.0 * np.abs(C0)))


@pytest.mark.parametrize("n,k", [(1, 1), (50, 3), (64, 64), (129, 64), (300, 200), (1000, 64)])
def test_dsyr2k_and_dsyrk_lower_triangle(gb, n, k):
    g = np.random.default_rng(n * 31 + k)
    A, B = g.uniform(-1, 1, (n, k)), g.uniform(-1, 1, (n, k))
    C0 = g.uniform(-1, 1, (n, n))
    sentinel = 12345.0
    C0u = np.tril(C0) + np.triu(np.full((n, n), sentinel), 1)
    Ad, lda = dev_cm(A, n + 1)
    Bd, ldb = dev_cm(B, n + 2)
    Cd, ldc = dev_cm(C0u, n + 1)
    gb.gb_dsyr2k(n, k, -1.0, Ad, lda, Bd, ldb, 1.0, Cd, ldc, torch.cuda.current_stream())
    got = host_cm(Cd, n, n)
    ref = C0 - (A @ B.T + B @ A.T)
    low = np.tril(np.ones((n, n), dtype=bool))
    b1 = bound(2 * k, np.abs(A) @ np.abs(B).T + np.abs(B) @ np.abs(A).T, np.abs(C0))
    assert np.all(np.abs(got[low] - ref[low]) <= b1[low])
    assert np.all(got[~low] == sentinel)
    # syrk: C = A2^T A2 (A2 k x n), beta = 0 on a NaN-filled lower triangle
    A2 = g.uniform(-1, 1, (k, n))
    A2d, lda2 = dev_cm(A2, k + 3)
    Cd2, ldc2 = dev_cm(np.tril(np.full((n, n), np.nan)) + np.triu(np.full((n, n), sentinel), 1), n)
    gb.gb_dsyrk(n, k, 1.0, A2d, lda2, 0.0, Cd2, ldc2, torch.cuda.current_stream())
    got2 = host_cm(Cd2, n, n)
    ref2 = A2.T @ A2
    assert np.all(np.abs(got2[low] - ref2[low]) <= bound(k, np.abs(A2).T @ np.abs(A2))[low])
    assert np.all(got2[~low] == sentinel)


def test_argument_errors(gb):
    f = gb.gb_dgemm
    assert f("X", "N", 1, 1, 1, 1.0, 256, 1, 256, 1, 0.0, 256, 1, None, 0, None, check=False) == -1
    assert f("N", "Q", 1, 1, 1, 1.0, 256, 1, 256, 1, 0.0, 256, 1, None, 0, None, check=False) == -2
    assert f("N", "N", -1, 1, 1, 1.0, 256, 1, 256, 1, 0.0, 256, 1, None, 0, None, check=False) == -3
    assert f("N", "N", 4, 1, 1, 1.0, 256, 3, 256, 1, 0.0, 256, 4, None, 0, None, check=False) == -8
    assert f("N", "N", 4, 1, 1, 1.0, 256, 4, 256, 1, 0.0, 256, 3, None, 0, None, check=False) == -13
    assert f("N", "N", 0, 5, 5, 1.0, None, 1, None, 1, 0.0, None, 1, None, 0, None, check=False) == 0
    assert gb.gb_dsymm("X", 1, 1, 1.0, 256, 1, 256, 1, 0.0, 256, 1, None, 0, None, check=False) == -1
    assert gb.gb_dsyr2k(3, 1, 1.0, 256, 2, 256, 3, 0.0, 256, 3, None, check=False) == -5
    assert gb.gb_dsyrk(3, 2, 1.0, 256, 1, 0.0, 256, 3, None, check=False) == -5
