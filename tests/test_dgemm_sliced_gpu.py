"""FP64 products on the bf16 tensor cores (gb_dgemm_sliced, gb_dsymm_sliced,
gb_dsyr2k_sliced, gb_dsyrk_sliced: exact digit slicing) against numpy's
float64 products: ragged shapes, padded leading dimensions, split-K shapes,
rows of very different magnitudes, the triangle / beta = 0 contracts, and
exactness where the FP64 product is exact (small integers)."""
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
    r, c = X.shape
    ld = ld or max(r, 1)
    buf = np.full((max(c, 1), ld), np.nan)
    buf[:c, :r] = X.T
    return torch.from_numpy(buf).cuda(), ld


def host_cm(T, rows, cols):
    return T.cpu().numpy()[:cols, :rows].T


def ws(nbytes):
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device="cuda"), nbytes


def ref_hp(opA, opB, alpha, beta, C0):
    """alpha opA opB + beta C0 in extended precision (np.longdouble: 64- or
    113-bit significand), so that the reference's own rounding does not
    enter the comparison."""
    L = np.longdouble
    return L(alpha) * (opA.astype(L) @ opB.astype(L)) + L(beta) * C0.astype(L)


def bound(opA, opB, alpha, beta, C0):
    """|C - exact| for the sliced product: k 2^-53 times the row maxima of
    op(A) and the column maxima of op(B) (the scales the digits are cut
    against), with a factor 4, plus the final FP64 roundings of the result
    and of the beta C term."""
    k = opA.shape[1]
    amax = np.abs(opA).max(axis=1, initial=0.0)[:, None]
    bmax = np.abs(opB).max(axis=0, initial=0.0)[None, :]
    prod = np.abs(alpha) * (np.abs(opA) @ np.abs(opB))
    return 4 * (k + 2) * U * abs(alpha) * amax * bmax + 4 * U * (prod + abs(beta) * np.abs(C0)) + 1e-300


def err(got, ref):
    return np.abs(got.astype(np.longdouble) - ref).astype(np.float64)


SHAPES = [(1, 1, 1), (37, 29, 13), (64, 64, 64), (65, 63, 200), (200, 77, 131), (513, 64, 1000),
          (64, 64, 5000), (20, 300, 2500), (130, 129, 0)]


@pytest.mark.parametrize("m,n,k", SHAPES)
@pytest.mark.parametrize("ta", "NT")
@pytest.mark.parametrize("tb", "NT")
def test_dgemm_sliced(gb, m, n, k, ta, tb):
    g = np.random.default_rng(m * 1000 + n * 10 + k + 5)
    A = g.uniform(-1, 1, (k, m) if ta == "T" else (m, k))
    B = g.uniform(-1, 1, (n, k) if tb == "T" else (k, n))
    C0 = g.uniform(-1, 1, (m, n))
    alpha, beta = 0.75, -1.25
    Ad, lda = dev_cm(A, A.shape[0] + 3)
    Bd, ldb = dev_cm(B, B.shape[0] + 1)
    Cd, ldc = dev_cm(C0, m + 2)
    w, wsb = ws(gb.gb_dgemm_sliced_workspace_bytes(m, n, k))
    gb.gb_dgemm_sliced(ta, tb, m, n, k, alpha, Ad, lda, Bd, ldb, beta, Cd, ldc, w, wsb, torch.cuda.current_stream())
    opA = A.T if ta == "T" else A
    opB = B.T if tb == "T" else B
    ref = ref_hp(opA, opB, alpha, beta, C0)
    got = host_cm(Cd, m, n)
    assert np.all(err(got, ref) <= bound(opA, opB, alpha, beta, C0))
    assert np.all(np.isnan(Cd.cpu().numpy()[:n, m:ldc]))   # padding rows untouched


def test_sliced_exact_on_small_integers(gb):
    """Integer entries up to 127 in magnitude: every digit but the first is
    zero, the level-0 sums are exact integers, so the result must equal the
    (exact) FP64 product bit for bit, beta = 0 not reading C."""
    m, n, k = 150, 90, 1000
    g = np.random.default_rng(11)
    A = g.integers(-127, 128, (m, k)).astype(np.float64)
    B = g.integers(-127, 128, (k, n)).astype(np.float64)
    Ad, lda = dev_cm(A)
    Bd, ldb = dev_cm(B)
    Cd = torch.full((n, m), float("nan"), dtype=torch.float64, device="cuda")
    w, wsb = ws(gb.gb_dgemm_sliced_workspace_bytes(m, n, k))
    gb.gb_dgemm_sliced("N", "N", m, n, k, 1.0, Ad, lda, Bd, ldb, 0.0, Cd, m, w, wsb, torch.cuda.current_stream())
    assert np.array_equal(host_cm(Cd, m, n), A @ B)


def test_sliced_rows_of_different_magnitude(gb):
    """Row and column scales spread over 2^-60 .. 2^60 (each row is scaled
    separately, so the relative accuracy per entry follows its own row)."""
    m, n, k = 96, 80, 700
    g = np.random.default_rng(12)
    ra = 2.0 ** g.integers(-60, 61, m)
    cb = 2.0 ** g.integers(-60, 61, n)
    A = g.standard_normal((m, k)) * ra[:, None]
    B = g.standard_normal((k, n)) * cb[None, :]
    Ad, lda = dev_cm(A)
    Bd, ldb = dev_cm(B)
    Cd, ldc = dev_cm(np.zeros((m, n)))
    w, wsb = ws(gb.gb_dgemm_sliced_workspace_bytes(m, n, k))
    gb.gb_dgemm_sliced("N", "N", m, n, k, 1.0, Ad, lda, Bd, ldb, 0.0, Cd, ldc, w, wsb, torch.cuda.current_stream())
    ref = ref_hp(A, B, 1.0, 0.0, np.zeros((m, n)))
    assert np.all(err(host_cm(Cd, m, n), ref) <= bound(A, B, 1.0, 0.0, np.zeros((m, n))))


@pytest.mark.parametrize("side", "LR")
@pytest.mark.parametrize("m,n", [(1, 1), (45, 17), (64, 64), (130, 70), (700, 64), (64, 700)])
def test_dsymm_sliced_reads_lower_only(gb, side, m, n):
    g = np.random.default_rng(m + 7 * n + 1)
    s = m if side == "L" else n
    S = g.uniform(-1, 1, (s, s))
    S = S + S.T
    S_lower = np.tril(S) + np.triu(np.full((s, s), np.nan), 1)
    B = g.uniform(-1, 1, (m, n))
    C0 = g.uniform(-1, 1, (m, n))
    Sd, lds = dev_cm(S_lower, s + 1)
    Bd, ldb = dev_cm(B, m + 3)
    Cd, ldc = dev_cm(C0, m)
    w, wsb = ws(gb.gb_dsymm_sliced_workspace_bytes(side, m, n))
    gb.gb_dsymm_sliced(side, m, n, -0.5, Sd, lds, Bd, ldb, 2.0, Cd, ldc, w, wsb, torch.cuda.current_stream())
    opA, opB = (S, B) if side == "L" else (B, S)
    ref = ref_hp(opA, opB, -0.5, 2.0, C0)
    assert np.all(err(host_cm(Cd, m, n), ref) <= bound(opA, opB, -0.5, 2.0, C0))


@pytest.mark.parametrize("n,k", [(1, 1), (50, 3), (64, 64), (129, 64), (300, 200), (1000, 64)])
def test_dsyr2k_and_dsyrk_sliced_lower_triangle(gb, n, k):
    g = np.random.default_rng(n * 31 + k + 2)
    A, B = g.uniform(-1, 1, (n, k)), g.uniform(-1, 1, (n, k))
    C0 = g.uniform(-1, 1, (n, n))
    sentinel = 12345.0
    C0u = np.tril(C0) + np.triu(np.full((n, n), sentinel), 1)
    Ad, lda = dev_cm(A, n + 1)
    Bd, ldb = dev_cm(B, n + 2)
    Cd, ldc = dev_cm(C0u, n + 1)
    w, wsb = ws(gb.gb_dsyr2k_sliced_workspace_bytes(n, k))
    gb.gb_dsyr2k_sliced(n, k, -1.0, Ad, lda, Bd, ldb, 1.0, Cd, ldc, w, wsb, torch.cuda.current_stream())
    got = host_cm(Cd, n, n)
    AB, BA = np.hstack([A, B]), np.hstack([B, A])
    ref = ref_hp(AB, BA.T, -1.0, 1.0, C0)
    low = np.tril(np.ones((n, n), dtype=bool))
    assert np.all((err(got, ref) <= bound(AB, BA.T, -1.0, 1.0, C0))[low])
    assert np.all(got[~low] == sentinel)
    A2 = g.uniform(-1, 1, (k, n))
    A2d, lda2 = dev_cm(A2, k + 3)
    Cd2, ldc2 = dev_cm(np.tril(np.full((n, n), np.nan)) + np.triu(np.full((n, n), sentinel), 1), n)
    w2, wsb2 = ws(gb.gb_dsyrk_sliced_workspace_bytes(n, k))
    gb.gb_dsyrk_sliced(n, k, 1.0, A2d, lda2, 0.0, Cd2, ldc2, w2, wsb2, torch.cuda.current_stream())
    got2 = host_cm(Cd2, n, n)
    ref2 = ref_hp(A2.T, A2, 1.0, 0.0, np.zeros((n, n)))
    assert np.all((err(got2, ref2) <= bound(A2.T, A2, 1.0, 0.0, np.zeros((n, n))))[low])
    assert np.all(got2[~low] == sentinel)


def test_sliced_argument_errors(gb):
    f = gb.gb_dgemm_sliced
    assert f("X", "N", 1, 1, 1, 1.0, 256, 1, 256, 1, 0.0, 256, 1, 256, 1 << 30, None, check=False) == -1
    assert f("N", "N", 4, 1, 1, 1.0, 256, 3, 256, 1, 0.0, 256, 4, 256, 1 << 30, None, check=False) == -8
    assert f("N", "N", 4, 1, 1, 1.0, 256, 4, 256, 1, 0.0, 256, 4, 128, 1 << 30, None, check=False) == -14
    assert f("N", "N", 4, 1, 1, 1.0, 256, 4, 256, 1, 0.0, 256, 4, 256, 16, None, check=False) == -15


@pytest.mark.parametrize("k", [128, 1024, 16384])
def test_sliced_syrk_long_sums_of_one_sign(gb, k):
    """A^T A with long k: the diagonal sums k squares (all of one sign), the
    hardest case for exact level accumulation."""
    n = 256
    g = np.random.default_rng(k)
    A = g.uniform(-0.5, 0.5, (k, n))
    Ad, lda = dev_cm(A)
    Cd, ldc = dev_cm(np.zeros((n, n)))
    w, wsb = ws(gb.gb_dsyrk_sliced_workspace_bytes(n, k))
    gb.gb_dsyrk_sliced(n, k, 1.0, Ad, lda, 0.0, Cd, ldc, w, wsb, torch.cuda.current_stream())
    got = host_cm(Cd, n, n)
    ref = ref_hp(A.T, A, 1.0, 0.0, np.zeros((n, n)))
    low = np.tril(np.ones((n, n), dtype=bool))
    e = err(got, ref)
    b = bound(A.T, A, 1.0, 0.0, np.zeros((n, n)))
    print(f"k={k} diag max err {np.diag(e).max():.3e} (bound {np.diag(b).min():.3e}), "
          f"offdiag max err {e[np.tril(low, -1)].max() if n > 1 else 0:.3e}")
    assert np.all((e <= b)[low])


# ---- complex forms ---------------------------------------------------------

def zdev_cm(X, ld=None):
    """Column-major complex128 device copy (interleaved), leading dimension ld,
    padding rows NaN."""
    r, c = X.shape
    ld = ld or max(r, 1)
    buf = np.full((max(c, 1), ld), np.nan + 1j * np.nan)
    buf[:c, :r] = X.T
    return torch.from_numpy(buf).cuda(), ld


def zbound(opA, opB, alpha, beta, C0):
    """Complex analogue of bound(): the expanded real product has 2k terms,
    scaled by the maxima of |Re| and |Im| of the rows and columns."""
    k = opA.shape[1]
    amax = np.maximum(np.abs(opA.real), np.abs(opA.imag)).max(axis=1, initial=0.0)[:, None]
    bmax = np.maximum(np.abs(opB.real), np.abs(opB.imag)).max(axis=0, initial=0.0)[None, :]
    prod = abs(alpha) * (np.abs(opA) @ np.abs(opB))
    return 8 * (2 * k + 2) * U * abs(alpha) * amax * bmax + 4 * U * (prod + abs(beta) * np.abs(C0)) + 1e-300


def zref(opA, opB, alpha, beta, C0):
    L = np.clongdouble
    return L(alpha) * (opA.astype(L) @ opB.astype(L)) + L(beta) * C0.astype(L)


def zerr(got, ref):
    return np.abs(got.astype(np.clongdouble) - ref).astype(np.float64)


def crandn(g, shape):
    return g.uniform(-1, 1, shape) + 1j * g.uniform(-1, 1, shape)


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (37, 29, 13), (64, 64, 64), (130, 70, 200), (64, 300, 2500)])
@pytest.mark.parametrize("ta", "NC")
def test_zgemm_sliced(gb, m, n, k, ta):
    g = np.random.default_rng(m * 7 + n * 3 + k)
    A = crandn(g, (k, m) if ta == "C" else (m, k))
    B = crandn(g, (k, n))
    C0 = crandn(g, (m, n))
    Ad, lda = zdev_cm(A, A.shape[0] + 2)
    Bd, ldb = zdev_cm(B, k + 1)
    Cd, ldc = zdev_cm(C0, m + 3)
    w, wsb = ws(gb.gb_zgemm_sliced_workspace_bytes(m, n, k))
    gb.gb_zgemm_sliced(ta, m, n, k, -0.5, Ad, lda, Bd, ldb, 1.5, Cd, ldc, w, wsb, torch.cuda.current_stream())
    opA = A.conj().T if ta == "C" else A
    got = Cd.cpu().numpy()[:n, :m].T
    assert np.all(zerr(got, zref(opA, B, -0.5, 1.5, C0)) <= zbound(opA, B, -0.5, 1.5, C0))
    assert np.all(np.isnan(Cd.cpu().numpy()[:n, m:ldc].real))


@pytest.mark.parametrize("m,n", [(1, 1), (45, 17), (130, 64), (600, 64)])
def test_zhemm_sliced_reads_lower_only(gb, m, n):
    g = np.random.default_rng(m + n)
    S = crandn(g, (m, m))
    S = S + S.conj().T                                    # Hermitian, real diagonal
    S_low = np.tril(S) + np.triu(np.full((m, m), np.nan + 1j * np.nan), 1)
    S_low[np.diag_indices(m)] += 1j * 7.0                 # the diagonal's imaginary part must be ignored
    B = crandn(g, (m, n))
    C0 = crandn(g, (m, n))
    Sd, lds = zdev_cm(S_low, m + 1)
    Bd, ldb = zdev_cm(B, m)
    Cd, ldc = zdev_cm(C0, m + 2)
    w, wsb = ws(gb.gb_zhemm_sliced_workspace_bytes(m, n))
    gb.gb_zhemm_sliced(m, n, 1.0, Sd, lds, Bd, ldb, 0.0, Cd, ldc, w, wsb, torch.cuda.current_stream())
    got = Cd.cpu().numpy()[:n, :m].T
    assert np.all(zerr(got, zref(S, B, 1.0, 0.0, C0)) <= zbound(S, B, 1.0, 0.0, C0))


@pytest.mark.parametrize("n,k", [(1, 1), (50, 3), (129, 64), (500, 64)])
def test_zher2k_sliced_lower_triangle(gb, n, k):
    g = np.random.default_rng(n * 5 + k)
    X, Y = crandn(g, (n, k)), crandn(g, (n, k))
    C0 = crandn(g, (n, n))
    C0 = C0 + C0.conj().T
    sentinel = 12345.0 + 0j
    C0u = np.tril(C0) + np.triu(np.full((n, n), sentinel), 1)
    Xd, ldx = zdev_cm(X, n + 1)
    Yd, ldy = zdev_cm(Y, n)
    Cd, ldc = zdev_cm(C0u, n + 2)
    w, wsb = ws(gb.gb_zher2k_sliced_workspace_bytes(n, k))
    gb.gb_zher2k_sliced(n, k, -1.0, Xd, ldx, Yd, ldy, 1.0, Cd, ldc, w, wsb, torch.cuda.current_stream())
    got = Cd.cpu().numpy()[:n, :n].T
    XY, YX = np.hstack([X, Y]), np.hstack([Y, X])
    ref = zref(XY, YX.conj().T, -1.0, 1.0, C0)
    low = np.tril(np.ones((n, n), dtype=bool))
    assert np.all((zerr(got, ref) <= zbound(XY, YX.conj().T, -1.0, 1.0, C0))[low])
    assert np.all(got.imag[np.diag_indices(n)] == 0.0)
    assert np.all(got[~low] == sentinel)


def fp32_bound(opA, opB, alpha, beta, C0):
    """|C - exact| for gb_dgemm_fp32split: (3 + 128) 2^-24 |alpha| sum_k
    |a_ik| |b_kj| (inputs rounded to FP32, dropped parts, FP32 sums over 128
    terms) plus the FP64 roundings of the result and of the beta C term."""
    prod = np.abs(alpha) * (np.abs(opA) @ np.abs(opB))
    return (3 + 128) * 2.0 ** -24 * prod + 4 * U * (prod + abs(beta) * np.abs(C0)) + 1e-300


@pytest.mark.parametrize("m,n,k", [(37, 29, 13), (65, 63, 200), (513, 64, 1000), (64, 64, 5000), (130, 129, 0)])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T")])
def test_dgemm_fp32split(gb, m, n, k, ta, tb):
    """The FP32 product: within the FP32 bound of every entry, with entries
    of very different magnitude in one row (per-entry exponents: a
    Householder-like column with a unit leading entry and 1e-3 others, rows
    scaled by 2^+-40), and clearly less accurate than the FP64 product (so
    the FP32 path is the one that ran)."""
    g = np.random.default_rng(m + 7 * n + 11 * k)
    A = g.uniform(-1, 1, (k, m) if ta == "T" else (m, k))
    B = g.uniform(-1, 1, (n, k) if tb == "T" else (k, n))
    if k:
        opB_view = B.T if tb == "T" else B
        opB_view[1:, 0] *= 1e-3                       # column 0 of op(B): 1, then small entries
        opA_view = A.T if ta == "T" else A
        opA_view[: m // 3] *= 2.0 ** 40
        opA_view[m // 3: 2 * m // 3] *= 2.0 ** -40
    C0 = g.uniform(-1, 1, (m, n))
    alpha, beta = 0.75, -1.25
    Ad, lda = dev_cm(A, A.shape[0] + 3)
    Bd, ldb = dev_cm(B, B.shape[0] + 1)
    Cd, ldc = dev_cm(C0, m + 2)
    w, wsb = ws(gb.gb_dgemm_sliced_workspace_bytes(m, n, k))
    gb.gb_dgemm_fp32split(ta, tb, m, n, k, alpha, Ad, lda, Bd, ldb, beta, Cd, ldc, w, wsb,
                          torch.cuda.current_stream())
    opA = A.T if ta == "T" else A
    opB = B.T if tb == "T" else B
    ref = ref_hp(opA, opB, alpha, beta, C0)
    got = host_cm(Cd, m, n)
    e = err(got, ref)
    assert np.all(e <= fp32_bound(opA, opB, alpha, beta, C0))
    if k >= 100:
        rel = e / (np.abs(alpha) * (np.abs(opA) @ np.abs(opB)))
        assert np.median(rel) > 1e-12                  # FP32, not FP64
        assert np.median(rel) < 2.0 ** -20
    assert np.all(np.isnan(Cd.cpu().numpy()[:n, m:ldc]))
