"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no step of the method: it only draws matrices and reflector
sets with the shapes, layouts and value distributions of the workloads.

Workloads (the paper measures FHI-aims Hamiltonians, Sec. 5, which are not
available; these seeded matrices stand in for them):

* band matrices B of band width b with entries iid U[-1, 1] or N(0, 1),
  symmetrised (complex: Hermitian, real and imaginary parts drawn alike);
* the tridiagonal Toeplitz matrix (2, -1) stored with band width b, whose
  eigenpairs have a closed form;
* eigenvector blocks Z with iid N(0, 1/n) entries;
* synthetic reflector sets in the bulge-chase storage layout (see
  ``include/elpa_gb300.h``): v[0] = 1, v[1:len] iid U[-1, 1] / sqrt(len),
  zero padding past len, and tau chosen so that I - tau v v^H is orthogonal
  (unitary): tau = (1 - exp(i theta)) / ||v||^2 with theta = pi in the real
  case and theta ~ U[pi/2, 3pi/2] in the complex case.  These have the same
  layout, lengths and tau range (Re tau in [0, 2]) as a bulge chase's output
  and stand in for it at sizes where a CPU bulge chase would take minutes.
"""
import numpy as np


def _rng(seed):
    return np.random.default_rng(np.random.SeedSequence([0x1811_01277 & 0xFFFFFFFF, int(seed)]))


def band_symmetric(n, b, seed, dist="uniform", cplx=False):
    """Dense n x n symmetric (Hermitian) matrix with b super-diagonals."""
    g = _rng(seed)
    draw = (lambda: g.uniform(-1.0, 1.0, (n, n))) if dist == "uniform" else (lambda: g.standard_normal((n, n)))
    A = draw()
    if cplx:
        A = A + 1j * draw()
    A = 0.5 * (A + A.conj().T)
    i, j = np.indices((n, n))
    A[np.abs(i - j) > b] = 0.0
    return np.asfortranarray(A)


def toeplitz_band(n, b, diag=2.0, off=-1.0, cplx=False):
    """The tridiagonal Toeplitz matrix (diag, off) held as a band-b matrix."""
    A = np.zeros((n, n), dtype=np.complex128 if cplx else np.float64, order="F")
    A[np.arange(n), np.arange(n)] = diag
    A[np.arange(1, n), np.arange(n - 1)] = off
    A[np.arange(n - 1), np.arange(1, n)] = off
    return A


def z_gaussian(n, nev, seed, cplx=False, ldz=None):
    """n x nev block with iid N(0, 1/n) entries (column-major, leading dim ldz)."""
    g = _rng(seed + 7919)
    ldz = n if ldz is None else ldz
    Z = g.standard_normal((ldz, nev))
    if cplx:
        Z = (Z + 1j * g.standard_normal((ldz, nev))) / np.sqrt(2.0)
    Z /= np.sqrt(n)
    return np.asfortranarray(Z)


def hh_layout(n, b):
    """Per-sweep reflector counts nk(s) = ceil((n-s)/b), s = 1..n-1, and the
    index of each sweep's first reflector."""
    s = np.arange(1, n, dtype=np.int64)
    nk = (n - s + b - 1) // b
    first = np.concatenate([[0], np.cumsum(nk)[:-1]]) if n > 1 else np.zeros(0, np.int64)
    return nk, first


def hh_lengths(n, b):
    """len(s, k) = min(b, n - s - k b) for every stored reflector, in storage order."""
    nk, first = hh_layout(n, b)
    total = int(nk.sum()) if nk.size else 0
    lens = np.empty(total, dtype=np.int64)
    sweep = np.repeat(np.arange(1, n, dtype=np.int64), nk)
    k = np.arange(total, dtype=np.int64) - np.repeat(first, nk)
    lens[:] = np.minimum(b, n - sweep - k * b)
    return lens


def synthetic_reflectors(n, b, seed, cplx=False):
    """Random orthogonal (unitary) reflectors in the bulge-chase layout.

    Returns (hh_v, hh_tau) with hh_v of shape (count * b,)."""
    g = _rng(seed + 104729)
    lens = hh_lengths(n, b)
    cnt = lens.size
    col = np.arange(b)[None, :]
    mask = col < lens[:, None]
    scale = 1.0 / np.sqrt(np.maximum(lens, 1))[:, None]
    V = g.uniform(-1.0, 1.0, (cnt, b)) * scale
    if cplx:
        V = (V + 1j * g.uniform(-1.0, 1.0, (cnt, b)) * scale) / np.sqrt(2.0)
    V = np.where(mask, V, 0.0)
    V[:, 0] = 1.0
    nrm2 = np.sum(np.abs(V) ** 2, axis=1)
    if cplx:
        theta = g.uniform(0.5 * np.pi, 1.5 * np.pi, cnt)
        tau = (1.0 - np.exp(1j * theta)) / nrm2
    else:
        tau = 2.0 / nrm2
    return np.ascontiguousarray(V.reshape(-1)), np.ascontiguousarray(tau)


def clustered_spectrum(n, seed, lo_exp=-3.0, hi=50.0, cluster_frac=0.1, cluster_size=8, width=1e-8):
    """Eigenvalues in [-hi, hi]: magnitudes 10^U[lo_exp, log10(hi)] with random
    signs, and cluster_frac of them in clusters of cluster_size spread over
    `width` around centres drawn the same way.  Sorted ascending."""
    g = _rng(seed + 31337)
    ncl = int(round(n * cluster_frac / cluster_size))
    nfree = n - ncl * cluster_size

    def draw(k):
        mag = 10.0 ** g.uniform(lo_exp, np.log10(hi), k)
        return mag * np.where(g.uniform(size=k) < 0.5, -1.0, 1.0)

    lam = list(draw(nfree))
    for c in draw(ncl):
        lam.extend(c + np.linspace(-0.5 * width, 0.5 * width, cluster_size))
    return np.sort(np.array(lam[:n]))


def gapped_uniform_spectrum(n, seed, cluster_frac=0.1, cluster_size=8, gap=1e-6):
    """Eigenvalues uniform in [-1, 1], with cluster_frac of them in groups of
    cluster_size whose consecutive members are `gap` apart (eigenvector
    clusters of condition ~1/gap).  Sorted ascending."""
    g = _rng(seed + 16180)
    ncl = int(round(n * cluster_frac / cluster_size))
    nfree = n - ncl * cluster_size
    lam = list(g.uniform(-1.0, 1.0, nfree))
    span = (cluster_size - 1) * gap
    for c in g.uniform(-1.0, 1.0 - span, ncl):
        lam.extend(c + gap * np.arange(cluster_size))
    return np.sort(np.array(lam[:n]))


def symmetric_with_spectrum(lam, seed, cplx=False):
    """A = Q diag(lam) Q^H with Q Haar-distributed (QR of a Gaussian matrix,
    phases fixed by R's diagonal); exactly symmetric (Hermitian)."""
    n = len(lam)
    g = _rng(seed + 271828)
    G = g.standard_normal((n, n))
    if cplx:
        G = G + 1j * g.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    dg = np.diag(R)
    Q = Q * (dg / np.abs(dg))[None, :]
    A = (Q * lam[None, :]) @ Q.conj().T
    return np.asfortranarray(0.5 * (A + A.conj().T))
