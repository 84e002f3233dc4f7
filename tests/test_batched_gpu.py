"""Batched solver (gb_solve_batched_d): independent problems of mixed sizes
on several streams give the same results as solving each alone (within the
tolerances), and each satisfies the eigenvalue / residual / orthogonality
checks; expected eigenvalues come from the oracle (one-stage Householder
tridiagonalisation + implicit QL), LAPACK only as a secondary check."""
import numpy as np
import pytest

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


def test_batched_mixed_sizes(gb):
    dev = torch.device("cuda")
    g = np.random.default_rng(3)
    sizes = [int(x) for x in g.integers(128, 600, 10)]
    nevs = [n if i % 2 == 0 else n // 4 for i, n in enumerate(sizes)]
    mats = [inputs.band_symmetric(n, n, seed=100 + i, dist="normal") for i, n in enumerate(sizes)]
    A = [torch.from_numpy(np.ascontiguousarray(M.T)).to(dev) for M in mats]
    ev = [torch.zeros(k, dtype=torch.float64, device=dev) for k in nevs]
    Z = [torch.zeros((k, n), dtype=torch.float64, device=dev) for n, k in zip(sizes, nevs)]
    streams = [torch.cuda.Stream() for _ in range(3)]
    es = [torch.cuda.Event(enable_timing=True) for _ in sizes]
    ee = [torch.cuda.Event(enable_timing=True) for _ in sizes]
    wsb = gb.gb_solve_batched_workspace_bytes(sizes, nevs, len(streams))
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    gb.gb_solve_batched_d(sizes, nevs, A, sizes, ev, Z, sizes, ws, wsb, streams, es, ee)
    torch.cuda.synchronize()
    for i, (n, k, M) in enumerate(zip(sizes, nevs, mats)):
        w = ev[i].cpu().numpy()
        Zi = Z[i].cpu().numpy().T
        nrm = np.linalg.norm(M, 2)
        d, e, _, _ = oracle.sytrd(M)
        lam = np.sort(oracle.tridiag_ql(d, e)[0])
        assert np.abs(w - lam[:k]).max() / nrm <= 1e-11
        assert np.abs(w - np.linalg.eigvalsh(M)[:k]).max() / nrm <= 1e-11     # secondary (LAPACK)
        assert np.linalg.norm(M @ Zi - Zi * w) / np.linalg.norm(M) <= 50 * n * U
        assert np.abs(Zi.T @ Zi - np.eye(k)).max() <= 50 * n * U
        assert es[i].elapsed_time(ee[i]) > 0
    # the same problem alone gives the same eigenvalues to rounding
    i = 1
    n, k = sizes[i], nevs[i]
    b = gb.gb_solve_default_nbw(n)
    wsb1 = gb.gb_solve_workspace_bytes(n, k, b)
    ws1 = torch.empty(wsb1, dtype=torch.uint8, device=dev)
    ev1 = torch.zeros(k, dtype=torch.float64, device=dev)
    Z1 = torch.zeros((k, n), dtype=torch.float64, device=dev)
    gb.gb_solve_d(n, k, b, A[i], n, ev1, Z1, n, ws1, wsb1, torch.cuda.current_stream(), 0)
    torch.cuda.synchronize()
    w1, wb = ev1.cpu().numpy(), ev[i].cpu().numpy()
    assert np.abs(w1 - wb).max() / np.linalg.norm(mats[i], 2) <= 1e-11
    # eigenvectors agree up to sign where the spectrum is simple
    Z1n, Zbn = Z1.cpu().numpy().T, Z[i].cpu().numpy().T
    gaps = np.minimum(np.diff(np.concatenate([[-np.inf], w1])), np.diff(np.concatenate([w1, [np.inf]])))
    simple = gaps > 1e-6 * np.linalg.norm(mats[i], 2)
    dots = np.abs(np.sum(Z1n * Zbn, axis=0))
    assert np.abs(dots[simple] - 1.0).max() <= 1e-8


def test_batched_graph_replays_and_reads_the_matrices_at_launch(gb):
    """The batch captured as one CUDA graph (per-problem band widths, three
    branches): a launch solves every problem (eigenvalues against the oracle,
    residual, orthogonality), a second launch gives bit-identical results,
    and after the matrices are shifted in place by c I a third launch returns
    eigenvalues shifted by c: the graph reads A at launch time.  The stream
    form with the same band widths agrees within the tolerances."""
    dev = torch.device("cuda")
    g = np.random.default_rng(9)
    sizes = [int(x) for x in g.integers(100, 520, 7)]
    nevs = [n if i % 3 else n // 3 for i, n in enumerate(sizes)]
    nbw = [[16, 32, 64][i % 3] for i in range(len(sizes))]
    mats = [inputs.band_symmetric(n, n, seed=300 + i, dist="normal") for i, n in enumerate(sizes)]
    A = [torch.from_numpy(np.ascontiguousarray(M.T)).to(dev) for M in mats]
    ev = [torch.zeros(k, dtype=torch.float64, device=dev) for k in nevs]
    Z = [torch.zeros((k, n), dtype=torch.float64, device=dev) for n, k in zip(sizes, nevs)]
    es = [torch.cuda.Event(enable_timing=True) for _ in sizes]
    ee = [torch.cuda.Event(enable_timing=True) for _ in sizes]
    wsb = gb.gb_solve_batched_workspace_bytes_nbw(sizes, nevs, nbw, 3)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    graph = gb.gb_solve_batched_graph_create(sizes, nevs, nbw, A, sizes, ev, Z, sizes, ws, wsb, 3, es, ee)
    try:
        assert gb.gb_solve_batched_graph_nodes(graph) > len(sizes)
        st = torch.cuda.current_stream()
        outs = []
        for _ in range(2):
            gb.gb_solve_batched_graph_launch(graph, st)
            torch.cuda.synchronize()
            outs.append(([e.cpu().numpy().copy() for e in ev], [z.cpu().numpy().copy() for z in Z]))
        for i, (n, k, M) in enumerate(zip(sizes, nevs, mats)):
            w, Zi = outs[0][0][i], outs[0][1][i].T
            nrm = np.linalg.norm(M, 2)
            d, e, _, _ = oracle.sytrd(M)
            lam = np.sort(oracle.tridiag_ql(d, e)[0])
            assert np.abs(w - lam[:k]).max() / nrm <= 1e-11
            assert np.linalg.norm(M @ Zi - Zi * w) / np.linalg.norm(M) <= 50 * n * U
            assert np.abs(Zi.T @ Zi - np.eye(k)).max() <= 50 * n * U
            assert np.array_equal(outs[0][0][i], outs[1][0][i]) and np.array_equal(outs[0][1][i], outs[1][1][i])
            assert es[i].elapsed_time(ee[i]) > 0
        c = 0.75
        for a in A:
            a.diagonal().add_(c)
        gb.gb_solve_batched_graph_launch(graph, st)
        torch.cuda.synchronize()
        for i, M in enumerate(mats):
            w = ev[i].cpu().numpy()
            assert np.abs(w - (outs[0][0][i] + c)).max() / (np.linalg.norm(M, 2) + c) <= 1e-11
    finally:
        assert gb.gb_solve_batched_graph_destroy(graph) == 0
    # the stream form with the same band widths
    for a in A:
        a.diagonal().sub_(c)
    streams = [torch.cuda.Stream() for _ in range(3)]
    gb.gb_solve_batched_nbw_d(sizes, nevs, nbw, A, sizes, ev, Z, sizes, ws, wsb, streams)
    torch.cuda.synchronize()
    for i, M in enumerate(mats):
        assert np.abs(ev[i].cpu().numpy() - outs[0][0][i]).max() / np.linalg.norm(M, 2) <= 1e-11


def test_batched_graph_argument_errors(gb):
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(gb.GbError) as e:
        gb.gb_solve_batched_graph_create([100], [10], [16], [x], [100], [x], [x], [100], None, 0, 1)
    assert e.value.status == -10
    assert gb.gb_solve_batched_graph_launch(None, None, check=False) == -1
    assert gb.gb_solve_batched_graph_nodes(None) == -1


def test_batched_staged_equals_stream_form(gb):
    """The batch stage by stage (all bulge chases in one launch) gives
    bit-identical results to the stream form with the same band widths (the
    same arithmetic per problem), and meets the oracle's eigenvalues and the
    residual/orthogonality bounds; the chase's status word reads 0."""
    dev = torch.device("cuda")
    g = np.random.default_rng(17)
    sizes = [int(x) for x in g.integers(70, 700, 11)]
    nevs = [n if i % 2 == 0 else max(1, n // 5) for i, n in enumerate(sizes)]
    nbw = [[16, 32, 64][i % 3] for i in range(len(sizes))]
    mats = [inputs.band_symmetric(n, n, seed=500 + i, dist="normal") for i, n in enumerate(sizes)]
    A = [torch.from_numpy(np.ascontiguousarray(M.T)).to(dev) for M in mats]
    streams = [torch.cuda.Stream() for _ in range(4)]
    outs = []
    for staged in (False, True):
        ev = [torch.zeros(k, dtype=torch.float64, device=dev) for k in nevs]
        Z = [torch.zeros((k, n), dtype=torch.float64, device=dev) for n, k in zip(sizes, nevs)]
        if staged:
            wsb = gb.gb_solve_batched_staged_workspace_bytes(sizes, nevs, nbw, len(streams))
            ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
            torch.cuda.synchronize()
            gb.gb_solve_batched_staged_d(sizes, nevs, nbw, A, sizes, ev, Z, sizes, ws, wsb, streams)
            assert gb.gb_solve_batched_staged_query(ws, sizes, nevs, nbw, streams) == 0
        else:
            wsb = gb.gb_solve_batched_workspace_bytes_nbw(sizes, nevs, nbw, len(streams))
            ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
            torch.cuda.synchronize()
            gb.gb_solve_batched_nbw_d(sizes, nevs, nbw, A, sizes, ev, Z, sizes, ws, wsb, streams)
        torch.cuda.synchronize()
        outs.append(([e.cpu().numpy() for e in ev], [z.cpu().numpy() for z in Z]))
    for i, (n, k, M) in enumerate(zip(sizes, nevs, mats)):
        assert np.array_equal(outs[0][0][i], outs[1][0][i]) and np.array_equal(outs[0][1][i], outs[1][1][i])
        w, Zi = outs[1][0][i], outs[1][1][i].T
        nrm = np.linalg.norm(M, 2)
        d, e, _, _ = oracle.sytrd(M)
        lam = np.sort(oracle.tridiag_ql(d, e)[0])
        assert np.abs(w - lam[:k]).max() / nrm <= 1e-11
        assert np.linalg.norm(M @ Zi - Zi * w) / np.linalg.norm(M) <= 50 * n * U
        assert np.abs(Zi.T @ Zi - np.eye(k)).max() <= 50 * n * U
