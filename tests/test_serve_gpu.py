"""Continuous-batching service (paper_1811_01277_gb300.serve): requests that
run concurrently in the mix give the same results as each run alone (within
the tolerances), every result matches its prescribed spectrum, and the HBM
budget limits how many requests are admitted at once.

Each system is A = Q diag(lam) Q^H and its re-submissions A + 1e-3 j E with
E = Q diag(mu) Q^H (same Q, ||E||_2 = 1), so the expected eigenvalues are
lam + 1e-3 j mu in closed form (LAPACK only as a secondary check)."""
import numpy as np
import pytest

from paper_1811_01277_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def serve():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_01277_gb300 as m
    from paper_1811_01277_gb300 import build
    from paper_1811_01277_gb300 import serve as s
    build.build()
    m.load()
    return s


def make_requests(serve):
    dev = torch.device("cuda")
    reqs, mats, spectra = [], [], []
    rid = 0
    for k, n in enumerate([256, 384, 512]):
        g = np.random.default_rng(40 + k)
        lam = g.uniform(-1.0, 1.0, n)
        mu = g.uniform(-1.0, 1.0, n)
        mu[np.argmax(np.abs(mu))] = 1.0
        A = inputs.symmetric_with_spectrum(lam, seed=40 + k, cplx=True)
        E = inputs.symmetric_with_spectrum(mu, seed=40 + k, cplx=True)   # same Q
        for j in range(2):        # the system re-submitted with a perturbed matrix
            M = A + 1e-3 * j * E
            mats.append(M)
            spectra.append(np.sort(lam + 1e-3 * j * mu))
            Ad = torch.from_numpy(np.ascontiguousarray(M.T)).to(dev)   # column-major data
            reqs.append(serve.Request(rid=rid, A=Ad, nev=int(0.3 * n), arrival=0.0))
            rid += 1
    return reqs, (mats, spectra)


def check(M, w, Z, lam):
    n, nev = M.shape[0], len(w)
    nrm = np.linalg.norm(M, 2)
    assert np.abs(w - lam[:nev]).max() / nrm <= 1e-11
    assert np.abs(w - np.linalg.eigvalsh(M)[:nev]).max() / nrm <= 1e-11   # secondary (LAPACK)
    assert np.linalg.norm(M @ Z - Z * w) / np.linalg.norm(M) <= 50 * n * U
    assert np.abs(Z.conj().T @ Z - np.eye(nev)).max() <= 50 * n * U


def test_mix_equals_alone(serve):
    reqs, (mats, spectra) = make_requests(serve)
    srv = serve.EigenServer(slots=3)
    done = srv.run(reqs)
    assert len(done) == len(reqs) and all(r.status == 0 for r in done)
    mix = {r.rid: (r.ev.cpu().numpy(), r.Z.cpu().numpy().T) for r in done}
    alone_reqs, _ = make_requests(serve)
    for r in alone_reqs:
        srv1 = serve.EigenServer(slots=1)
        (d,) = srv1.run([r])
        wa, Za = d.ev.cpu().numpy(), d.Z.cpu().numpy().T
        wm, Zm = mix[r.rid]
        M = mats[r.rid]
        check(M, wm, Zm, spectra[r.rid])
        assert np.abs(wa - wm).max() / np.linalg.norm(M, 2) <= 1e-11
        gaps = np.minimum(np.diff(np.concatenate([[-np.inf], wa])), np.diff(np.concatenate([wa, [np.inf]])))
        simple = gaps > 1e-6 * np.linalg.norm(M, 2)
        assert np.abs(np.abs(np.sum(Za.conj() * Zm, axis=0))[simple] - 1.0).max() <= 1e-8
    s = serve.latency_summary(done)
    assert s["requests"] == len(reqs) and s["p99_ms"] >= s["p50_ms"] > 0


def test_hbm_budget_limits_admission(serve):
    reqs, (mats, spectra) = make_requests(serve)
    # any two requests together exceed the smallest footprint: one at a time
    # (a request larger than the budget is still admitted when nothing runs)
    need = min(serve.request_bytes(r.n, r.nev, True, 32) for r in reqs)
    srv = serve.EigenServer(slots=4, hbm_budget_bytes=need)
    peak = 0
    orig = srv._admit

    def admit():
        nonlocal peak
        orig()
        peak = max(peak, len(srv.active))
    srv._admit = admit
    done = srv.run(reqs)
    assert peak == 1
    for r in done:
        check(mats[r.rid], r.ev.cpu().numpy(), r.Z.cpu().numpy().T, spectra[r.rid])


def test_matrix_built_on_the_device_right_before_submit(serve):
    """A_{k+1} = A_k + 1e-3 E computed on the current stream (not synchronised)
    just before submit: the served result equals the one-at-a-time result, and
    the source tensors may be dropped right after submit."""
    dev = torch.device("cuda")
    n = 384
    g = np.random.default_rng(7)
    lam = g.uniform(-1.0, 1.0, n)
    mu = g.uniform(-1.0, 1.0, n)
    mu[np.argmax(np.abs(mu))] = 1.0
    A0 = torch.from_numpy(np.ascontiguousarray(inputs.symmetric_with_spectrum(lam, seed=7, cplx=True).T)).to(dev)
    E = torch.from_numpy(np.ascontiguousarray(inputs.symmetric_with_spectrum(mu, seed=7, cplx=True).T)).to(dev)
    torch.cuda.synchronize()
    srv = serve.EigenServer(slots=2)
    reqs = []
    for j in range(1, 4):
        big = torch.randn(4096, 4096, dtype=torch.float64, device=dev)   # keeps the stream busy
        big = big @ big
        Aj = A0 + (1e-3 * j) * E                                         # written on the current stream
        reqs.append(serve.Request(rid=j, A=Aj, nev=100, arrival=0.0))
        del big
    done = srv.run(reqs)
    assert all(r.status == 0 for r in done)
    for r in done:
        lamj = np.sort(lam + 1e-3 * r.rid * mu)
        M = (A0 + (1e-3 * r.rid) * E).cpu().numpy().T
        check(M, r.ev.cpu().numpy(), r.Z.cpu().numpy().T, lamj)


def test_stage_batching_equals_one_call_solves(serve):
    """With stage batching the bulge chases of the requests whose first
    stage has finished run in one launch; every result is bit-identical to
    the one-call solve of the same request, and matches its spectrum."""
    import paper_1811_01277_gb300 as m
    reqs, (mats, spectra) = make_requests(serve)
    srv = serve.EigenServer(slots=6, stage_batching=True)
    done = srv.run(reqs)
    assert len(done) == len(reqs) and all(r.status == 0 for r in done)
    assert max(srv.chase_sizes) >= 2 and sum(srv.chase_sizes) == len(reqs)   # chases were merged
    dev = torch.device("cuda")
    for r in done:
        n, nev = r.n, r.nev
        wsb = m.gb_solve_workspace_bytes_z(n, nev, r.nbw)
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        ev = torch.empty(nev, dtype=torch.float64, device=dev)
        Z = torch.empty((nev, n), dtype=torch.complex128, device=dev)
        st = torch.cuda.current_stream()
        m.gb_solve_z(n, nev, r.nbw, r.A, n, ev, Z, n, ws, wsb, st, 0)
        assert m.gb_solve_query_z(ws, n, nev, r.nbw, st) == 0
        assert torch.equal(ev, r.ev) and torch.equal(Z, r.Z)
        check(mats[r.rid], r.ev.cpu().numpy(), r.Z.cpu().numpy().T, spectra[r.rid])


def test_stage_api_real_equals_one_call(serve):
    """gb_solve_stage_front / _chase_batched / _back on three real problems
    (their chases in one launch) give the same bits as gb_solve_d."""
    import paper_1811_01277_gb300 as m
    dev = torch.device("cuda")
    st = torch.cuda.current_stream()
    probs = []
    for k, (n, nev, nbw) in enumerate([(300, 300, 32), (520, 100, 64), (200, 60, 16)]):
        M = inputs.band_symmetric(n, n, seed=70 + k, dist="normal")
        A = torch.from_numpy(np.ascontiguousarray(M.T)).to(dev)
        wsb = m.gb_solve_workspace_bytes(n, nev, nbw)
        probs.append((n, nev, nbw, A, wsb, torch.empty(wsb, dtype=torch.uint8, device=dev)))
    for n, nev, nbw, A, wsb, ws in probs:
        m.gb_solve_stage_front(0, n, nev, nbw, A, n, ws, wsb, st)
    tb = m.gb_solve_stage_table_bytes(len(probs))
    table = torch.empty(tb, dtype=torch.uint8, device=dev)
    m.gb_solve_stage_chase_batched(0, [p[0] for p in probs], [p[1] for p in probs], [p[2] for p in probs],
                                   [p[5] for p in probs], table, tb, st)
    outs = []
    for n, nev, nbw, A, wsb, ws in probs:
        ev = torch.empty(nev, dtype=torch.float64, device=dev)
        Z = torch.empty((nev, n), dtype=torch.float64, device=dev)
        m.gb_solve_stage_back(0, n, nev, nbw, ev, Z, n, ws, wsb, st)
        outs.append((ev, Z))
    assert m.gb_trans_ev_query(table, 256, st) == 0
    for (n, nev, nbw, A, wsb, ws), (ev, Z) in zip(probs, outs):
        ws1 = torch.empty(wsb, dtype=torch.uint8, device=dev)
        ev1 = torch.empty(nev, dtype=torch.float64, device=dev)
        Z1 = torch.empty((nev, n), dtype=torch.float64, device=dev)
        m.gb_solve_d(n, nev, nbw, A, n, ev1, Z1, n, ws1, wsb, st, 0)
        torch.cuda.synchronize()
        assert torch.equal(ev, ev1) and torch.equal(Z, Z1)
