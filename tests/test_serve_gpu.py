"""Continuous-batching service (paper_1811_01277_gb300.serve): requests that
run concurrently in the mix give the same results as each run alone (within
the tolerances), every result passes the LAPACK checks, and the HBM budget
limits how many requests are admitted at once."""
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
    reqs, mats = [], []
    rid = 0
    for k, n in enumerate([256, 384, 512]):
        A = inputs.band_symmetric(n, n, seed=40 + k, cplx=True)
        E = inputs.band_symmetric(n, n, seed=80 + k, cplx=True)
        E /= np.linalg.norm(E, 2)
        for j in range(2):        # the system re-submitted with a perturbed matrix
            M = A + 1e-3 * j * E
            mats.append(M)
            Ad = torch.from_numpy(np.ascontiguousarray(M.T)).to(dev)   # column-major data
            reqs.append(serve.Request(rid=rid, A=Ad, nev=int(0.3 * n), arrival=0.0))
            rid += 1
    return reqs, mats


def check(M, w, Z):
    n, nev = M.shape[0], len(w)
    nrm = np.linalg.norm(M, 2)
    assert np.abs(w - np.linalg.eigvalsh(M)[:nev]).max() / nrm <= 1e-11
    assert np.linalg.norm(M @ Z - Z * w) / np.linalg.norm(M) <= 50 * n * U
    assert np.abs(Z.conj().T @ Z - np.eye(nev)).max() <= 50 * n * U


def test_mix_equals_alone(serve):
    reqs, mats = make_requests(serve)
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
        check(M, wm, Zm)
        assert np.abs(wa - wm).max() / np.linalg.norm(M, 2) <= 1e-11
        gaps = np.minimum(np.diff(np.concatenate([[-np.inf], wa])), np.diff(np.concatenate([wa, [np.inf]])))
        simple = gaps > 1e-6 * np.linalg.norm(M, 2)
        assert np.abs(np.abs(np.sum(Za.conj() * Zm, axis=0))[simple] - 1.0).max() <= 1e-8
    s = serve.latency_summary(done)
    assert s["requests"] == len(reqs) and s["p99_ms"] >= s["p50_ms"] > 0


def test_hbm_budget_limits_admission(serve):
    reqs, mats = make_requests(serve)
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
        check(mats[r.rid], r.ev.cpu().numpy(), r.Z.cpu().numpy().T)
