"""Serving: continuous batching of solve requests on one GPU."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _serve():
    from paper_2301_01868_gb300 import serve
    return serve


def _reqs(max_steps, tol=1e-30):
    S = _serve()
    R = S.Request
    return [R("planar_couette", 9, 16, 8, 0.8, 0.01, tol=tol, arrival=0.0, max_steps=max_steps),
            R("circular_couette", 21, 12, 48, 0.9, 0.01, tol=tol, arrival=0.0, max_steps=max_steps),
            R("planar_poiseuille", 21, 20, 6, 0.7, 0.02, tol=tol, arrival=0.0, max_steps=max_steps),
            R("circular_poiseuille", 9, 16, 40, 1.0, 0.01, tol=tol, arrival=0.01, max_steps=max_steps),
            R("planar_couette", 21, 9, 5, 0.6, 0.005, tol=tol, arrival=0.02, max_steps=max_steps)]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_each_result_same_alone_and_in_the_mix(precision, tol):
    """Every request of a mixed stream ends with the same velocity profile as
    when it is solved alone (step counts fixed by the cap)."""
    S = _serve()
    srv = S.Server(precision=precision, chunk=50, tune=False)
    futs = [srv.submit(r) for r in _reqs(400)]
    srv.run()
    mixed = {f.result()["rid"]: f.result() for f in futs}
    alone, _ = S.serve_serial(_reqs(400), precision=precision, chunk=50)
    for k, a in enumerate(alone):
        m = mixed[k]
        assert m["steps"] == a["steps"] == 400
        u, v = m["Ut2_profile"], a["Ut2_profile"]
        assert np.linalg.norm(u - v) <= tol * np.linalg.norm(v)


def test_admission_respects_the_hbm_budget():
    S = _serve()
    from paper_2301_01868_gb300 import clbm
    reqs = _reqs(200)
    biggest = max(clbm.workspace_bytes(r.lattice, clbm.FP32, r.n1, r.n2) for r in reqs)
    srv = S.Server(precision="fp32", chunk=50, hbm_budget=biggest * 1.5, tune=False)
    for r in reqs:
        srv.submit(r)
    st = srv.run()
    assert st["solves"] == len(reqs)
    # intervals [t_admit, t_done) never overlap beyond the budget
    ev = sorted([(d["t_admit"], 1, d["rid"]) for d in srv.done] + [(d["t_done"], -1, d["rid"]) for d in srv.done])
    need = {r.rid: clbm.workspace_bytes(r.lattice, clbm.FP32, r.n1, r.n2) for r in reqs}
    used = 0
    for t, kind, rid in ev:
        used += kind * need[rid]
        assert used <= biggest * 1.5 + 1


def test_poisson_stream_converges():
    S = _serve()
    reqs = S.poisson_requests(12, rate=50.0, n1_range=(8, 24), n2_range=(8, 48), tol=1e-7,
                              max_steps=40000)
    srv = S.Server(precision="fp32", chunk=100)
    futs = [srv.submit(r) for r in reqs]
    st = srv.run()
    assert st["solves"] == 12 and all(f.done() for f in futs)
    for r, f in zip(reqs, futs):
        d = f.result()
        print("\nSERVE %s D2Q%d %dx%d tau=%.3f: %s after %d steps, residual %.2e"
              % (r.case, r.lattice, r.n1, r.n2, r.tau, d["status"], d["steps"], d["residual"]))
        # D2Q9 on polar grids may diverge (its inner-wall mode); every other
        # request converges
        if not (r.lattice == 9 and r.case.startswith("circular")):
            assert d["status"] == "converged"
    assert st["converged"] >= 10
    assert st["p50_s"] <= st["p99_s"]
