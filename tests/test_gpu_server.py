"""GPU tests of the request server: admission by a memory budget, potentials
held on the device until release, results equal to the batched solver's and
within the oracle tolerances, and its error paths."""
import threading

import numpy as np
import pytest
import torch

import oracle as O
from solve_checks import check_truth, stop_tol
from paper_2605_30267_gb300 import binding as B
from paper_2605_30267_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


def request(seed, n, m, d, eps, kind="sqeuclid", scale=True):
    g = np.random.default_rng(seed)
    X = g.random((n, d)).astype(np.float32)
    Y = g.random((m, d)).astype(np.float32)
    if kind == "cosine":
        X = W.unit_gaussian_points(g, n, d)
        Y = W.unit_gaussian_points(g, m, d)
    a, b = W.dirichlet1(g, n), W.dirichlet1(g, m)
    return {"X": X, "Y": Y, "a": a, "b": b, "eps": eps, "kind": kind, "scale": scale}


def submit(srv, r, **kw):
    pr = B.problem_host(r["a"], r["b"], X=r["X"], Y=r["Y"], kind=r["kind"],
                        scale_to_max=r["scale"])
    return srv.submit(pr, B.default_params(eps=r["eps"], tol=1e-6, **kw))


def batch_reference(reqs):
    ctx = B.Context(0)
    try:
        structs, params, fs, gs, keep = [], [], [], [], []
        for r in reqs:
            X, Y = torch.from_numpy(r["X"]).to(DEV), torch.from_numpy(r["Y"]).to(DEV)
            a, b = torch.from_numpy(r["a"]).to(DEV), torch.from_numpy(r["b"]).to(DEV)
            structs.append(B.problem_points(X, Y, r["kind"], a, b, r["scale"]))
            params.append(B.default_params(eps=r["eps"], tol=1e-6))
            fs.append(torch.empty(len(r["a"]), dtype=torch.float64, device=DEV))
            gs.append(torch.empty(len(r["b"]), dtype=torch.float64, device=DEV))
        res = ctx.accsink_solve_batch(structs, params, fs, gs)
        torch.cuda.synchronize()
        return [f.cpu().numpy() for f in fs], [g.cpu().numpy() for g in gs], res
    finally:
        ctx.close()


def mix():
    return [request(1, 64, 80, 2, 1e-2), request(2, 300, 257, 5, 1e-3),
            request(3, 129, 700, 16, 5e-2), request(4, 513, 400, 64, 1e-2),
            request(5, 40, 35, 30, 2e-2, kind="cosine", scale=False),
            request(6, 1, 7, 3, 5e-2), request(7, 700, 900, 3, 1e-3)]


def test_server_results_equal_the_batch_and_the_oracle():
    reqs = mix()
    srv = B.Server(0, 4 << 30)
    try:
        tickets = [submit(srv, r) for r in reqs]
        out = []
        for t in tickets:
            rc, res, lat = srv.wait(t, 120000)
            assert rc == B.OK and res.status == 0, (rc, res.status)
            assert lat > 0
            assert srv.poll(t) == B.REQ_DONE
            out.append(srv.copy_potentials(t))
        st = srv.stats()
        assert st["solved"] == len(reqs) and st["failed"] == 0 and st["queued"] == 0
        assert st["resident_bytes"] > 0
        fref, gref, rres = batch_reference(reqs)
        for k, (f, g) in enumerate(out):
            np.testing.assert_array_equal(f, fref[k])
            np.testing.assert_array_equal(g, gref[k])
        for t in tickets:
            srv.release(t)
        assert srv.stats()["resident_bytes"] == 0
        # two against the oracle
        for k in (0, 4):
            r = reqs[k]
            cost = O.Cost(X=r["X"], Y=r["Y"], kind=r["kind"], scale_to_max=r["scale"])
            ref = O.solve(cost, r["a"], r["b"], r["eps"], stop_tol(1e-6))
            f, g = out[k]
            sh = g.mean() - ref["g"].mean()
            if rres[k].sinkhorn_steps == ref["sinkhorn_steps"]:
                assert max(np.abs(g - sh - ref["g"]).max(),
                           np.abs(f + sh - ref["f"]).max()) <= 1e-3 * r["eps"]
            ev = O.evaluate(cost, r["eps"], ref["a"], ref["b"], f, g)
            check_truth(ev, 1e-6)
    finally:
        srv.close()


def test_budget_rejects_oversized_requests_and_waits_for_releases():
    small = request(11, 100, 120, 3, 1e-2)
    big = request(12, 3000, 3000, 3, 1e-2)       # 72 MB of cost: over the budget
    srv = B.Server(0, 24 << 20)
    try:
        t_big = submit(srv, big)
        t1 = submit(srv, small)
        rc, res, _ = srv.wait(t_big, 60000)
        assert rc == B.ERR_BUDGET and srv.poll(t_big) == B.REQ_FAILED
        rc, res, _ = srv.wait(t1, 60000)
        assert rc == B.OK
        srv.release(t_big)
        # hold potentials: more requests still fit next to them (small)
        t2 = submit(srv, small)
        assert srv.wait(t2, 60000)[0] == B.OK
        st = srv.stats()
        assert st["peak_bytes"] <= st["budget_bytes"]
        srv.release(t1)
        srv.release(t2)
    finally:
        srv.close()


def test_tickets_and_arguments_are_checked():
    srv = B.Server(0, 1 << 30)
    try:
        with pytest.raises(B.AccsinkError):
            srv.release(12345)
        with pytest.raises(B.AccsinkError):
            srv.poll(12345)
        r = request(21, 20, 30, 3, 1e-2)
        pr = B.problem_host(r["a"], r["b"], X=r["X"], Y=r["Y"])
        bad = B.default_params(eps=-1.0)
        with pytest.raises(B.AccsinkError) as e:
            srv.submit(pr, bad)
        assert e.value.code == B.ERR_INVALID_ARG
        t = submit(srv, r)
        assert srv.wait(t, 60000)[0] == B.OK
        f_dev, g_dev = srv.potentials_dev(t)
        assert f_dev and g_dev
        srv.release(t)
        with pytest.raises(B.AccsinkError):
            srv.release(t)
    finally:
        srv.close()


def test_concurrent_clients():
    reqs = [request(100 + k, 50 + 13 * k, 60 + 7 * k, 2 + k % 5, 1e-2) for k in range(24)]
    srv = B.Server(0, 2 << 30)
    results = {}

    def client(idx):
        for k in idx:
            t = submit(srv, reqs[k])
            rc, res, lat = srv.wait(t, 120000)
            results[k] = (rc, srv.copy_potentials(t) if rc == B.OK else None)
            srv.release(t)

    try:
        th = [threading.Thread(target=client, args=(list(range(j, 24, 4)),)) for j in range(4)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        assert sorted(results) == list(range(24))
        assert all(results[k][0] == B.OK for k in results)
        fref, gref, _ = batch_reference(reqs)
        for k in range(24):
            np.testing.assert_array_equal(results[k][1][0], fref[k])
            np.testing.assert_array_equal(results[k][1][1], gref[k])
        assert srv.stats()["resident_bytes"] == 0
    finally:
        srv.close()


def test_requests_finish_with_their_own_problem():
    """A batch hands each problem back as soon as the kernel finishes it: small
    requests submitted with a large one complete (and may be released) while
    the large one still runs; results and the accounting stay exact."""
    import time
    big = request(200, 3000, 2800, 3, 1e-3)
    smalls = [request(201 + k, 48 + 5 * k, 40 + 3 * k, 2, 5e-2) for k in range(8)]
    blocker = request(199, 2000, 2000, 3, 1e-3)
    srv = B.Server(0, 4 << 30)
    try:
        # while the blocker runs, the large and the small requests queue up,
        # so they share the next batch
        t0 = submit(srv, blocker)
        time.sleep(0.002)
        tb = submit(srv, big)
        ts = [submit(srv, r) for r in smalls]
        got, before_big = {}, 0
        for k, t in enumerate(ts):
            rc, res, lat = srv.wait(t, 120000)
            assert rc == B.OK, (rc, srv.last_error())
            if srv.poll(tb) == B.REQ_RUNNING:
                before_big += 1
            got[k] = srv.copy_potentials(t)
            srv.release(t)               # possibly while the batch still runs
        rc, res, lat = srv.wait(tb, 300000)
        assert rc == B.OK, (rc, srv.last_error())
        fbig, gbig = srv.copy_potentials(tb)
        srv.release(tb)
        assert srv.wait(t0, 300000)[0] == B.OK
        srv.release(t0)
        time.sleep(0.05)
        st = srv.stats()
        assert st["solved"] == 10 and st["failed"] == 0, st
        assert st["resident_bytes"] == 0 and st["queued"] == 0, st
        fref, gref, _ = batch_reference(smalls + [big])
        for k in range(8):
            np.testing.assert_array_equal(got[k][0], fref[k])
            np.testing.assert_array_equal(got[k][1], gref[k])
        np.testing.assert_array_equal(fbig, fref[8])
        np.testing.assert_array_equal(gbig, gref[8])
        assert before_big >= 1, before_big
    finally:
        srv.close()


def test_group_limit_runs_requests_alone_with_the_same_results():
    """With a group limit of one cost entry every request runs as a batch of
    its own; the potentials are those of the one joint batch, bit for bit
    (a problem's arithmetic does not depend on the group it runs in)."""
    reqs = mix()
    srv = B.Server(0, 4 << 30)
    try:
        with pytest.raises(B.AccsinkError):
            srv.set_limits(-1)
        srv.set_limits(1)
        tickets = [submit(srv, r) for r in reqs]
        out = []
        for t in tickets:
            rc, res, lat = srv.wait(t, 120000)
            assert rc == B.OK and res.status == 0, (rc, res.status)
            out.append(srv.copy_potentials(t))
            srv.release(t)
        st = srv.stats()
        assert st["batches"] == len(reqs) and st["solved"] == len(reqs)
        fref, gref, _ = batch_reference(reqs)
        for k, (f, g) in enumerate(out):
            np.testing.assert_array_equal(f, fref[k])
            np.testing.assert_array_equal(g, gref[k])
    finally:
        srv.close()
