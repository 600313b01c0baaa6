"""The request server (hz_server_*) on the GPU.

- Every request served in a mix (several admitted at once, their restart
  cycles overlapping on the device) returns bit for bit the solution and the
  iteration count of the same problem solved alone with hz_solve: each
  request runs the same kernels and deterministic reductions on its own
  hierarchy and stream.
- A failing request (non-finite medium) is reported and the others finish.
- A request above the whole budget is refused at submission.
- A request that runs out of iterations reports HZ_ERR_NOT_CONVERGED with its
  last iterate, equal to the solo one.
- The asynchronous single-solve calls give the blocking solve's result.
- Grouping: queued requests of one problem (only the source differs) are
  solved together as one multi-RHS solve, in groups of a power of two; each
  member's iteration count is the oracle's +-1 and its solution agrees with
  the oracle's at the same tolerance (1e-5 mixed); a request of another
  problem in between stays alone and equals its solo solve bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from pairs import medium  # noqa: E402

REQS = [
    dict(dim=2, n=513, seed=3, kind="layered", levels=5, patch="rb", intergrid="leveldep", alpha=0.1, layer=10),
    dict(dim=2, n=65, seed=0, kind="layered", levels=3, patch="rb", intergrid="leveldep", alpha=0.25, layer=8),
    dict(dim=2, n=129, seed=0, kind="homogeneous", levels=4, patch="plus", intergrid="leveldep", alpha=0.25),
    dict(dim=3, n=17, seed=1, kind="layered", levels=3, patch="element", intergrid="linear", alpha=0.5, layer=3),
    dict(dim=2, n=33, seed=2, kind="layered", levels=3, patch="element", intergrid="cubic", alpha=0.25),
    dict(dim=2, n=65, seed=4, kind="layered", levels=3, patch="plus", intergrid="leveldep", alpha=0.25,
         precision="fp64"),
    dict(dim=3, n=9, seed=5, kind="layered", levels=2, patch="plus", intergrid="leveldep", alpha=0.25),
    dict(dim=2, n=257, seed=6, kind="layered", levels=4, patch="rb", intergrid="leveldep", alpha=0.1, layer=6),
]


def _problem(r):
    import workloads
    h, omega, kappa, gamma = medium(r["dim"], r["n"], r["seed"], r.get("layer", 0), r.get("ppw", 10.0), r["kind"])
    n, dim = r["n"], r["dim"]
    src = tuple([(n - 1) // 2 + (r["seed"] % 3)] * dim)
    q = workloads.point_source((n,) * dim, src, h).ravel()
    opts = dict(patch=r["patch"], intergrid=r["intergrid"], precision=r.get("precision", "mixed"), tol=1e-7,
                max_iter=r.get("max_iter", 2000))
    return kappa, gamma, omega, q, opts


def _solo(r):
    from paper_2511_16808_gb300.solver import HelmholtzSolver
    kappa, gamma, omega, q, opts = _problem(r)
    s = HelmholtzSolver(r["dim"], [r["n"]] * r["dim"], kappa, omega, gamma, r["alpha"], r["levels"], **opts)
    p, info = s.solve(q, np.zeros_like(q))
    s.close()
    return p, info


def _submit(srv, r):
    kappa, gamma, omega, q, opts = _problem(r)
    return srv.submit(r["dim"], r["n"], kappa, omega, q, gamma=gamma, alpha=r["alpha"], levels=r["levels"], **opts)


def test_served_mix_equals_solo():
    from paper_2511_16808_gb300.serve import Server
    with Server(max_active=4) as srv:
        tickets = [_submit(srv, r) for r in REQS]
        results = [srv.wait(t, timeout=300) for t in tickets]
        st = srv.stats()
    assert st["done"] == len(REQS) and st["failed"] == 0 and st["bytes_in_use"] == 0
    assert 0 < st["peak_bytes"] <= st["budget"]
    for r, (p, d) in zip(REQS, results):
        assert d["state"] == "done" and d["status"] == "HZ_OK", d
        p1, info1 = _solo(r)
        assert d["iters"] == info1.iters, (r, d["iters"], info1.iters)
        assert np.array_equal(p, p1), r
        assert d["t_submit"] <= d["t_admit"] <= d["t_start"] <= d["t_done"]
    # the big first request was still solving while later ones ran
    spans = [(d["t_start"], d["t_done"]) for _, d in results]
    overlaps = sum(1 for i in range(len(spans)) for j in range(i + 1, len(spans))
                   if spans[i][0] < spans[j][1] and spans[j][0] < spans[i][1])
    assert overlaps >= 1, spans


def test_failing_request_is_isolated():
    from paper_2511_16808_gb300.serve import Server
    good = [REQS[1], REQS[2]]
    with Server(max_active=2) as srv:
        t0 = _submit(srv, good[0])
        kappa, gamma, omega, q, opts = _problem(REQS[4])
        kappa = kappa.copy()
        kappa[5] = np.nan
        tb = srv.submit(2, REQS[4]["n"], kappa, omega, q, gamma=gamma, alpha=0.25, levels=3, **opts)
        t1 = _submit(srv, good[1])
        pb, db = srv.wait(tb, timeout=300)
        res = [srv.wait(t, timeout=300) for t in (t0, t1)]
        st = srv.stats()
    assert db["state"] == "failed" and db["status"] == "HZ_ERR_INVALID_ARG" and "kappa" in db["message"]
    assert st["failed"] == 1 and st["done"] == 2 and st["bytes_in_use"] == 0
    for r, (p, d) in zip(good, res):
        p1, info1 = _solo(r)
        assert d["status"] == "HZ_OK" and d["iters"] == info1.iters and np.array_equal(p, p1)


def test_oversize_request_refused():
    from paper_2511_16808_gb300 import hz
    from paper_2511_16808_gb300.serve import Server
    with Server(hbm_budget=1 << 20) as srv:
        with pytest.raises(hz.HzError) as e:
            _submit(srv, REQS[1])
        assert e.value.status == 2                      # HZ_ERR_OOM
        assert srv.stats()["queued"] == 0


def test_not_converged_request_keeps_last_iterate():
    from paper_2511_16808_gb300.serve import Server
    r = dict(REQS[1], max_iter=7)
    with Server() as srv:
        p, d = srv.wait(_submit(srv, r), timeout=300)
    p1, info1 = _solo(r)
    assert d["state"] == "done" and d["status"] == "HZ_ERR_NOT_CONVERGED" and not d["converged"]
    assert d["iters"] == info1.iters == 7
    assert np.array_equal(p, p1) and np.any(p != 0)


def test_async_solve_matches_blocking():
    from paper_2511_16808_gb300 import hz
    from paper_2511_16808_gb300.solver import HelmholtzSolver
    r = REQS[2]
    kappa, gamma, omega, q, opts = _problem(r)
    s = HelmholtzSolver(r["dim"], [r["n"]] * r["dim"], kappa, omega, gamma, r["alpha"], r["levels"], **opts)
    p_block, info = s.solve(torch.tensor(q, device="cuda"))
    qd = torch.tensor(q, device="cuda")
    hz.hz_solve_begin(s.ctx, qd)
    steps = 0
    while not hz.hz_solve_step(s.ctx, block=False):
        steps += 1
    p_async = torch.empty_like(qd)
    ok, info2 = hz.hz_solve_end(s.ctx, p_async)
    assert ok and info2.iters == info.iters and steps >= 1
    assert torch.equal(p_async, p_block)
    with pytest.raises(hz.HzError):
        hz.hz_solve_step(s.ctx)                      # nothing in flight any more
    s.close()


def test_async_solve_host_buffers():
    from paper_2511_16808_gb300 import hz
    from paper_2511_16808_gb300.solver import HelmholtzSolver
    r = REQS[1]
    kappa, gamma, omega, q, opts = _problem(r)
    s = HelmholtzSolver(r["dim"], [r["n"]] * r["dim"], kappa, omega, gamma, r["alpha"], r["levels"], **opts)
    p_block, info = s.solve(q, np.zeros_like(q))
    hz.hz_solve_begin(s.ctx, q)                       # host source, staged by the library
    while not hz.hz_solve_step(s.ctx, block=True):
        pass
    p_async = np.zeros_like(q)
    ok, info2 = hz.hz_solve_end(s.ctx, p_async)      # host output
    assert ok and info2.iters == info.iters and np.array_equal(p_async, p_block)
    s.close()


def test_many_small_requests():
    """A burst of small 2D / 3D requests through few slots: all finish, the
    slots and bytes are all returned, and sampled results equal solo solves."""
    from paper_2511_16808_gb300.serve import Server
    small = [REQS[1], REQS[3], REQS[4], REQS[6]]
    reqs = [dict(small[i % 4], seed=10 + i) for i in range(24)]
    with Server(max_active=6, setup_threads=3) as srv:
        tickets = [_submit(srv, r) for r in reqs]
        res = [srv.wait(t, timeout=300) for t in tickets]
        st = srv.stats()
    assert st["done"] == len(reqs) and st["failed"] == 0 and st["bytes_in_use"] == 0
    assert st["kernel_launches"] > 0
    for i in (0, 7, 13, 22):
        p, d = res[i]
        p1, info1 = _solo(reqs[i])
        assert d["status"] == "HZ_OK" and d["iters"] == info1.iters and np.array_equal(p, p1)


def test_grouped_requests_share_one_solve():
    from oracle import solver as osolver
    from pairs import check_agreement
    from paper_2511_16808_gb300 import hz
    from paper_2511_16808_gb300.serve import Server
    import workloads
    g = dict(dim=2, n=129, seed=7, kind="layered", levels=4, patch="rb", intergrid="leveldep", alpha=0.1, layer=6)
    kappa, gamma, omega, _, opts = _problem(g)
    n = g["n"]
    h = 1.0 / (n - 1)
    rng = np.random.default_rng(21)
    srcs = [tuple(int(v) for v in rng.integers(10, n - 10, size=2)) for _ in range(6)]
    qs = [workloads.point_source((n, n), sd, h).ravel() for sd in srcs]
    with pytest.raises(hz.HzError):
        Server(group_max=3)
    # one slot: the first (unrelated) request holds it while the rest queue up
    with Server(max_active=1, setup_threads=1, group_max=8) as srv:
        t_block = _submit(srv, REQS[0])
        tickets = []
        for k, q in enumerate(qs):
            tickets.append(srv.submit(2, n, kappa, omega, q, gamma=gamma, alpha=g["alpha"], levels=g["levels"],
                                      **opts))
            if k == 2:
                t_other = _submit(srv, REQS[1])          # another problem, in between
        res = [srv.wait(t, timeout=600) for t in tickets]
        p_other, d_other = srv.wait(t_other, timeout=600)
        p_block, d_block = srv.wait(t_block, timeout=600)
        st = srv.stats()
    assert st["done"] == len(qs) + 2 and st["failed"] == 0 and st["bytes_in_use"] == 0
    # six requests of one problem: a group of four, then one of two
    assert st["groups"] == 2 and st["grouped"] == 6, st
    assert sorted(d["group_size"] for _, d in res) == [2, 2, 4, 4, 4, 4]
    assert d_other["group_size"] == 1 and d_block["group_size"] == 1
    p1, info1 = _solo(REQS[1])
    assert d_other["iters"] == info1.iters and np.array_equal(p_other, p1)
    orc = osolver.Problem((n, n), h, kappa, omega, gamma, g["alpha"], g["levels"], g["patch"], g["intergrid"])
    for q, (p, d) in zip(qs, res):
        assert d["state"] == "done" and d["status"] == "HZ_OK", d
        p_o, info_o = orc.solve(q.copy(), tol=1e-7)
        assert abs(d["iters"] - info_o.iters) <= 1, (d["iters"], info_o.iters)
        check_agreement(p, p_o, None, "mixed", f"grouped request, group of {d['group_size']}")
    # members of a group start and finish together
    by_size = {}
    for _, d in res:
        by_size.setdefault(d["group_size"], set()).add((d["t_start"], d["t_done"]))
    assert all(len(v) == 1 for v in by_size.values()), by_size
