"""The serving loop on the GPU: a request's solution does not depend on which
requests it was batched with or which other solves ran beside it on another
stream, factors are cached and evicted within the memory budget, and every
solution meets the tolerance by the oracle's own residual."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import operator

pytestmark = pytest.mark.gpu

N, OMEGA, GAMMA, B = 47, 5 * math.pi, 5, 4
KEYS = 3


def requests(serving):
    out = []
    rid = 0
    for rnd in range(3):
        for v in range(KEYS):
            P = W.small_problem(2, N, OMEGA, GAMMA, B, "layered", nrhs=1 + (rid % 2), seed=100 + rid)
            c = W.layered_velocity(N, 40 + v, dim=2)
            out.append(serving.Request(("layered", v), c, OMEGA, GAMMA, B, P.f, tol=1e-6, precision="c128",
                                       rid=rid))
            rid += 1
    return out


def run(serving, reqs, **kw):
    srv = serving.Server(start=False, **kw)
    futs = [srv.submit(r) for r in reqs]
    srv.start()
    res = [f.result(timeout=300) for f in futs]
    stats, used, budget = dict(srv.stats), srv.used_bytes, srv.memory_budget
    srv.close()
    return res, stats, used, budget


def test_batched_concurrent_solutions_match_alone():
    from paper_1504_04058_gb300 import asp_footprint_bytes, serving
    reqs = requests(serving)
    alone, st_a, _, _ = run(serving, reqs, memory_budget=1 << 34, workers=1, max_rhs=8, batching=False)
    assert st_a["solves"] == len(reqs) and st_a["factorizations"] == KEYS
    assert all(r.batched_with == rq.nrhs for r, rq in zip(alone, reqs))

    probe = serving.Server(1 << 34, workers=1, max_rhs=8, start=False)
    fp = asp_footprint_bytes(probe._params(reqs[0]))
    probe.close()
    mixed, st_m, used, budget = run(serving, reqs, memory_budget=int(2.5 * fp), workers=2, max_rhs=8)
    # one batch per key, two keys resident at a time: the third evicts one
    assert st_m["solves"] == KEYS and st_m["factorizations"] == KEYS
    assert st_m["evictions"] >= 1 and used <= budget
    assert all(r.batched_with == sum(q.nrhs for q in reqs if q.key() == rq.key())
               for r, rq in zip(mixed, reqs))

    for rq, a, m in zip(reqs, alone, mixed):
        assert a.rid == m.rid == rq.rid
        assert a.iterations == m.iterations, (rq.rid, a.iterations, m.iterations)
        err = np.linalg.norm(m.u - a.u) / np.linalg.norm(a.u)
        assert err <= 1e-9, (rq.rid, err)
        r = rq.f - operator.apply_A(2, N, OMEGA, rq.c, GAMMA, 20.0, m.u)
        for k in range(rq.nrhs):
            rel = np.linalg.norm(r[..., k]) / np.linalg.norm(rq.f[..., k])
            assert rel <= rq.tol, (rq.rid, k, rel)
            assert m.rel_res_true[k] <= rq.tol

    lat = serving.percentiles([m.latency_s for m in mixed])
    assert 0 < lat["p50"] <= lat["p99"] < 300


def test_concurrent_handles_of_different_sizes():
    """Two host threads drive handles of different widths on their own streams
    (as the serving workers do); every kernel's shared-memory limit only grows,
    so neither thread's launches can fail, and results equal the serial ones."""
    import threading

    import torch

    import paper_1504_04058_gb300 as asp
    probs = [W.small_problem(2, 47, 6 * math.pi, 6, 4, "lens", nrhs=12, seed=1),
             W.small_problem(2, 95, 12 * math.pi, 12, 4, "layered", nrhs=16, seed=2)]
    handles, ref = [], []
    for P in probs:
        prm = asp.make_params(P.n, P.omega, P.pml, P.b, precision="c64", max_rhs=P.nrhs)
        h = asp.asp_setup(P.c, prm)
        h.factor()
        handles.append(h)
        ref.append(h.apply_preconditioner(torch.from_numpy(P.f).cuda()).cpu().numpy())
    errors = []

    def drive(k):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                f = torch.from_numpy(probs[k].f).cuda()
                for _ in range(30):
                    z = handles[k].apply_preconditioner(f, stream=s)
                s.synchronize()
                errors.append((k, float(np.abs(z.cpu().numpy() - ref[k]).max())))
        except Exception as ex:  # reported below
            errors.append((k, repr(ex)))

    ts = [threading.Thread(target=drive, args=(k,)) for k in range(2)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert sorted(e[0] for e in errors) == [0, 1], errors
    assert all(isinstance(e[1], float) and e[1] == 0.0 for e in errors), errors
