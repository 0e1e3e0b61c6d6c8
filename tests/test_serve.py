"""The continuous-batching relaxation server (space-homogeneous requests).

Runs on the GPU through the C ABI; the oracle is not involved except through
the BKW closed form (an exact solution, not oracle output).
"""
import numpy as np
import pytest
import torch

from paper_1301_4195_gb300 import inputs as I

pytestmark = pytest.mark.gpu
L = 6.0


@pytest.fixture(scope="module")
def srv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1301_4195_gb300 import build
    build.build()
    from paper_1301_4195_gb300 import serve
    return serve


def _req(serve, rid, N, lam, t_end, arrival=0.0, first_id=0):
    f0 = I.random_mixture_cells(N, L, 1, first_id=first_id)[0]
    return serve.Request(rid=rid, N=N, lam=lam, f0=f0, t_end=t_end, arrival=arrival)


def test_result_is_the_same_alone_and_in_the_mix(srv):
    alone = srv.Server(L=L)
    a = alone.run([_req(srv, 0, 16, 1.0, 0.06, first_id=7)])[0].result
    alone.close()
    mix = srv.Server(L=L)
    reqs = [_req(srv, 0, 16, 1.0, 0.06, first_id=7)]
    for i in range(1, 40):  # same class and others, arriving before and while it runs
        N = (12, 16, 24)[i % 3]
        reqs.append(_req(srv, i, N, float(i % 2), 0.02 + 0.01 * (i % 5), arrival=0.0005 * i, first_id=100 + i))
    done = {r.rid: r for r in mix.run(reqs)}
    mix.close()
    assert len(done) == 40
    assert np.array_equal(done[0].result, a)


def test_batched_and_per_class_iterations_agree(srv):
    """One cs_relax_batched per iteration (float classes' convolutions in one
    launch) and one cs_relax per class on its own stream give the same
    states bit for bit."""
    reqs = lambda: [_req(srv, i, (12, 16, 24, 32)[i % 4], float(i % 2), 0.02 + 0.01 * (i % 3),
                         arrival=0.0003 * i, first_id=300 + i) for i in range(12)]
    a = {r.rid: r.result for r in srv.Server(L=L, batched=True).run(reqs())}
    b = {r.rid: r.result for r in srv.Server(L=L, batched=False).run(reqs())}
    assert sorted(a) == sorted(b) == list(range(12))
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_served_result_equals_direct_relaxation(srv):
    from paper_1301_4195_gb300 import api
    s = srv.Server(L=L)
    r = s.run([_req(srv, 0, 12, 0.0, 0.05, first_id=3)])[0]
    s.close()
    h = api.Handle(12, L, 0.0, "fp32")
    f = torch.from_numpy(I.random_mixture_cells(12, L, 1, first_id=3)).cuda()
    h.relax(f, 0.01, r.steps_total)
    assert np.array_equal(f.cpu().numpy()[0], r.result)
    h.close()


def test_maxwell_molecule_request_follows_bkw(srv):
    """lambda = 0 with BKW initial data (K0 = 0.6): the served state tracks the
    closed form K(t) = 1 - (1 - K0) exp(-t/6) to the discretisation error."""
    N, K0, t = 24, 0.6, 0.5
    f0 = I.bkw(N, 8.0, K0)
    s = srv.Server(L=8.0, dt=0.01)
    r = s.run([srv.Request(rid=0, N=N, lam=0.0, f0=f0, t_end=t)])[0]
    s.close()
    K = 1 - (1 - K0) * np.exp(-t / 6)
    ref = I.bkw(N, 8.0, K)
    change = np.abs(ref - f0).max()
    assert np.abs(r.result - ref).max() < 0.02 * change


def test_admission_waits_for_memory_and_evicts_idle_classes(srv):
    s = srv.Server(L=L, radius_fallback=False)
    one = {N: s._class_bytes(N) + 32 * s._cell_bytes(N) for N in (16, 24)}
    s.mem_budget = int(1.01 * max(one.values()))  # room for one class at a time
    assert sum(one.values()) > s.mem_budget
    reqs = [_req(srv, i, 16, 1.0, 0.02, first_id=i) for i in range(3)]
    reqs += [_req(srv, 10 + i, 24, 1.0, 0.02, first_id=20 + i) for i in range(2)]
    done = s.run(reqs)
    assert sorted(r.rid for r in done) == [0, 1, 2, 10, 11]
    # the N = 24 requests could only start once the N = 16 class was evicted
    first24 = min(r.admitted for r in done if r.N == 24)
    last16 = max(r.finished for r in done if r.N == 16)
    assert first24 >= last16
    assert len(s.classes) <= 1
    s.close()


def test_class_without_room_for_its_table_runs_from_the_radius_tables(srv):
    """An N = 32 class whose 0.9 GB table does not fit the budget is admitted
    with the radius tables alone; its result equals a direct relaxation by a
    handle built the same way, bit for bit."""
    from paper_1301_4195_gb300 import api
    s = srv.Server(L=L)
    s.mem_budget = s._class_bytes(32, True) + 64 * s._cell_bytes(32)
    assert s._class_bytes(32) > s.mem_budget
    r = s.run([_req(srv, 0, 32, 1.0, 0.02, first_id=9)])[0]
    assert s.classes[(32, 1.0)].radius
    s.close()
    h = api.Handle(32, L, 1.0, "fp32-radius")
    f = torch.from_numpy(I.random_mixture_cells(32, L, 1, first_id=9)).cuda()
    h.relax(f, 0.01, r.steps_total)
    assert np.array_equal(f.cpu().numpy()[0], r.result)
    h.close()


def test_poisson_run_reports_latencies(srv):
    rng = np.random.default_rng(5)
    t = 0.0
    reqs = []
    for i in range(24):
        t += rng.exponential(0.01)
        N = int(rng.choice([12, 16, 24, 32]))
        reqs.append(_req(srv, i, N, float(rng.integers(0, 2)), float(rng.uniform(0.02, 0.06)), t, i))
    s = srv.Server(L=L)
    done = s.run(reqs)
    s.close()
    lat = [r.latency for r in done]
    assert len(done) == 24 and min(lat) > 0
    assert srv.percentile(lat, 50) <= srv.percentile(lat, 99)
    for r in done:
        assert r.steps_done == r.steps_total and np.isfinite(r.result).all()
